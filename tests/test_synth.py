"""The seeded input generator: the solar-irradiance table integrates to the
solar constant, the counter-based normals are standard normal and depend
only on (seed, pixel, band), and the configs have the stated shapes."""
import math

import numpy as np

import synth


def test_solar_constant():
    lam = np.linspace(100.0, 1e5, 2_000_000)
    total = np.trapezoid(synth.scenes.solar_irradiance_fine(lam), lam)
    # sigma T^4 (R_sun / AU)^2 for T = 5778 K, minus the tails beyond 0.1-100 um
    expect = 5.670374419e-8 * 5778.0 ** 4 * (6.957e8 / 1.495978707e11) ** 2
    assert abs(total - expect) / expect < 2e-3
    assert abs(expect - 1366.8) < 1.0


def test_splitmix64_reference_values():
    # SplitMix64 from state 0: the first outputs of the published generator
    z = synth.splitmix64(np.uint64(0))
    assert int(z) == 0xE220A8397B1DCDAF
    z2 = synth.splitmix64(np.uint64(0x9E3779B97F4A7C15))
    assert int(z2) == 0x6E789E6AA1B965F4


def test_noise_normals_statistics_and_counter_property():
    z = synth.noise_normals(3, np.arange(2000), 284)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    sub = synth.noise_normals(3, np.array([17, 1999]), 284)
    assert np.array_equal(sub, z[[17, 1999]])
    assert not np.array_equal(synth.noise_normals(4, [17], 284), sub[:1])


def test_config_shapes():
    t = synth.make_tables()
    assert t.n_bands == 284 and t.n_wv == 16 and t.n_endm == 3
    assert abs(t.wavelength_nm[0] - 380) < 1e-4 and abs(t.wavelength_nm[-1] - 2510) < 1e-3
    assert np.all((t.tau_up > 0) & (t.tau_up <= 1)) and np.all(t.tau_down <= t.tau_up + 1e-7)
    tr = synth.make_config1_truth()
    assert tr.n_pix == 4096 and (tr.kind == 1).sum() == 205
    assert np.allclose(tr.x_surf.sum(1), 1)
    a = tr.single[tr.kind == 1, 0]
    T = tr.single[tr.kind == 1, 1]
    assert a.min() >= 1e-4 and a.max() <= 0.5 and T.min() >= 500 and T.max() <= 1500
    t5 = synth.make_tables(n_bands=285)
    assert t5.n_bands == 285
    assert synth.block_mean_shape(1240, 2048) == (103, 170)


def test_config2_fronts_small():
    tr = synth.make_config2_truth(width=124, height=204)
    nf = (tr.kind == 2).sum()
    assert nf == round(0.02 * 124 * 204)
    m = tr.mix[tr.kind == 2]
    assert m[:, 0].min() >= 600 and m[:, 0].max() <= 1400
    assert m[:, 1].min() >= 50 and m[:, 1].max() <= 300
    assert np.all(m[:, 4] == 1.0)


def test_config3_dims():
    dims = synth.make_config3_scenes()
    assert len(dims) == 32 and dims[0][:2] == (256, 256) and dims[-1][:2] == (1240, 4096)
    assert all(w % 8 == 0 and h % 8 == 0 for w, h, _, _ in dims)
    assert all(0.001 <= f <= 0.2 for _, _, f, _ in dims)
