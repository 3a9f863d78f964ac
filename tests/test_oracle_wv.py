"""Pins of the oracle's input-side steps. The water-vapour presolve (Sec.
2.5): the depth table against flat-surface radiance formed here in closed
form, the block median and the quantisation against an independent numpy
restatement (single precision where the decision is an integer), recovery
of known per-block bins from the forward model, ragged edge blocks and empty
blocks. The thermal injection (Eq. inject) against the forward model."""
import numpy as np
import pytest

import oracle
import synth
from scenes import NOISE_ABS, NOISE_REL

LAMS = oracle.WV_LAMBDAS


def _bands(t):
    lam = np.asarray(t.wavelength_nm, np.float64)
    return [int(np.argmin(np.abs(lam - l))) for l in LAMS]


def _flat_radiance(t, bins, rho=0.3):
    """L_b = E0_b cos(theta_s) / pi rho tau_down_b tau_up_b: a flat surface,
    no path radiance, no fire."""
    A = np.asarray(t.solar_irr, np.float64) * t.cos_sza / np.pi
    td = np.asarray(t.tau_down, np.float64)[bins]
    tu = np.asarray(t.tau_up, np.float64)[bins]
    return (A * rho * td * tu).astype(np.float32)


def _numpy_presolve(t, L, width, height, block):
    """Independent restatement: depth per pixel (continuum by interpolation,
    float32), lower median per block, fractional index between bracketing
    table depths, nearest bin."""
    lo, c, hi = _bands(t)
    lam = np.asarray(t.wavelength_nm, np.float64)
    cf = np.float32((lam[c] - lam[lo]) / (lam[hi] - lam[lo]))
    Lf = L.astype(np.float32)
    d = Lf[:, hi] - Lf[:, lo]                    # rounded to single, as in the oracle
    cont32 = (d.astype(np.float64) * np.float64(cf) + Lf[:, lo]).astype(np.float32)   # fmaf
    with np.errstate(all="ignore"):
        D = np.where(np.isfinite(Lf[:, [lo, c, hi]]).all(1) & (cont32 > 0),
                     np.float32(1) - Lf[:, c] / cont32, np.float32(np.nan)).astype(np.float32)
    Dj = oracle.wv_depth_table(t)
    bins = np.empty(width * height, np.uint16)
    img = D.reshape(height, width)
    for by in range(0, height, block):
        for bx in range(0, width, block):
            v = img[by:by + block, bx:bx + block].ravel()
            v = np.sort(v[np.isfinite(v)])
            if v.size == 0:
                b = 0xFFFF
            else:
                med = v[(v.size - 1) // 2]
                J = Dj.size
                if not med > Dj[0]:
                    f = np.float32(0)
                elif not med < Dj[-1]:
                    f = np.float32(J - 1)
                else:
                    j = int(np.argmax(med < Dj[1:]))
                    f = np.float32(j) + (med - Dj[j]) / (Dj[j + 1] - Dj[j])
                b = int(min(max(np.floor(f + np.float32(0.5)), 0), J - 1))
            blk = np.zeros((height, width), bool)
            blk[by:by + block, bx:bx + block] = True
            bins[blk.ravel()] = b
    return bins, D


def test_depth_table_is_the_flat_surface_depth_of_each_bin():
    t = synth.make_tables()
    L = _flat_radiance(t, np.arange(t.n_wv))
    lo, c, hi = _bands(t)
    lam = np.asarray(t.wavelength_nm, np.float64)
    f = (lam[c] - lam[lo]) / (lam[hi] - lam[lo])
    Lw = L.astype(np.float64)
    D = 1 - Lw[:, c] / (Lw[:, lo] + (Lw[:, hi] - Lw[:, lo]) * f)
    assert np.allclose(oracle.wv_depth_table(t), D, rtol=1e-6)
    assert np.all(np.diff(oracle.wv_depth_table(t)) > 0)          # deeper with more water


def test_flat_surface_blocks_recover_their_bins():
    """A flat surface per 12 x 12 block, one bin per block: every block gets
    its own bin back."""
    t = synth.make_tables()
    W, H = 48, 48                               # 4 x 4 blocks
    bins_blk = np.arange(16).reshape(4, 4) % t.n_wv
    bins = np.repeat(np.repeat(bins_blk, 12, 0), 12, 1).ravel()
    L = _flat_radiance(t, bins)
    got, _ = oracle.wv_presolve(t, L, W, H)
    assert np.array_equal(got, bins)


def test_median_and_quantisation_match_an_independent_restatement():
    t = synth.make_tables()
    rng = np.random.default_rng(3)
    W, H = 61, 37                               # ragged edge blocks on both axes
    bins = rng.integers(0, t.n_wv, W * H)
    L = _flat_radiance(t, bins, rho=1.0) * rng.uniform(0.05, 0.6, (W * H, 1)).astype(np.float32)
    L *= (1 + 0.01 * rng.standard_normal(L.shape)).astype(np.float32)
    L[rng.choice(W * H, 40, replace=False), _bands(t)[1]] = np.nan      # some pixels without a depth
    got, depth = oracle.wv_presolve(t, L, W, H)
    ref, Dref = _numpy_presolve(t, L, W, H, 12)
    fin = np.isfinite(Dref)
    assert np.array_equal(np.isfinite(depth), fin)
    assert np.allclose(depth[fin], Dref[fin], rtol=0, atol=2e-7)
    assert np.array_equal(got, ref)


def test_scene_bins_from_the_forward_model():
    """The coarsened scene's fine truth (water vapour constant per 12 x 12
    block, 5 % fire sub-pixels): noise-free, every block's bin is recovered;
    with the configs' noise, at least 95 % of the blocks (the median of 144
    depths carries the noise of about a dozen)."""
    t = synth.make_tables()
    tr = synth.make_config5_fine_truth(seed=4, width=240, height=120)
    L0 = oracle.forward(t, 1, tr.state1(), tr.wv_bin).astype(np.float32)
    got, _ = oracle.wv_presolve(t, L0, 240, 120)
    assert np.mean(got == tr.wv_bin) == 1.0
    z = synth.noise_normals(4, np.arange(tr.n_pix), t.n_bands)
    L = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, z, NOISE_REL, NOISE_ABS)
    got, _ = oracle.wv_presolve(t, L, 240, 120)
    blocks = got.reshape(10, 12, 20, 12)[:, 0, :, 0] == tr.wv_bin.reshape(10, 12, 20, 12)[:, 0, :, 0]
    assert blocks.mean() >= 0.95, blocks.mean()


def test_empty_block_gets_the_invalid_bin():
    t = synth.make_tables()
    bins = np.zeros(24 * 12, np.int64)
    L = _flat_radiance(t, bins)
    L[:, :] = np.where(np.arange(24 * 12)[:, None] % 24 < 12, np.nan, L)   # left block all NaN
    got, _ = oracle.wv_presolve(t, L, 24, 12)
    img = got.reshape(12, 24)
    assert np.all(img[:, :12] == 0xFFFF) and np.all(img[:, 12:] == 0)


@pytest.mark.parametrize("n_fire", [10, 60])
def test_fire_pixels_below_half_the_block_do_not_move_its_bin(n_fire):
    t = synth.make_tables()
    tr = synth.make_config1_truth(seed=8, width=12, height=12, fire_frac=0.0)
    tr.wv_bin[:] = 7
    st = tr.state1()
    rng = np.random.default_rng(n_fire)
    hot = rng.choice(144, n_fire, replace=False)
    st[hot, 3] = 0.3
    st[hot, 4] = 1400.0
    L = oracle.forward(t, 1, st, tr.wv_bin).astype(np.float32)
    got, _ = oracle.wv_presolve(t, L, 12, 12)
    assert np.all(got == 7)


def test_even_block_takes_the_lower_median():
    """72 pixels at bin 3's depth and 72 at bin 9's: the lower median (rank
    (n - 1) / 2) is bin 3's depth; one more bin-9 pixel flips it."""
    t = synth.make_tables()
    bins = np.array([3] * 72 + [9] * 72)
    got, _ = oracle.wv_presolve(t, _flat_radiance(t, bins), 12, 12)
    assert np.all(got == 3)
    bins[0] = 9
    got, _ = oracle.wv_presolve(t, _flat_radiance(t, bins), 12, 12)
    assert np.all(got == 9)


def test_injection_is_the_forward_models_thermal_term():
    """Eq. (inject) onto a noise-free background equals the forward model of
    the same surface with that single-temperature fire (alpha, T): the
    thermal term alpha tau_up B(lambda, T) is the only difference; alpha = 0
    returns the background."""
    t = synth.make_tables()
    tr, alpha, T = synth.make_injection_experiment(seed=3, n=64)
    bg = oracle.forward(t, 1, tr.state1(), tr.wv_bin).astype(np.float32)
    inj = oracle.inject(t, bg, tr.wv_bin, alpha, T)
    st = tr.state1()
    st[:, 3], st[:, 4] = alpha, T
    fire = oracle.forward(t, 1, st, tr.wv_bin)
    assert np.allclose(inj, fire, rtol=2e-7, atol=1e-12)
    assert np.array_equal(oracle.inject(t, bg, tr.wv_bin, np.zeros(64), T), bg)
