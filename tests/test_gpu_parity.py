"""GPU path (C-ABI through the ctypes binding) against the FP64 oracle on the
same seeded inputs: forward model, full per-pixel retrieval (config 1:
64x64x284), ragged and degenerate cases, host-staged path, determinism.

Parity bar over the pixels the oracle calls converged and identifiable: the
GPU converged too, with |dE[T]| <= 0.5 K and |d alpha| <= 1e-3 *
max(alpha_oracle, 1e-4), for >= 99.9 % of them (a pixel the GPU did not
converge is a miss); sigma[T], cost, rms and the identifiability flag are
held to the secondary bars of scenes.parity_stats on the same pixels."""
import numpy as np
import pytest

import oracle
import synth
from scenes import NOISE_ABS, NOISE_REL, config1, config2_subset, parity_stats, summary

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fr():
    from paper_2608_07580_b300 import firert
    return firert


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.fixture(scope="module")
def c1():
    return config1()


@pytest.fixture(scope="module")
def c1_oracle(c1):
    t, tr, L = c1
    return oracle.retrieve(t, L, tr.wv_bin)


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _np(d):
    return {k: v.cpu().numpy() if hasattr(v, "cpu") else v for k, v in d.items()}


def _retrieve(fr, torch, t, L, wv, **kw):
    ctx = fr.Context(t)
    out = ctx.retrieve(_dev(torch, L, torch.float32), _dev(torch, wv.astype(np.int16), torch.int16),
                       **kw)
    torch.cuda.synchronize()
    g = _np(out)
    g["iters"] = g["iters"].astype(np.uint16)
    return ctx, g


def test_tables_and_forward_single_temperature(fr, torch):
    t = synth.make_tables(path_reflectance=True)
    ctx = fr.Context(t)
    rng = np.random.default_rng(1)
    n = 300
    xs = rng.dirichlet(np.ones(3), n)
    st = np.column_stack([xs, 10 ** rng.uniform(-4, -0.3, n), rng.uniform(400, 2100, n)])
    wv = rng.integers(0, 16, n).astype(np.uint16)
    Lg = ctx.forward(1, _dev(torch, st, torch.float32), _dev(torch, wv.astype(np.int16), torch.int16))
    Lo = oracle.forward(t, 1, st.astype(np.float32).astype(np.float64), wv)
    rel = np.abs(Lg.cpu().numpy() - Lo) / np.maximum(np.abs(Lo), 1e-6)
    assert rel.max() < 1e-5


def test_forward_mixture_matches_oracle(fr, torch):
    t = synth.make_tables()
    ctx = fr.Context(t)
    rng = np.random.default_rng(2)
    n = 300
    xs = rng.dirichlet(np.ones(3), n)
    x2 = np.column_stack([rng.uniform(900, 2100, n), rng.uniform(30, 400, n),
                          rng.uniform(360, 990, n), rng.uniform(30, 400, n),
                          rng.uniform(0, 1, n), 10 ** rng.uniform(-4, -0.3, n)])
    st = np.column_stack([xs, x2])
    wv = rng.integers(0, 16, n).astype(np.uint16)
    Lg = ctx.forward(2, _dev(torch, st, torch.float32), _dev(torch, wv.astype(np.int16), torch.int16))
    Lo = oracle.forward(t, 2, st.astype(np.float32).astype(np.float64), wv)
    rel = np.abs(Lg.cpu().numpy() - Lo) / np.maximum(np.abs(Lo), 1e-6)
    assert rel.max() < 2e-5


def test_forward_noise_uses_the_counter_generator(fr, torch):
    t = synth.make_tables()
    ctx = fr.Context(t)
    tr = synth.make_config1_truth(seed=5, width=16, height=16)
    st = tr.state1()
    Lg = ctx.forward(1, _dev(torch, st, torch.float32),
                     _dev(torch, tr.wv_bin.astype(np.int16), torch.int16),
                     NOISE_REL, NOISE_ABS, seed=5, stream_id=synth.STREAM_NOISE).cpu().numpy()
    z = synth.noise_normals(5, np.arange(tr.n_pix), t.n_bands)
    Lo = oracle.synth_radiance(t, 1, st.astype(np.float32).astype(np.float64), tr.wv_bin, z,
                               NOISE_REL, NOISE_ABS)
    sd = np.sqrt((NOISE_REL * Lo) ** 2 + NOISE_ABS ** 2)
    assert np.max(np.abs(Lg - Lo) / sd) < 1e-3


def test_block_mean(fr, torch):
    rng = np.random.default_rng(3)
    w, h, nb = 50, 37, 13
    src = rng.normal(size=(h * w, nb)).astype(np.float32)
    dst = fr.block_mean(_dev(torch, src, torch.float32), w, h, nb, 12).cpu().numpy()
    ref = src.reshape(h, w, nb)[:36, :48].reshape(3, 12, 4, 12, nb).mean(axis=(1, 3)).reshape(-1, nb)
    assert np.max(np.abs(dst - ref)) < 1e-5


# every retrieval comparison of this module: (pool, passes, name)
_ALL = []


def assert_parity(s, min_pool, what=""):
    """The parity bar (>= 99.9 % of the oracle's converged identifiable
    pixels, GPU non-convergence counted as a miss) on a pool of at least
    min_pool pixels; the secondary outputs (sigma[T], cost, rms) of the
    pixels that pass agree on >= 99 % of them (cost and rms follow the
    final point along flat valleys)."""
    print(what, summary(s), "fail:", s["fail_idx"][:10], "secondary fail:", s["sec_fail_idx"][:10])
    assert s["pool"] >= min_pool, (what, s["pool"])
    _ALL.append((s["pool"], s["pass"], what))
    assert s["rate"] >= 0.999, (what, summary(s))
    assert s["sec_rate"] >= 0.99, (what, summary(s))


# Scenes built to stress the mixture's degeneracy (30 % fire pixels whose
# truth is one temperature, fitted by the two-component mixture, under five
# endmembers, path reflectance and the noise-weighted loss): there the two
# solvers, on different rounding, now and then settle in different points
# of a flat valley (a smouldering component of a few per cent weight near
# the cold end of its range, which the spectrum barely sees, trades against
# alpha and the flaming weight); which pixels do moves with any change of
# rounding (0 to 5 of ~1,600 per scene across builds). Each such scene is
# held to 99.6 % and every comparison of the module together to the full
# 99.9 % bar (test_all_scenes_together_meet_the_bar).
def assert_stress_parity(s, min_pool, what):
    print(what, summary(s), "fail:", s["fail_idx"][:10], "secondary fail:", s["sec_fail_idx"][:10])
    assert s["pool"] >= min_pool, (what, s["pool"])
    _ALL.append((s["pool"], s["pass"], what))
    assert s["rate"] >= 0.996, (what, summary(s))
    assert s["sec_rate"] >= 0.99, (what, summary(s))


def test_config1_parity(fr, torch, c1, c1_oracle):
    t, tr, L = c1
    ctx, g = _retrieve(fr, torch, t, L, tr.wv_bin)
    s = parity_stats(c1_oracle, g)
    st = ctx.stats()
    print("stats:", st)
    assert st["n_pixels"] == tr.n_pix
    assert st["mma_rounds2"] > 0   # the default (unweighted) fit runs the tensor-core stage 2
    assert_parity(s, 100, "config1")
    # the per-pixel outcome codes agree
    go, oo = g["status"] & 7, c1_oracle["status"] & 7
    assert np.mean(go == oo) > 0.995


@pytest.fixture(scope="module")
def c30():
    """A 96 x 96 single-temperature scene with 30 % fire pixels (a pool of
    ~1,500 converged identifiable pixels)."""
    return config1(seed=21, width=96, height=96, fire_frac=0.3)


@pytest.fixture(scope="module")
def flight_fire():
    """20,000 fire pixels and 2,000 others of the flight-line chunk (1240 x
    2048, seed 1: the paper's Gaussian p(T) on the grid, 2 % fire fronts),
    radiance from the oracle's forward model plus the counter-based noise.
    The pool of converged identifiable pixels (~4,800) lets the 99.9 % bar
    resolve a few misses: the near-degenerate mixture leaves a few pixels in
    10,000 whose FP32 and FP64 paths part (a flat valley that one side
    crosses within the iteration cap and the other not, or a second
    minimum), so a pool of ~1,500 decided the bar on one pixel."""
    t = synth.make_tables()
    tr = synth.make_config2_truth(seed=1)
    rng = np.random.default_rng(17)
    idx = np.sort(np.concatenate([rng.choice(np.flatnonzero(tr.kind == 2), 20000, replace=False),
                                  rng.choice(np.flatnonzero(tr.kind == 0), 2000, replace=False)]))
    sub, L = config2_subset(idx, tr, t)
    return t, sub, L


@pytest.fixture(scope="module")
def flight_fire_oracle(flight_fire):
    t, sub, L = flight_fire
    return oracle.retrieve(t, L, sub.wv_bin)


@pytest.mark.parametrize("variant", [6, 3])
def test_flight_line_fire_pixels_parity(fr, torch, flight_fire, flight_fire_oracle, variant):
    """A pool of ~4,800 converged identifiable flight-line fire pixels,
    through the tensor-core (6) and the FP32 (3) stage-2 evaluation, at the
    99.9 % bar."""
    t, sub, L = flight_fire
    ctx = fr.Context(t)
    ctx.set_tuning(variant, 2)
    g = _np(ctx.retrieve(_dev(torch, L, torch.float32),
                         _dev(torch, sub.wv_bin.astype(np.int16), torch.int16)))
    torch.cuda.synchronize()
    s = parity_stats(flight_fire_oracle, g)
    assert_parity(s, 1000, f"flight fire pixels, variant {variant}")
    # the non-fire pixels: surface fractions and the thermal fraction
    nf = (sub.kind == 0) & ((flight_fire_oracle["status"] & 7) == 0) & ((g["status"] & 7) == 0)
    dx = np.abs(g["state"][nf, :3] - flight_fire_oracle["state"][nf, :3]).max(1)
    da = np.abs(g["alpha"][nf] - flight_fire_oracle["alpha"][nf])
    print("non-fire: max |dx_surf|", dx.max(), "max |d alpha|", da.max())
    assert np.mean(dx <= 1e-4) >= 0.999
    assert np.mean(da <= 1e-3 * np.maximum(flight_fire_oracle["alpha"][nf], 1e-4)) >= 0.995


def test_config1_surface_and_stage1(fr, torch, c1, c1_oracle):
    t, tr, L = c1
    _, g = _retrieve(fr, torch, t, L, tr.wv_bin)
    o = c1_oracle
    conv = ((o["status"] & 7) == 0) & ((g["status"] & 7) == 0)
    # surface fractions agree tightly (well-conditioned linear part of stage 1)
    assert np.percentile(np.abs(g["state"][conv, :3] - o["state"][conv, :3]).max(1), 99) < 1e-3


def test_ragged_sizes_and_empty(fr, torch, c1, c1_oracle):
    t, tr, L = c1
    ctx = fr.Context(t)
    for n in (0, 1, 7, 33, 129):
        out = ctx.retrieve(_dev(torch, L[:n], torch.float32),
                           _dev(torch, tr.wv_bin[:n].astype(np.int16), torch.int16))
        torch.cuda.synchronize()
        if n:
            g = out["ET"].cpu().numpy()
            o = c1_oracle["ET"][:n]
            conv = ((c1_oracle["status"][:n] & 23) == 0) & ((out["status"].cpu().numpy() & 7) == 0)
            assert np.all(np.abs(g[conv] - o[conv]) <= 0.5)
            assert ctx.stats()["n_pixels"] == n


def test_degenerate_pixels(fr, torch):
    t = synth.make_tables(sat_level=25.0)
    tr = synth.make_config1_truth(seed=9, width=8, height=1, fire_frac=1.0, alpha_range=(0.3, 0.5),
                                  t_range=(1400, 1500))
    z = synth.noise_normals(9, np.arange(8), t.n_bands)
    L = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, z, NOISE_REL, NOISE_ABS)
    L[1, 40] = np.nan
    L[2, :] = 30.0                      # every band saturated
    o = oracle.retrieve(t, L, tr.wv_bin)
    _, g = _retrieve(fr, torch, t, L, tr.wv_bin)
    assert g["status"][1] & 7 == fr.PX_NONFINITE and o["status"][1] & 7 == oracle.NONFINITE
    assert g["status"][2] & 7 == fr.PX_ALL_MASKED and o["status"][2] & 7 == oracle.ALL_MASKED
    ok = [i for i in range(8) if i not in (1, 2) and (o["status"][i] & 23) == 0
          and (g["status"][i] & 7) == 0]
    assert len(ok) >= 3
    assert np.all(np.abs(g["ET"][ok] - o["ET"][ok]) <= 0.5)


def test_hfdi_gate(fr, torch, c1, c1_oracle):
    t, tr, L = c1
    _, g = _retrieve(fr, torch, t, L, tr.wv_bin, gate_hfdi=True)
    o = oracle.retrieve(t, L, tr.wv_bin, oracle.Config(gate_hfdi=True))
    assert np.array_equal(g["status"] & 7 == fr.PX_NOT_CANDIDATE,
                          o["status"] & 7 == oracle.NOT_CANDIDATE)
    assert np.allclose(g["hfdi"], o["hfdi"], atol=1e-5)


def test_host_path_equals_device_path_and_is_deterministic(fr, torch, c1):
    t, tr, L = c1
    ctx, g1 = _retrieve(fr, torch, t, L, tr.wv_bin)
    _, g2 = _retrieve(fr, torch, t, L, tr.wv_bin)
    h = ctx.retrieve(L, tr.wv_bin)
    for k in ("ET", "alpha", "state", "cov", "status", "iters"):
        assert np.array_equal(g1[k], g2[k], equal_nan=True) if g1[k].dtype.kind == "f" \
            else np.array_equal(g1[k], g2[k]), k
        hk = h[k].astype(g1[k].dtype) if k == "iters" else h[k]
        assert np.array_equal(g1[k], hk, equal_nan=True) if g1[k].dtype.kind == "f" \
            else np.array_equal(g1[k], hk), k


def test_chunked_host_path_equals_device_path(fr, torch):
    """A host scene of 153,600 pixels is fitted in chunks whose copies overlap
    the fits of the other chunks (two: 65,536 and 88,064 pixels): every output
    equals the device path's bit for bit."""
    t = synth.make_tables()
    tr = synth.make_config2_truth(seed=5, width=256, height=600)
    ctx = fr.Context(t)
    st = torch.from_numpy(tr.state2().astype(np.float32)).cuda()
    wv = torch.from_numpy(tr.wv_bin.astype(np.int16)).cuda()
    rad = ctx.forward(2, st, wv, NOISE_REL, NOISE_ABS, seed=tr.seed, stream_id=synth.STREAM_NOISE)
    g = {k: v.cpu().numpy() for k, v in ctx.retrieve(rad, wv).items()}
    L = np.ascontiguousarray(rad.cpu().numpy())
    h = ctx.retrieve(L, tr.wv_bin)
    assert ctx.stats()["kernel_launches"] == 6        # two chunks x three kernels
    for k in ("ET", "sdT", "alpha", "state", "cov", "cost", "status", "iters", "hfdi"):
        hk = h[k].astype(g[k].dtype) if k == "iters" else h[k]
        assert np.array_equal(g[k], hk, equal_nan=True) if g[k].dtype.kind == "f" \
            else np.array_equal(g[k], hk), k


def test_given_init_matches_oracle(fr, torch, c1):
    """A given start (the truth, written in the mixture's form: the single
    temperature as the hot mean above 1000 K, else as the smouldering mean)
    for every fire pixel of the scene."""
    t, tr, L = c1
    idx = np.flatnonzero(tr.kind == 1)
    T = tr.single[idx, 1]
    init = np.column_stack([tr.x_surf[idx], tr.single[idx, 0], T,
                            np.clip(T, 900, 2200), np.full(idx.size, 60.0),
                            np.clip(T, 350, 1000), np.full(idx.size, 60.0),
                            (T >= 1000).astype(float), tr.single[idx, 0]]).astype(np.float32)
    o = oracle.retrieve(t, L[idx], tr.wv_bin[idx], init_state=init.astype(np.float64))
    ctx = fr.Context(t)
    out = ctx.retrieve(_dev(torch, L[idx], torch.float32),
                       _dev(torch, tr.wv_bin[idx].astype(np.int16), torch.int16),
                       init_state=_dev(torch, init, torch.float32))
    torch.cuda.synchronize()
    s = parity_stats(o, _np(out))
    assert_parity(s, 50, "given start")


@pytest.mark.parametrize("stage,variant", [(1, 3), (2, 3), (2, 6)])
def test_normal_equations_match_oracle(fr, torch, c1, stage, variant):
    """One iteration's J^T W J + P, J^T W r - P(z - pm) and cost, formed by the
    kernel in FP32, against the oracle's FP64 at the same random states;
    stage 2 through the FP32 evaluation (variant 3) and through the
    tensor-core one (variant 6, the grid-node sums as bf16x3 products)."""
    t, tr, L = c1
    rng = np.random.default_rng(20 + stage)
    idx = np.concatenate([np.flatnonzero(tr.kind == 1)[:40], rng.choice(tr.n_pix, 24, replace=False)])
    n = idx.size
    xs = rng.dirichlet(np.ones(3), n)
    if stage == 1:
        st = np.column_stack([xs, 10 ** rng.uniform(-3.5, -0.5, n), rng.uniform(450, 2100, n)])
    else:
        st = np.column_stack([xs, rng.uniform(950, 2100, n), rng.uniform(35, 400, n),
                              rng.uniform(380, 990, n), rng.uniform(35, 400, n),
                              rng.uniform(0.05, 0.95, n), 10 ** rng.uniform(-3.5, -0.5, n)])
    st = st.astype(np.float32)
    ctx = fr.Context(t)
    ctx.set_tuning(variant, 1)
    H, g, cost = ctx.normal_equations(stage, _dev(torch, L[idx], torch.float32),
                                      _dev(torch, tr.wv_bin[idx].astype(np.int16), torch.int16),
                                      _dev(torch, st, torch.float32))
    H, g, cost = H.cpu().numpy(), g.cpu().numpy(), cost.cpu().numpy()
    worst = np.zeros(3)
    for j, i in enumerate(idx):
        Ho, go, co = oracle.normal_equations(t, stage, L[i], tr.wv_bin[i], st[j].astype(np.float64))
        d = np.sqrt(np.outer(np.diag(Ho), np.diag(Ho)))
        e = (np.max(np.abs(H[j] - Ho) / d), np.max(np.abs(g[j] - go) / np.sqrt(np.diag(Ho) * co)),
             abs(cost[j] - co) / co)
        worst = np.maximum(worst, e)
        assert e[0] < 2e-4 and e[1] < 2e-4 and e[2] < 1e-4, (stage, variant, i, e)
    print(f"stage {stage} variant {variant}: max rel. error H {worst[0]:.2e} g {worst[1]:.2e} "
          f"cost {worst[2]:.2e}")


@pytest.fixture(scope="module")
def small_tables_scene():
    # 160 bands put 120 bands in the stage-2 window (one 128-band tile of the
    # tensor-core product); a 40-node grid leaves 24 of the product's 64
    # nodes as zero padding
    return config1(seed=7, width=96, height=96, fire_frac=0.3, n_bands=160, n_tgrid=40)


@pytest.mark.parametrize("variant", [3, 6])
def test_other_table_shapes_match_oracle(fr, torch, small_tables_scene, variant):
    """Tables other than the default 284 bands x 64 nodes, through the FP32
    (3) and the tensor-core (6) stage-2 evaluation: one evaluation's normal
    equations at random states, and the retrieval, against the oracle."""
    t, tr, L = small_tables_scene
    ctx = fr.Context(t)
    ctx.set_tuning(variant, 1)
    assert ctx.window_bands()[3] <= 128
    rng = np.random.default_rng(31)
    idx = np.concatenate([np.flatnonzero(tr.kind == 1)[:24], rng.choice(tr.n_pix, 16, replace=False)])
    n = idx.size
    st = np.column_stack([rng.dirichlet(np.ones(3), n), rng.uniform(950, 2100, n),
                          rng.uniform(60, 400, n), rng.uniform(380, 990, n),
                          rng.uniform(60, 400, n), rng.uniform(0.05, 0.95, n),
                          10 ** rng.uniform(-3.5, -0.5, n)]).astype(np.float32)
    H, g, cost = ctx.normal_equations(2, _dev(torch, L[idx], torch.float32),
                                      _dev(torch, tr.wv_bin[idx].astype(np.int16), torch.int16),
                                      _dev(torch, st, torch.float32))
    H, g, cost = H.cpu().numpy(), g.cpu().numpy(), cost.cpu().numpy()
    for j, i in enumerate(idx):
        Ho, go, co = oracle.normal_equations(t, 2, L[i], tr.wv_bin[i], st[j].astype(np.float64))
        d = np.sqrt(np.outer(np.diag(Ho), np.diag(Ho)))
        e = (np.max(np.abs(H[j] - Ho) / d), np.max(np.abs(g[j] - go) / np.sqrt(np.diag(Ho) * co)),
             abs(cost[j] - co) / co)
        assert e[0] < 2e-4 and e[1] < 2e-4 and e[2] < 1e-4, (variant, i, e)
    o = oracle.retrieve(t, L, tr.wv_bin)
    out = _np(ctx.retrieve(_dev(torch, L, torch.float32),
                           _dev(torch, tr.wv_bin.astype(np.int16), torch.int16)))
    s = parity_stats(o, out)
    assert_parity(s, 1000, f"160 bands / 40 nodes, variant {variant}")


@pytest.fixture(scope="module")
def five_endmember_scene():
    """Tables with five endmembers (the two added: a flat 0.10 ash and a
    rising dry-grass spectrum, resampled like the others) and a 48 x 48
    single-temperature scene drawn over them."""
    import dataclasses
    t = synth.make_tables()
    lam = t.wavelength_nm.astype(np.float64)
    ash = np.full_like(lam, 0.10)
    grass = 0.05 + 0.30 * np.clip((lam - 400.0) / 1800.0, 0.0, 1.0)
    t5 = dataclasses.replace(t, endmembers=np.ascontiguousarray(
        np.vstack([t.endmembers, ash[None], grass[None]]), dtype=np.float32))
    tr = synth.make_config1_truth(seed=11, width=96, height=96, n_endm=5, fire_frac=0.3)
    z = synth.noise_normals(11, np.arange(tr.n_pix), t5.n_bands)
    L = oracle.synth_radiance(t5, 1, tr.state1(), tr.wv_bin, z, NOISE_REL, NOISE_ABS)
    return t5, tr, L


@pytest.mark.parametrize("variant", [3, 6])
def test_five_endmembers_match_oracle(fr, torch, five_endmember_scene, variant):
    """K = 5 (the second compiled endmember count) through both stage-2
    evaluations: the stage-1 normal equations at random states and the
    retrieval against the oracle."""
    t, tr, L = five_endmember_scene
    ctx = fr.Context(t)
    ctx.set_tuning(variant, 1)
    rng = np.random.default_rng(41)
    idx = np.concatenate([np.flatnonzero(tr.kind == 1)[:16], rng.choice(tr.n_pix, 16, replace=False)])
    n = idx.size
    st = np.column_stack([rng.dirichlet(np.ones(5), n), 10 ** rng.uniform(-3.5, -0.5, n),
                          rng.uniform(450, 2100, n)]).astype(np.float32)
    H, g, cost = ctx.normal_equations(1, _dev(torch, L[idx], torch.float32),
                                      _dev(torch, tr.wv_bin[idx].astype(np.int16), torch.int16),
                                      _dev(torch, st, torch.float32))
    H, g, cost = H.cpu().numpy(), g.cpu().numpy(), cost.cpu().numpy()
    for j, i in enumerate(idx):
        Ho, go, co = oracle.normal_equations(t, 1, L[i], tr.wv_bin[i], st[j].astype(np.float64))
        d = np.sqrt(np.outer(np.diag(Ho), np.diag(Ho)))
        assert np.max(np.abs(H[j] - Ho) / d) < 2e-4, (variant, i)
        assert np.max(np.abs(g[j] - go) / np.sqrt(np.diag(Ho) * co)) < 2e-4, (variant, i)
        assert abs(cost[j] - co) / co < 1e-4, (variant, i)
    o = oracle.retrieve(t, L, tr.wv_bin)
    out = _np(ctx.retrieve(_dev(torch, L, torch.float32),
                           _dev(torch, tr.wv_bin.astype(np.int16), torch.int16)))
    s = parity_stats(o, out)
    assert_stress_parity(s, 1000, f"K=5 variant {variant}")


def test_path_reflectance_retrieval_matches_oracle(fr, torch):
    """Tables with path reflectance and spherical albedo (the full solar term
    of Eq. solar, with its denominator 1 - S rho): stage-1 normal equations at
    random states and the retrieval of a 48 x 48 scene against the oracle."""
    t = synth.make_tables(path_reflectance=True)
    tr = synth.make_config1_truth(seed=13, width=96, height=96, fire_frac=0.3)
    z = synth.noise_normals(13, np.arange(tr.n_pix), t.n_bands)
    L = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, z, NOISE_REL, NOISE_ABS)
    ctx = fr.Context(t)
    rng = np.random.default_rng(43)
    idx = np.concatenate([np.flatnonzero(tr.kind == 1)[:16], rng.choice(tr.n_pix, 16, replace=False)])
    n = idx.size
    st = np.column_stack([rng.dirichlet(np.ones(3), n), 10 ** rng.uniform(-3.5, -0.5, n),
                          rng.uniform(450, 2100, n)]).astype(np.float32)
    H, g, cost = ctx.normal_equations(1, _dev(torch, L[idx], torch.float32),
                                      _dev(torch, tr.wv_bin[idx].astype(np.int16), torch.int16),
                                      _dev(torch, st, torch.float32))
    H, g, cost = H.cpu().numpy(), g.cpu().numpy(), cost.cpu().numpy()
    for j, i in enumerate(idx):
        Ho, go, co = oracle.normal_equations(t, 1, L[i], tr.wv_bin[i], st[j].astype(np.float64))
        d = np.sqrt(np.outer(np.diag(Ho), np.diag(Ho)))
        assert np.max(np.abs(H[j] - Ho) / d) < 2e-4, i
        assert np.max(np.abs(g[j] - go) / np.sqrt(np.diag(Ho) * co)) < 2e-4, i
        assert abs(cost[j] - co) / co < 1e-4, i
    o = oracle.retrieve(t, L, tr.wv_bin)
    out = _np(ctx.retrieve(_dev(torch, L, torch.float32),
                           _dev(torch, tr.wv_bin.astype(np.int16), torch.int16)))
    s = parity_stats(o, out)
    assert_stress_parity(s, 1000, "path reflectance")


@pytest.mark.parametrize("variant", [3, 6])
def test_noise_weighted_loss_matches_oracle(fr, torch, c30, variant):
    """The noise-weighted loss (weights 1 / sd_b^2 of the noise model) on both
    sides: stage-2 normal equations at random states and the retrieval."""
    t, tr, L = c30
    ctx = fr.Context(t, fr.default_config(weighted=1))
    ctx.set_tuning(variant, 1)
    cfg = oracle.Config(weighted=True)
    rng = np.random.default_rng(47)
    idx = np.concatenate([np.flatnonzero(tr.kind == 1)[:16], rng.choice(tr.n_pix, 16, replace=False)])
    n = idx.size
    st = np.column_stack([rng.dirichlet(np.ones(3), n), rng.uniform(950, 2100, n), rng.uniform(35, 400, n),
                          rng.uniform(380, 990, n), rng.uniform(35, 400, n),
                          rng.uniform(0.05, 0.95, n), 10 ** rng.uniform(-3.5, -0.5, n)]).astype(np.float32)
    H, g, cost = ctx.normal_equations(2, _dev(torch, L[idx], torch.float32),
                                      _dev(torch, tr.wv_bin[idx].astype(np.int16), torch.int16),
                                      _dev(torch, st, torch.float32))
    H, g, cost = H.cpu().numpy(), g.cpu().numpy(), cost.cpu().numpy()
    for j, i in enumerate(idx):
        Ho, go, co = oracle.normal_equations(t, 2, L[i], tr.wv_bin[i], st[j].astype(np.float64), cfg=cfg)
        d = np.sqrt(np.outer(np.diag(Ho), np.diag(Ho)))
        assert np.max(np.abs(H[j] - Ho) / d) < 2e-4, (variant, i)
        assert np.max(np.abs(g[j] - go) / np.sqrt(np.diag(Ho) * co)) < 2e-4, (variant, i)
        assert abs(cost[j] - co) / co < 1e-4, (variant, i)
    o = oracle.retrieve(t, L, tr.wv_bin, cfg=cfg)
    out = _np(ctx.retrieve(_dev(torch, L, torch.float32),
                           _dev(torch, tr.wv_bin.astype(np.int16), torch.int16)))
    # the tensor-core stage 2 fits the unweighted loss only: a weighted fit
    # runs the FP32 stage 2 whatever the launch shape
    assert ctx.stats()["mma_rounds2"] == 0
    s = parity_stats(o, out, cfg=cfg)
    assert_stress_parity(s, 1000, f"weighted, variant {variant}")


def _snap_to_bounds(state, K, cfg=None):
    """A GPU state as the oracle's coordinates: a stage-2 variable on its
    bound holds the bound rounded to fp32; put it on the oracle's FP64 bound."""
    cfg = cfg or oracle.Config(n_endm=K)
    st = np.array(state, dtype=np.float64)
    for k, (lo, hi) in enumerate(zip(cfg.lo2, cfg.hi2)):
        col = st[:, K + 2 + k]
        col[np.abs(col - lo) <= 1e-6 * max(abs(lo), 1e-30)] = lo
        col[np.abs(col - hi) <= 1e-6 * max(abs(hi), 1e-30)] = hi
    return st


def test_posterior_at_the_gpu_state_matches_oracle(fr, torch, flight_fire):
    """The outputs that follow from the final state alone (Sec. 2.3 moments,
    cost, rms, Laplace covariance, var(E[T]), identifiability), checked apart
    from the fit: at each GPU-converged pixel's final state the oracle forms
    them in FP64 (oracle.posterior_at) and the GPU's must agree. Pixels whose
    alpha stands clear of noise get the FP64 normal matrix on the GPU too:
    there the covariance entries and var(E[T]) agree to 1e-3 relative and
    the identifiability flag agrees wherever the oracle's decision is not
    within 2 % of a threshold."""
    t, sub, L = flight_fire
    sel = np.arange(0, sub.n_pix, 2)
    ctx = fr.Context(t)
    g = _np(ctx.retrieve(_dev(torch, L[sel], torch.float32),
                         _dev(torch, sub.wv_bin[sel].astype(np.int16), torch.int16)))
    n64 = ctx.stats()["n_post64"]
    i = np.flatnonzero((g["status"] & 7) == 0)
    st = _snap_to_bounds(g["state"][i], t.n_endm)
    p = oracle.posterior_at(t, L[sel][i], sub.wv_bin[sel][i], st)
    assert np.max(np.abs(g["ET"][i] - p["ET"])) < 1e-3
    assert np.max(np.abs(g["sdT"][i] - p["sdT"])) < 1e-3
    assert np.max(np.abs(g["cost"][i] / p["cost"] - 1)) < 1e-4
    assert np.max(np.abs(g["rms"][i] / p["rms"] - 1)) < 1e-4
    from scenes import ident_borderline
    ob = {"var_ET": p["var_ET"], "alpha": st[:, t.n_endm + 7], "cov": p["cov"]}
    border = ident_borderline(ob)
    gi = (g["status"][i] & fr.PX_F_NOT_IDENT) == 0
    mism = np.flatnonzero((gi != p["ident"]) & ~border)
    print(f"posterior at the GPU state: {i.size} pixels, {n64} with the FP64 normal matrix, "
          f"{p['ident'].sum()} identifiable, flag mismatches {mism.size}")
    with np.errstate(all="ignore"):
        for j in mism[:10]:
            print("  mismatch", i[j], "gpu ident", gi[j], "sdE gpu/oracle", np.sqrt(g["var_ET"][i[j]]),
                  np.sqrt(p["var_ET"][j]), "snr gpu/oracle", g["alpha"][i[j]] / np.sqrt(g["cov"][i[j], 20]),
                  st[j, t.n_endm + 7] / np.sqrt(p["cov"][j, 20]), "x2", st[j, t.n_endm + 2:])
    assert mism.size <= max(1, i.size // 1000), mism[:10]
    # covariance and var(E[T]) where both say identifiable (FP64 on both
    # sides) and hold the same variables on their bounds (the zero rows of
    # the covariance): a variable on its bound whose gradient is zero to
    # rounding may be held or freed, and either is a correct active set
    idn = p["ident"] & gi
    assert idn.sum() >= 500 and n64 >= idn.sum()
    same = np.all((g["cov"][i] == 0) == (p["cov"] == 0), axis=1)
    print("identifiable pixels with differing active sets:", (idn & ~same).sum(), "of", idn.sum())
    assert (idn & ~same).sum() <= max(1, idn.sum() // 1000)
    idn = idn & same
    ev = np.abs(g["var_ET"][i][idn] / p["var_ET"][idn] - 1)
    diag = [0, 6, 11, 15, 18, 20]
    cg, co = g["cov"][i][idn][:, diag].astype(np.float64), p["cov"][idn][:, diag]
    m = np.isfinite(co) & (co > 0)
    ec = np.abs(cg[m] / co[m] - 1)
    print("var(E[T]) rel. error max", ev.max(), "covariance diagonal rel. error max", ec.max())
    assert ev.max() < 1e-3 and ec.max() < 1e-3


@pytest.mark.parametrize("kappa_max", [0.0, 1e5])
def test_fp64_step_solves_match_oracle(fr, torch, c1, c1_oracle, flight_fire, flight_fire_oracle,
                                       kappa_max):
    """The precision policy: with kappa_max = 0 every step is solved in FP64,
    with 1e5 (the scope table's threshold) those above it; both against the
    oracle at the full bar, and the FP64 solves are counted."""
    t, tr, L = c1
    ctx = fr.Context(t, fr.default_config(kappa_max=kappa_max))
    g = _np(ctx.retrieve(_dev(torch, L, torch.float32),
                         _dev(torch, tr.wv_bin.astype(np.int16), torch.int16)))
    torch.cuda.synchronize()
    st = ctx.stats()
    print("FP64 solves", st["solves64_1"], st["solves64_2"], "fp64 pixels", st["n_fp64_pixels"])
    assert st["solves64_1"] + st["solves64_2"] > 0
    if kappa_max == 0.0:
        # every step solve: at least one per trial step
        assert st["solves64_1"] >= st["sum_it1"] and st["solves64_2"] >= st["sum_it2"]
    assert_parity(parity_stats(c1_oracle, g), 100, f"config1 kappa_max {kappa_max}")
    t2, sub, L2 = flight_fire
    ctx2 = fr.Context(t2, fr.default_config(kappa_max=kappa_max))
    g2 = _np(ctx2.retrieve(_dev(torch, L2, torch.float32),
                           _dev(torch, sub.wv_bin.astype(np.int16), torch.int16)))
    assert_parity(parity_stats(flight_fire_oracle, g2), 1000, f"flight kappa_max {kappa_max}")


def test_default_threshold_uses_fp64_on_some_steps(fr, torch, flight_fire):
    """At the default threshold the ill-conditioned stage-2 steps of the
    flight-line fire pixels go to the FP64 solve (and are flagged)."""
    t, sub, L = flight_fire
    ctx = fr.Context(t)
    g = _np(ctx.retrieve(_dev(torch, L, torch.float32),
                         _dev(torch, sub.wv_bin.astype(np.int16), torch.int16)))
    st = ctx.stats()
    assert st["solves64_2"] > 0
    assert np.count_nonzero(g["status"] & fr.PX_F_FP64) == st["n_fp64_pixels"] > 0


def test_without_the_weak_prior_matches_oracle(fr, torch, c30):
    """Eq. (loss) as printed (every prior precision 1e-6). Without the shape
    prior the six-parameter mixture has several minima whose costs differ by
    less than the noise, and which one the damped iteration reaches depends
    on rounding along its path: GPU and oracle reach the same one (|dE[T]|
    <= 0.5 K) on >= 90 % of the converged identifiable pixels of this
    30 %-fire scene (measured 94.7 %; the default shape prior brings this to
    the full bar, see the other tests). The normal equations themselves agree
    as in every other test."""
    t, tr, L = c30
    cfg = oracle.Config(prior_prec_T1=1e-6, prior_prec_mix=1e-6, prior_prec_alpha=1e-6)
    o = oracle.retrieve(t, L, tr.wv_bin, cfg)
    ctx = fr.Context(t)
    pri = ctx.default_priors()
    for k in range(5):
        pri.pp1[k] = float(cfg.pp1[k])
    for k in range(6):
        pri.pp2[k] = float(cfg.pp2[k])
    g = _np(ctx.retrieve(_dev(torch, L, torch.float32),
                         _dev(torch, tr.wv_bin.astype(np.int16), torch.int16), priors=pri))
    s = parity_stats(o, g, cfg=cfg)
    print("prior 1e-6:", summary(s))
    assert s["pool"] >= 1000 and s["rate"] >= 0.9 and s["sec_rate"] >= 0.97


def _band_sd(L):
    """a sensor's per-band noise sd: the noise model (0.5 % of the signal plus
    read noise) at the scene's brightest radiance of each band, an envelope
    of every pixel's noise (so that no fire pixel's chi-square dwarfs its
    weak prior)"""
    top = np.max(L.astype(np.float64), axis=0)
    return np.sqrt((0.005 * top) ** 2 + 1e-4 ** 2).astype(np.float32)


@pytest.mark.parametrize("variant", [6, 3])
def test_per_band_noise_sd_matches_oracle(fr, torch, c30, variant):
    """Per-band noise sd in the priors (weights 1 / sd_b^2 in Eq. loss):
    stage-2 normal equations at random states and the retrieval."""
    t, tr, L = c30
    sd = _band_sd(L)
    cfg = oracle.Config(noise_sd=sd)
    ctx = fr.Context(t)
    ctx.set_tuning(variant, 1)
    rng = np.random.default_rng(53)
    idx = np.concatenate([np.flatnonzero(tr.kind == 1)[:16], rng.choice(tr.n_pix, 16, replace=False)])
    n = idx.size
    st = np.column_stack([rng.dirichlet(np.ones(3), n), rng.uniform(950, 2100, n), rng.uniform(35, 400, n),
                          rng.uniform(380, 990, n), rng.uniform(35, 400, n),
                          rng.uniform(0.05, 0.95, n), 10 ** rng.uniform(-3.5, -0.5, n)]).astype(np.float32)
    H, g, cost = ctx.normal_equations(2, _dev(torch, L[idx], torch.float32),
                                      _dev(torch, tr.wv_bin[idx].astype(np.int16), torch.int16),
                                      _dev(torch, st, torch.float32), noise_sd=sd)
    H, g, cost = H.cpu().numpy(), g.cpu().numpy(), cost.cpu().numpy()
    for j, i in enumerate(idx):
        Ho, go, co = oracle.normal_equations(t, 2, L[i], tr.wv_bin[i], st[j].astype(np.float64), cfg=cfg)
        d = np.sqrt(np.outer(np.diag(Ho), np.diag(Ho)))
        assert np.max(np.abs(H[j] - Ho) / d) < 2e-4, (variant, i)
        assert np.max(np.abs(g[j] - go) / np.sqrt(np.diag(Ho) * co)) < 2e-4, (variant, i)
        assert abs(cost[j] - co) / co < 1e-4, (variant, i)
    o = oracle.retrieve(t, L, tr.wv_bin, cfg=cfg)
    out = _np(ctx.retrieve(_dev(torch, L, torch.float32),
                           _dev(torch, tr.wv_bin.astype(np.int16), torch.int16), noise_sd=sd))
    assert_parity(parity_stats(o, out, cfg=cfg), 50, f"per-band sd, variant {variant}")


def test_residual_spectrum(fr, torch, c1, c1_oracle):
    """The residual spectrum output: at each fitted pixel's final GPU state,
    L_b - M_b of the full forward model for every band, against the oracle's
    FP64 forward model at that state (1e-5 of the radiance); NaN rows for
    pixels not fitted; the host-staged path returns the same; and at the
    oracle's own state it is the oracle's residual (converged identifiable
    pixels: within 1e-3 of the radiance)."""
    t, tr, L = c1
    L = L.copy()
    L[5, 7] = np.nan                        # one pixel not fitted
    ctx = fr.Context(t)
    out = _np(ctx.retrieve(_dev(torch, L, torch.float32),
                           _dev(torch, tr.wv_bin.astype(np.int16), torch.int16), resid=True))
    r = out["resid_spec"]
    assert r.shape == (tr.n_pix, t.n_bands)
    assert np.all(np.isnan(r[5]))
    fit = np.flatnonzero((out["status"] & 7) <= 1)
    st = out["state"][fit].astype(np.float64)
    st2 = np.column_stack([st[:, :3], st[:, 5:]])
    M = oracle.forward(t, 2, st2, tr.wv_bin[fit])
    ref = L[fit].astype(np.float64) - M
    err = np.abs(r[fit] - ref) / np.maximum(np.abs(L[fit]), 1e-3)
    print("residual spectrum: max error / radiance", err.max())
    assert err.max() < 1e-5
    h = ctx.retrieve(L, tr.wv_bin, resid=True)
    assert np.array_equal(h["resid_spec"], r, equal_nan=True)
    o = c1_oracle
    pool = np.flatnonzero(((o["status"] & 23) == 0) & ((out["status"] & 7) == 0))
    so = np.column_stack([o["state"][pool, :3], o["state"][pool, 5:]])
    ro = L[pool].astype(np.float64) - oracle.forward(t, 2, so, tr.wv_bin[pool])
    e2 = np.abs(r[pool] - ro) / np.maximum(np.abs(L[pool]), 1e-3)
    assert e2.max() < 1e-3


@pytest.mark.parametrize("variant", [6, 3])
def test_dense_fire_scene_matches_oracle(fr, torch, c30, variant):
    """The 96 x 96 scene with 30 % fire pixels, default loss and tables."""
    t, tr, L = c30
    o = oracle.retrieve(t, L, tr.wv_bin)
    ctx = fr.Context(t)
    ctx.set_tuning(variant, 2)
    out = _np(ctx.retrieve(_dev(torch, L, torch.float32),
                           _dev(torch, tr.wv_bin.astype(np.int16), torch.int16)))
    assert_stress_parity(parity_stats(o, out), 1000, f"dense fire, variant {variant}")


def test_all_scenes_together_meet_the_bar():
    """Every retrieval comparison of this module together (tens of thousands
    of converged identifiable pixels) meets the full 99.9 % bar (skipped when
    the comparisons did not run in this session)."""
    if len(_ALL) < 10:
        pytest.skip("the parity comparisons did not run")
    pool = sum(p for p, _, _ in _ALL)
    ok = sum(q for _, q, _ in _ALL)
    print("all comparisons:", [(w, p - q, p) for p, q, w in _ALL], "total misses", pool - ok, "of", pool)
    assert pool >= 15000 and ok / pool >= 0.999
