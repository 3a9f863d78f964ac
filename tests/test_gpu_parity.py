"""GPU path (C-ABI through the ctypes binding) against the FP64 oracle on the
same seeded inputs: forward model, full per-pixel retrieval (config 1:
64x64x284), ragged and degenerate cases, host-staged path, determinism.

Parity bar (per converged, identifiable pixel): |dE[T]| <= 0.5 K and
|d alpha| <= 1e-3 * max(alpha_oracle, 1e-4), for >= 99.9 % of the pool."""
import numpy as np
import pytest

import oracle
import synth
from scenes import NOISE_ABS, NOISE_REL, config1, parity_stats

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


def test_config1_parity(fr, torch, c1, c1_oracle):
    t, tr, L = c1
    ctx, g = _retrieve(fr, torch, t, L, tr.wv_bin)
    s = parity_stats(c1_oracle, g)
    print("config1 parity:", {k: v for k, v in s.items() if k != "fail_idx"},
          "fail:", s["fail_idx"][:10])
    st = ctx.stats()
    print("stats:", st)
    assert st["n_pixels"] == tr.n_pix
    assert s["pool"] >= 0.8 * s["oracle_conv_ident"]
    assert s["rate"] >= 0.999
    # the per-pixel outcome codes agree wherever the oracle's is not MAXITER
    go, oo = g["status"] & 7, c1_oracle["status"] & 7
    assert np.mean(go == oo) > 0.95


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
    print("given start:", {k: v for k, v in s.items() if k != "fail_idx"})
    assert s["rate"] >= 0.99 and s["pool"] > 50


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
    return config1(seed=7, width=48, height=48, n_bands=160, n_tgrid=40)


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
    print(f"variant {variant}:", {k: v for k, v in s.items() if k != "fail_idx"})
    assert s["pool"] >= 0.8 * s["oracle_conv_ident"] and s["pool"] >= 15
    assert s["rate"] >= 0.97


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
    tr = synth.make_config1_truth(seed=11, width=48, height=48, n_endm=5)
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
    print(f"K=5 variant {variant}:", {k: v for k, v in s.items() if k != "fail_idx"})
    assert s["pool"] >= 0.8 * s["oracle_conv_ident"] and s["pool"] >= 15
    assert s["rate"] >= 0.97


def test_path_reflectance_retrieval_matches_oracle(fr, torch):
    """Tables with path reflectance and spherical albedo (the full solar term
    of Eq. solar, with its denominator 1 - S rho): stage-1 normal equations at
    random states and the retrieval of a 48 x 48 scene against the oracle."""
    t = synth.make_tables(path_reflectance=True)
    tr = synth.make_config1_truth(seed=13, width=48, height=48)
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
    print("path reflectance:", {k: v for k, v in s.items() if k != "fail_idx"})
    assert s["pool"] >= 0.8 * s["oracle_conv_ident"] and s["pool"] >= 15
    assert s["rate"] >= 0.97


@pytest.mark.parametrize("variant", [3, 6])
def test_noise_weighted_loss_matches_oracle(fr, torch, c1, variant):
    """The noise-weighted loss (weights 1 / sd_b^2 of the noise model) on both
    sides: stage-2 normal equations at random states and the retrieval."""
    t, tr, L = c1
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
    s = parity_stats(o, out)
    print(f"weighted, variant {variant}:", {k: v for k, v in s.items() if k != "fail_idx"})
    assert s["pool"] >= 0.8 * s["oracle_conv_ident"] and s["pool"] >= 15
    assert s["rate"] >= 0.97
