"""Batched uneven scenes in one persistent launch, CUDA-graph replay of that
launch, and the launch-shape autotuner. Each pixel's fit is the same
arithmetic whichever scene table, claim size or graph it runs under, so the
batched outputs equal, bit for bit, those of fitting the scenes one by one."""
import numpy as np
import pytest

import oracle
import synth
from scenes import config1, config2_subset, parity_stats, summary

pytestmark = pytest.mark.gpu

KEYS = ("state", "ET", "sdT", "alpha", "cov", "var_ET", "cost", "rms", "hfdi", "status", "iters")


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


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _np(d):
    return {k: v.cpu().numpy() for k, v in d.items() if hasattr(v, "cpu")}


def _same(a, b):
    for k in KEYS:
        if a[k].dtype.kind == "f":
            assert np.array_equal(a[k], b[k], equal_nan=True), k
        else:
            assert np.array_equal(a[k], b[k]), k


def _split(n, sizes):
    edges = np.cumsum([0] + list(sizes))
    assert edges[-1] <= n
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:])]


def test_batch_equals_scene_by_scene(fr, torch, c1):
    t, tr, L = c1
    ctx = fr.Context(t)
    Ld = _dev(torch, L, torch.float32)
    wd = _dev(torch, tr.wv_bin.astype(np.int16), torch.int16)
    whole = _np(ctx.retrieve(Ld, wd))
    parts = _split(tr.n_pix, [0, 1, 37, 500, 2048, 3, tr.n_pix - 2589])
    scenes = [(Ld[a:b], wd[a:b]) for a, b in parts]
    outs = ctx.retrieve_batch(scenes)
    torch.cuda.synchronize()
    assert ctx.stats()["n_pixels"] == tr.n_pix
    for (a, b), o in zip(parts, outs):
        o = _np(o)
        _same({k: whole[k][a:b] for k in KEYS}, o)


def test_batch_hfdi_gate_and_rejects_learned_start(fr, torch, c1):
    t, tr, L = c1
    ctx = fr.Context(t)
    Ld = _dev(torch, L, torch.float32)
    wd = _dev(torch, tr.wv_bin.astype(np.int16), torch.int16)
    whole = _np(ctx.retrieve(Ld, wd, gate_hfdi=True))
    parts = _split(tr.n_pix, [1000, 96, tr.n_pix - 1096])
    outs = ctx.retrieve_batch([(Ld[a:b], wd[a:b]) for a, b in parts], gate_hfdi=True)
    torch.cuda.synchronize()
    for (a, b), o in zip(parts, outs):
        _same({k: whole[k][a:b] for k in KEYS}, _np(o))
    pri = ctx.default_priors()
    pri.init_mode = fr.FIRE_INIT_MLP
    with pytest.raises(fr.FireError):
        ctx.retrieve_batch([(Ld[:10], wd[:10])], priors=pri)


def test_graph_replay_follows_new_inputs(fr, torch, c1):
    t, tr, L = c1
    ctx = fr.Context(t)
    n = tr.n_pix
    parts = _split(n, [700, 1, n - 701])
    Lbuf = _dev(torch, L, torch.float32)
    wbuf = _dev(torch, tr.wv_bin.astype(np.int16), torch.int16)
    scenes = [(Lbuf[a:b], wbuf[a:b]) for a, b in parts]
    outs = [ctx.alloc_outputs(b - a) for a, b in parts]
    g = ctx.capture_batch(scenes, outs)
    # new inputs in the same buffers: the scene reversed pixel-wise
    perm = np.arange(n)[::-1].copy()
    Lbuf.copy_(_dev(torch, L[perm], torch.float32))
    wbuf.copy_(_dev(torch, tr.wv_bin[perm].astype(np.int16), torch.int16))
    for _ in range(2):                                   # replays are repeatable
        g.launch()
        torch.cuda.synchronize()
        got = [_np(o) for o in outs]
        ref = _np(fr.Context(t).retrieve(_dev(torch, L[perm], torch.float32),
                                         _dev(torch, tr.wv_bin[perm].astype(np.int16), torch.int16)))
        for (a, b), o in zip(parts, got):
            _same({k: ref[k][a:b] for k in KEYS}, o)


def test_claim_size_does_not_change_results(fr, torch, c1):
    t, tr, L = c1
    ctx = fr.Context(t)
    Ld = _dev(torch, L[:1500], torch.float32)
    wd = _dev(torch, tr.wv_bin[:1500].astype(np.int16), torch.int16)
    for variant in (0, 6):          # FP32 stage 2 with 32 lanes; tensor-core stage 2
        base = None
        for claim in (1, 2, 8, 32):
            ctx.set_tuning(variant, claim)
            o = _np(ctx.retrieve(Ld, wd))
            if base is None:
                base = o
            else:
                _same(base, o)
    with pytest.raises(fr.FireError):
        ctx.set_tuning(9, 4)


def test_autotune_picks_a_valid_shape_and_keeps_parity(fr, torch, c1):
    t, tr, L = c1
    ctx = fr.Context(t)
    Ld = _dev(torch, L, torch.float32)
    wd = _dev(torch, tr.wv_bin.astype(np.int16), torch.int16)
    best = ctx.autotune(Ld, wd)
    print("autotune:", best)
    assert best["variant"] in range(9) and best["claim"] in (1, 2, 4, 8) and best["ms"] > 0
    o = oracle.retrieve(t, L, tr.wv_bin)
    for variant in range(9):
        ctx.set_tuning(variant, 4)
        g = _np(ctx.retrieve(Ld, wd))
        s = parity_stats(o, g)
        print(variant, summary(s))
        assert s["pool"] >= 100
        assert s["rate"] >= 0.999 and s["sec_rate"] >= 0.999, (variant, summary(s))


def test_batch_against_the_oracle(fr, torch):
    """Uneven scenes in one batched launch, each compared with the oracle:
    a 64 x 64 single-temperature scene and a flight-line sample (fire
    pixels and others) split into three scenes of 1, 1,999 and 3,000 pixels."""
    t = synth.make_tables()
    t1, tr1, L1 = config1(seed=3)
    tr2 = synth.make_config2_truth(seed=1)
    rng = np.random.default_rng(29)
    idx = np.sort(np.concatenate([rng.choice(np.flatnonzero(tr2.kind == 2), 6000, replace=False),
                                  rng.choice(np.flatnonzero(tr2.kind == 0), 1000, replace=False)]))
    sub, L2 = config2_subset(idx, tr2, t)
    parts = [(L1, tr1.wv_bin), (L2[:1], sub.wv_bin[:1]), (L2[1:2000], sub.wv_bin[1:2000]),
             (L2[2000:], sub.wv_bin[2000:])]
    ctx = fr.Context(t)
    outs = ctx.retrieve_batch([(_dev(torch, a, torch.float32), _dev(torch, w.astype(np.int16), torch.int16))
                               for a, w in parts])
    torch.cuda.synchronize()
    o1 = oracle.retrieve(t, L1, tr1.wv_bin)
    o2 = oracle.retrieve(t, L2, sub.wv_bin)
    s1 = parity_stats(o1, _np(outs[0]))
    g2 = [_np(o) for o in outs[1:]]
    cat = {k: np.concatenate([g[k] for g in g2]) for k in g2[0]}
    s2 = parity_stats(o2, cat)
    print("batch scene 0:", summary(s1), "batch flight sample:", summary(s2))
    assert s1["pool"] >= 100 and s2["pool"] >= 1000
    for s in (s1, s2):
        assert s["rate"] >= 0.999 and s["sec_rate"] >= 0.999, summary(s)


def test_tensor_core_shape_falls_back_beyond_its_tables(fr, torch):
    """With 512 bands the stage-2 window holds 384 bands, beyond the
    tensor-core product's two band tiles: launch shape 6 then runs the FP32
    stage 2 with 16 lanes per pixel, so its results equal shape 3's bit for
    bit, and so do its normal equations."""
    t = synth.make_tables(n_bands=512)
    tr = synth.make_config1_truth(seed=9, width=24, height=16, fire_frac=0.3)
    z = synth.noise_normals(9, np.arange(tr.n_pix), t.n_bands)
    L = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, z, 0.005, 1e-4)
    ctx = fr.Context(t)
    assert ctx.window_bands()[3] > 256
    Ld = _dev(torch, L, torch.float32)
    wd = _dev(torch, tr.wv_bin.astype(np.int16), torch.int16)
    outs = []
    for variant in (3, 6):
        ctx.set_tuning(variant, 1)
        outs.append(_np(ctx.retrieve(Ld, wd)))
    _same(outs[0], outs[1])
    assert np.isfinite(outs[0]["ET"][(outs[0]["status"] & 7) == 0]).any()
