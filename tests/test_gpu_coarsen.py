"""Resolution rescaling (the paper's coarsening experiment): a fine scene is
block-averaged 12 x 12 in radiance space, the retrieval runs at both
resolutions, and the Quantile Error Curve QEC(q) = Q_coarse(q) - Q_fine(q)
compares the coarse pixel's moment-matched Gaussian N(E[T], Var[T]) with the
empirical distribution of the fine retrievals' E[T] inside its footprint.

Checked here: the library's block mean against numpy's, the coarse
retrieval against the oracle on every coarse pixel, and the QEC of the
library's two-resolution pipeline against the QEC of the oracle's."""
import numpy as np
import pytest
from scipy.stats import norm

import oracle
import synth
from scenes import NOISE_ABS, NOISE_REL, parity_stats, summary

pytestmark = pytest.mark.gpu

QS = (0.05, 0.10, 0.25, 0.50, 0.75, 0.90, 0.95)
BLK = 12


@pytest.fixture(scope="module")
def scene():
    t = synth.make_tables()
    W, H = 120, 240
    tr = synth.make_config5_fine_truth(seed=4, width=W, height=H, fire_frac=0.2)
    z = synth.noise_normals(4, np.arange(tr.n_pix), t.n_bands)
    Lf = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, z, NOISE_REL, NOISE_ABS)
    cw, ch = synth.block_mean_shape(W, H, BLK)
    Lc = Lf.reshape(ch, BLK, cw, BLK, t.n_bands).mean(axis=(1, 3)).reshape(-1, t.n_bands)
    wvc = tr.wv_bin.reshape(ch, BLK, cw, BLK)[:, 0, :, 0].reshape(-1)
    return t, tr, Lf, Lc.astype(np.float32), wvc, W, H


def _fit(fr, torch, t, L, wv):
    ctx = fr.Context(t)
    out = ctx.retrieve(torch.from_numpy(np.ascontiguousarray(L, np.float32)).cuda(),
                       torch.from_numpy(wv.astype(np.int16)).cuda())
    return {k: v.cpu().numpy() for k, v in out.items()}


def _ident(r):
    return ((r["status"] & 7) == 0) & ((r["status"] & 16) == 0)


def _qec(fine, coarse, W, H, c_ok):
    """Mean over the coarse pixels c_ok (with >= 3 identifiable fine fits in
    the footprint) of Q_coarse(q) - Q_fine(q)."""
    cw, ch = W // BLK, H // BLK
    fET = np.where(_ident(fine), fine["ET"], np.nan).reshape(H, W)[: ch * BLK, : cw * BLK]
    fET = fET.reshape(ch, BLK, cw, BLK).transpose(0, 2, 1, 3).reshape(ch * cw, BLK * BLK)
    rows = []
    for i in np.flatnonzero(c_ok):
        f = fET[i][np.isfinite(fET[i])]
        if f.size < 3:
            continue
        qc = coarse["ET"][i] + coarse["sdT"][i] * norm.ppf(QS)
        rows.append(qc - np.quantile(f, QS))
    return np.mean(rows, axis=0), len(rows)


def test_block_mean_matches_numpy(scene):
    import torch
    from paper_2608_07580_b300 import firert as fr
    t, tr, Lf, Lc, wvc, W, H = scene
    got = fr.block_mean(torch.from_numpy(Lf.astype(np.float32)).cuda(), W, H, t.n_bands, BLK)
    got = got.cpu().numpy()
    ref = Lf.astype(np.float32).astype(np.float64)
    cw, ch = W // BLK, H // BLK
    ref = ref.reshape(ch, BLK, cw, BLK, t.n_bands).mean(axis=(1, 3)).reshape(-1, t.n_bands)
    # 144 fp32 additions of positive terms: at most 144 ulp-halvings of the
    # running sum, 144 * 2^-24 = 8.6e-6 relative
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-6)) < 8.6e-6


@pytest.fixture(scope="module")
def coarse_scene():
    """A 480 x 720 fine scene (20 % fire sub-pixels, each its own
    temperature) block-averaged 12 x 12 into 40 x 60 coarse pixels whose
    radiance carries a temperature mixture with 12x less noise."""
    t = synth.make_tables()
    W, H = 480, 720
    tr = synth.make_config5_fine_truth(seed=14, width=W, height=H, fire_frac=0.2)
    z = synth.noise_normals(14, np.arange(tr.n_pix), t.n_bands)
    Lf = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, z, NOISE_REL, NOISE_ABS)
    cw, ch = synth.block_mean_shape(W, H, BLK)
    Lc = Lf.reshape(ch, BLK, cw, BLK, t.n_bands).mean(axis=(1, 3)).reshape(-1, t.n_bands)
    wvc = tr.wv_bin.reshape(ch, BLK, cw, BLK)[:, 0, :, 0].reshape(-1)
    return t, Lc.astype(np.float32), wvc


def test_coarse_retrieval_matches_oracle(coarse_scene):
    import torch
    from paper_2608_07580_b300 import firert as fr
    t, Lc, wvc = coarse_scene
    o = oracle.retrieve(t, Lc, wvc)
    g = _fit(fr, torch, t, Lc, wvc)
    s = parity_stats(o, g)
    print("coarse parity:", summary(s))
    assert s["pool"] >= 200
    assert s["rate"] >= 0.999 and s["sec_rate"] >= 0.999, summary(s)


def test_qec_of_library_pipeline_matches_oracle_pipeline(scene):
    import torch
    from paper_2608_07580_b300 import firert as fr
    t, tr, Lf, Lc, wvc, W, H = scene
    gf, gc = _fit(fr, torch, t, Lf, tr.wv_bin), _fit(fr, torch, t, Lc, wvc)
    of, oc = oracle.retrieve(t, Lf, tr.wv_bin), oracle.retrieve(t, Lc, wvc)
    both = _ident(gc) & _ident(oc)          # the same coarse pixels on both sides
    gq, gn = _qec(gf, gc, W, H, both)
    oq, on = _qec(of, oc, W, H, both)
    print("QEC library", np.round(gq, 1), "over", gn, "px; oracle", np.round(oq, 1), "over", on, "px")
    assert gn >= 10 and abs(gn - on) <= 2
    assert np.all(np.abs(gq - oq) <= 5.0)
