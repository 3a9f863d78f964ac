"""The water-vapour presolve (Sec. 2.5) on the GPU against the oracle's:
the depth table, every pixel's depth and every block's bin bit for bit
(the decision chain is single precision on both sides), ragged images,
pixels without a depth, saturated bands, block sizes, and the retrieval
driven by the presolved bins."""
import numpy as np
import pytest

import oracle
import synth
from scenes import NOISE_ABS, NOISE_REL, parity_stats, summary

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
def fine():
    """240 x 120 fine pixels of the coarsened scene's truth (water vapour
    constant per 12 x 12 block, 5 % fire sub-pixels), noisy radiance."""
    t = synth.make_tables()
    tr = synth.make_config5_fine_truth(seed=4, width=240, height=120)
    z = synth.noise_normals(4, np.arange(tr.n_pix), t.n_bands)
    L = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, z, NOISE_REL, NOISE_ABS)
    return t, tr, L


def _gpu(fr, torch, t, L, W, H, block=12, lams=None):
    ctx = fr.Context(t)
    bins, depth = ctx.wv_presolve(torch.from_numpy(np.ascontiguousarray(L)).cuda(), W, H, block=block,
                                  lams=lams, depth=True)
    torch.cuda.synchronize()
    return ctx, bins.cpu().numpy().view(np.uint16), depth.cpu().numpy()


def test_depth_table_matches_oracle(fr, fine):
    t, _, _ = fine
    ctx = fr.Context(t)
    assert np.array_equal(ctx.wv_depth_table(), oracle.wv_depth_table(t))
    lams = (880.0, 945.0, 1020.0)
    assert np.array_equal(ctx.wv_depth_table(lams), oracle.wv_depth_table(t, lams))


def test_presolve_matches_oracle_bit_for_bit(fr, torch, fine):
    t, tr, L = fine
    _, bins, depth = _gpu(fr, torch, t, L, 240, 120)
    ob, od = oracle.wv_presolve(t, L, 240, 120)
    assert np.array_equal(depth, od, equal_nan=True)
    assert np.array_equal(bins, ob)
    blocks = bins.reshape(10, 12, 20, 12)[:, 0, :, 0] == tr.wv_bin.reshape(10, 12, 20, 12)[:, 0, :, 0]
    print("blocks with the truth's bin:", blocks.mean())
    assert blocks.mean() >= 0.95


@pytest.mark.parametrize("block", [1, 5, 12, 16])
def test_ragged_image_gaps_and_block_sizes(fr, torch, block):
    t = synth.make_tables()
    rng = np.random.default_rng(block)
    W, H = 61, 37
    tr = synth.make_config1_truth(seed=block, width=W, height=H, fire_frac=0.05)
    L = oracle.forward(t, 1, tr.state1(), tr.wv_bin).astype(np.float32)
    L *= (1 + 0.005 * rng.standard_normal(L.shape)).astype(np.float32)
    lam = np.asarray(t.wavelength_nm)
    c = int(np.argmin(np.abs(lam - 940.0)))
    L[rng.choice(W * H, 60, replace=False), c] = np.nan
    L[:block, :] = np.where(np.arange(L.shape[1]) % 7 == 0, np.inf, L[:block, :])
    _, bins, depth = _gpu(fr, torch, t, L, W, H, block=block)
    ob, od = oracle.wv_presolve(t, L, W, H, block=block)
    assert np.array_equal(depth, od, equal_nan=True)
    assert np.array_equal(bins, ob)


def test_saturated_bands_and_empty_blocks(fr, torch):
    t = synth.make_tables(sat_level=25.0)
    tr = synth.make_config1_truth(seed=2, width=36, height=24, fire_frac=0.2)
    L = oracle.forward(t, 1, tr.state1(), tr.wv_bin).astype(np.float32)
    lam = np.asarray(t.wavelength_nm)
    lo = int(np.argmin(np.abs(lam - 870.0)))
    L[::3, lo] = 30.0                                   # above the saturation level
    L[np.arange(36 * 24) % 36 < 12, :] = np.nan          # the left block column has no depth
    _, bins, depth = _gpu(fr, torch, t, L, 36, 24)
    ob, od = oracle.wv_presolve(t, L, 36, 24)
    assert np.array_equal(depth, od, equal_nan=True)
    assert np.array_equal(bins, ob)
    assert np.all(bins.reshape(24, 36)[:, :12] == 0xFFFF)


def test_presolve_rejects_bad_arguments(fr, torch):
    t = synth.make_tables()
    ctx = fr.Context(t)
    L = torch.zeros((24, t.n_bands), dtype=torch.float32, device="cuda")
    for block in (0, 17):
        with pytest.raises(fr.FireError):
            ctx.wv_presolve(L, 6, 4, block=block)
    with pytest.raises(fr.FireError):
        ctx.wv_presolve(L, 6, 4, lams=(1010.0, 940.0, 870.0))      # shoulders out of order
    out = ctx.wv_presolve(L[:0], 0, 0)
    assert out.numel() == 0


def test_retrieval_on_presolved_bins_matches_oracle(fr, torch, fine):
    """The presolved bins drive the fit: GPU presolve + GPU fit against the
    oracle's presolve + oracle fit, on the fire pixels and a sample of the
    others (the bins are identical, so this is the retrieval's own parity)."""
    t, tr, L = fine
    ctx, bins, _ = _gpu(fr, torch, t, L, 240, 120)
    ob, _ = oracle.wv_presolve(t, L, 240, 120)
    rng = np.random.default_rng(1)
    idx = np.sort(np.concatenate([np.flatnonzero(tr.kind == 1),
                                  rng.choice(np.flatnonzero(tr.kind == 0), 1500, replace=False)]))
    g = ctx.retrieve(torch.from_numpy(L[idx]).cuda(), torch.from_numpy(bins[idx].astype(np.int16)).cuda())
    g = {k: v.cpu().numpy() for k, v in g.items()}
    o = oracle.retrieve(t, L[idx], ob[idx])
    s = parity_stats(o, g)
    print("retrieval on presolved bins:", summary(s))
    assert s["pool"] >= 200 and s["rate"] >= 0.999
