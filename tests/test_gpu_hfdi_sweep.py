"""The HFDI threshold study of the paper's appendix on the GPU: for a flat
surface (reflectance 0.5) under 1.8 cm of water vapour, the forward model
of a single-temperature fire (T from 300 to 2000 K, gray-body scaling
alpha in {1, 0.5, 0.1}) at several solar zenith angles, the HFDI of every
spectrum (fire_forward + fire_hfdi) against the oracle's, and the minimum
detectable temperature at each threshold (the lowest swept T whose HFDI
meets it) against the same search on the oracle's HFDI."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

T_SWEEP = np.arange(300.0, 2000.5, 1.0)
ALPHAS = (1.0, 0.5, 0.1)
THRESHOLDS = np.round(np.arange(-0.6, 0.601, 0.01), 4)


@pytest.fixture(scope="module")
def fr():
    from paper_2608_07580_b300 import firert
    return firert


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def sweep_states(K=3):
    st = np.zeros((len(ALPHAS) * T_SWEEP.size, K + 2))
    st[:, :K] = 1.0 / K
    st[:, K] = np.repeat(ALPHAS, T_SWEEP.size)
    st[:, K + 1] = np.tile(T_SWEEP, len(ALPHAS))
    return st


def min_detectable(h):
    """[alpha][threshold] lowest swept T with HFDI >= threshold (NaN: none)."""
    h = h.reshape(len(ALPHAS), T_SWEEP.size)
    out = np.full((len(ALPHAS), THRESHOLDS.size), np.nan)
    for a in range(len(ALPHAS)):
        for k, th in enumerate(THRESHOLDS):
            hit = np.flatnonzero(h[a] >= th)
            if hit.size:
                out[a, k] = T_SWEEP[hit[0]]
    return out


@pytest.mark.parametrize("sza", [10.0, 45.0, 85.0])
def test_hfdi_sweep_matches_oracle(fr, torch, sza):
    t = synth.make_tables(cos_sza=math.cos(math.radians(sza)), wv_values=[1.8], flat_reflectance=0.5)
    st = sweep_states()
    wv = np.zeros(st.shape[0], np.uint16)
    ctx = fr.Context(t)
    L = ctx.forward(1, torch.from_numpy(st.astype(np.float32)).cuda(), torch.from_numpy(wv.astype(np.int16)).cuda())
    hg = ctx.hfdi(L).cpu().numpy().astype(np.float64)
    Lo = oracle.forward(t, 1, st, wv).astype(np.float32)
    ho = np.array([oracle.hfdi(t, row) for row in Lo])
    print(f"SZA {sza}: max |dHFDI| {np.abs(hg - ho).max():.3g}")
    assert np.abs(hg - ho).max() < 2e-5
    mg, mo = min_detectable(hg), min_detectable(ho)
    same = (mg == mo) | (np.isnan(mg) & np.isnan(mo))
    near = same | (np.abs(mg - mo) <= 1.0)
    at = THRESHOLDS.tolist().index(-0.1)
    print(f"SZA {sza}: min detectable T at HFDI >= -0.1: GPU {mg[:, at]}, oracle {mo[:, at]}; "
          f"curves equal at {same.mean():.4f} of the points")
    assert near.all() and same.mean() >= 0.99
