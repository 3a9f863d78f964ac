"""The injection experiment of Sec. 2.8 / 3.1 (Eq. inject) on the GPU: the
injection kernel against the oracle's, then the retrieval of the injected
spectra against the oracle's retrieval of its own injected spectra, and
E[T] against the injected temperatures (RMSE, MAE, R^2, printed beside the
paper's 41.8 K, 34.1 K, 0.987 on its own data)."""
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
def experiment():
    t = synth.make_tables()
    tr, alpha, T = synth.make_injection_experiment(seed=7, n=4096)
    z = synth.noise_normals(7, np.arange(tr.n_pix), t.n_bands)
    bg = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, z, NOISE_REL, NOISE_ABS)
    return t, tr, alpha.astype(np.float32), T.astype(np.float32), bg


def _stats(ET, T, m):
    e = ET[m] - T[m]
    return (float(np.sqrt(np.mean(e ** 2))), float(np.mean(np.abs(e))),
            float(1 - np.sum(e ** 2) / np.sum((T[m] - T[m].mean()) ** 2)))


def test_injection_kernel_matches_oracle(fr, torch, experiment):
    t, tr, alpha, T, bg = experiment
    ctx = fr.Context(t)
    dev = lambda a, d: torch.from_numpy(np.ascontiguousarray(a)).to(d).cuda()  # noqa: E731
    got = ctx.inject(dev(bg, torch.float32), dev(tr.wv_bin.astype(np.int16), torch.int16),
                     dev(alpha, torch.float32), dev(T, torch.float32)).cpu().numpy()
    ref = oracle.inject(t, bg, tr.wv_bin, alpha.astype(np.float64), T.astype(np.float64))
    rel = np.abs(got.astype(np.float64) - ref) / np.maximum(np.abs(ref), 1e-12)
    print("injection: max relative difference", rel.max(), "share bit-equal", np.mean(got == ref))
    assert rel.max() < 2e-7
    wv = tr.wv_bin.astype(np.int16).copy()
    wv[:3] = t.n_wv                                  # invalid bins give NaN rows
    got = ctx.inject(dev(bg, torch.float32), dev(wv, torch.int16), dev(alpha, torch.float32),
                     dev(T, torch.float32)).cpu().numpy()
    assert np.all(np.isnan(got[:3])) and np.all(np.isfinite(got[3:]))


@pytest.mark.parametrize("solver", ["lm"])
def test_injected_spectra_retrieval_matches_oracle(fr, torch, experiment, solver):
    t, tr, alpha, T, bg = experiment
    ctx = fr.Context(t)
    dev = lambda a, d: torch.from_numpy(np.ascontiguousarray(a)).to(d).cuda()  # noqa: E731
    wv = dev(tr.wv_bin.astype(np.int16), torch.int16)
    L = ctx.inject(dev(bg, torch.float32), wv, dev(alpha, torch.float32), dev(T, torch.float32))
    g = {k: v.cpu().numpy() for k, v in ctx.retrieve(L, wv).items()}
    Lo = oracle.inject(t, bg, tr.wv_bin, alpha.astype(np.float64), T.astype(np.float64))
    o = oracle.retrieve(t, Lo, tr.wv_bin)
    s = parity_stats(o, g)
    print("injected spectra, GPU against oracle:", summary(s))
    assert s["pool"] >= 1000 and s["rate"] >= 0.999
    T64 = T.astype(np.float64)
    conv = ((g["status"] & 7) == 0) & np.isfinite(g["ET"])
    ident = (g["status"] & 23) == 0
    for name, m in (("converged", conv), ("identifiable", ident)):
        rmse, mae, r2 = _stats(g["ET"].astype(np.float64), T64, m)
        print(f"E[T] against the injected T, {name} ({m.sum()} of {m.size}): RMSE {rmse:.1f} K, "
              f"MAE {mae:.1f} K, R^2 {r2:.3f} (paper, on its own data: 41.8 K, 34.1 K, 0.987)")
    rmse, mae, r2 = _stats(g["ET"].astype(np.float64), T64, ident)
    assert r2 > 0.9
