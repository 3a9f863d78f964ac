"""The paper's Adam solver (Sec. 2.6, Eq. adam) on the GPU against the FP64
oracle's Adam on the same inputs.

Adam runs a fixed number of steps and stops wherever the last step lands;
far from a minimum that end point can depend sharply on rounding: on about
a third of the identifiable fire pixels, the oracle's own end point moves by
more than 0.05 K when every band's model value is perturbed by a relative
1e-6 at each step, and two correct FP64 implementations that only sum in
another order end kelvins apart there. Parity is therefore held in two
forms:
- the first steps of each stage, where the trajectories cannot have
  separated: the GPU state within 2e-4 in every z coordinate of the
  oracle's on >= 99.5 % of the pixels;
- the full 30 + 100 steps on the pixels whose end point is well defined:
  identifiable in the oracle's LM fit (a thermal signal the data fix) and
  stable under the oracle's rounding probe: two seeded runs with the model
  values perturbed by a relative 1e-5 per band and step (the size of the
  GPU's single-precision evaluation error, whose normal equations differ
  from the oracle's by ~8e-6 of their diagonal scale) move E[T] by < 0.05 K
  and alpha by < 1e-4 relative; there the GPU meets the retrieval bar
  (|dE[T]| <= 0.5 K, |d alpha| <= 1e-3 max(alpha, 1e-4)) on >= 99.9 %."""
import numpy as np
import pytest

import oracle
from scenes import config1

pytestmark = pytest.mark.gpu

K = 3


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


def _gpu(fr, torch, t, L, wv, variant=6, **cfg):
    ctx = fr.Context(t, fr.default_config(solver="adam", **cfg))
    ctx.set_tuning(variant, 2)
    out = ctx.retrieve(torch.from_numpy(np.ascontiguousarray(L)).cuda(),
                       torch.from_numpy(wv.astype(np.int16)).cuda())
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    return ctx, g


def _z(state, cfg):
    lo = np.concatenate([np.asarray(cfg.lo1)[:K + 2], np.asarray(cfg.lo2)])
    hi = np.concatenate([np.asarray(cfg.hi1)[:K + 2], np.asarray(cfg.hi2)])
    return 2 * (np.asarray(state, np.float64) - lo) / (hi - lo) - 1


@pytest.mark.parametrize("variant", [6, 3])
@pytest.mark.parametrize("steps", [(1, 0), (2, 0), (5, 0), (0, 1), (0, 3)])
def test_first_adam_steps_match_oracle(fr, torch, c1, variant, steps):
    t, tr, L = c1
    s1, s2 = steps
    ocfg = oracle.Config(n_endm=K, solver="adam", adam_steps1=s1, adam_steps2=s2)
    o = oracle.retrieve(t, L, tr.wv_bin, cfg=ocfg)
    ctx, g = _gpu(fr, torch, t, L, tr.wv_bin, variant, adam_steps1=s1, adam_steps2=s2)
    ok = ((o["status"] & 7) == 0) & ((g["status"] & 7) == 0)
    assert ok.mean() > 0.99
    assert np.all(g["iters"][ok, 0] == s1) and np.all(g["iters"][ok, 1] == s2)
    zo, zg = _z(o["state"][ok], ocfg), _z(g["state"][ok], ocfg)
    dz = np.abs(zg - zo).max(1)
    print(f"steps {steps} variant {variant}: max |dz| {dz.max():.3g}, p99 {np.percentile(dz, 99):.3g}, "
          f"share within 2e-4 {np.mean(dz <= 2e-4):.5f}")
    assert np.mean(dz <= 2e-4) >= 0.995


@pytest.fixture(scope="module")
def c30():
    """A 96 x 96 single-temperature scene with 30 % fire pixels."""
    return config1(seed=21, width=96, height=96, fire_frac=0.3)


@pytest.fixture(scope="module")
def adam_oracle(c30):
    """The oracle's Adam on the dense-fire scene, plus two runs under its
    rounding probe, and its LM fit (for identifiability)."""
    t, tr, L = c30
    runs = [oracle.retrieve(t, L, tr.wv_bin, cfg=oracle.Config(n_endm=K, solver="adam"))]
    for seed in (1, 2):
        runs.append(oracle.retrieve(t, L, tr.wv_bin, cfg=oracle.Config(
            n_endm=K, solver="adam", adam_gnoise=1e-5, adam_gseed=seed)))
    lm = oracle.retrieve(t, L, tr.wv_bin)
    return runs, lm


def _stable(runs):
    o = runs[0]
    st = (o["status"] & 7) == 0
    with np.errstate(invalid="ignore"):
        for p in runs[1:]:
            st &= (p["status"] & 7) == 0
            st &= np.abs(p["ET"] - o["ET"]) < 0.05
            st &= np.abs(p["alpha"] - o["alpha"]) < 1e-4 * np.maximum(o["alpha"], 1e-4)
    return st & np.isfinite(o["ET"])


@pytest.mark.parametrize("variant", [6, 3])
def test_full_adam_run_matches_oracle_where_the_end_point_is_defined(fr, torch, c30, adam_oracle, variant):
    t, tr, L = c30
    runs, lm = adam_oracle
    o = runs[0]
    stable = _stable(runs)
    ident = (lm["status"] & 23) == 0
    ctx, g = _gpu(fr, torch, t, L, tr.wv_bin, variant)
    st = ctx.stats()
    done = (g["status"] & 7) == 0
    assert np.all(g["iters"][done, 0] == 30) and np.all(g["iters"][done, 1] == 100)
    assert st["sum_it1"] == 30 * done.sum() and st["sum_it2"] == 100 * done.sum()
    with np.errstate(invalid="ignore"):
        dT = np.abs(g["ET"].astype(np.float64) - o["ET"])
        da = np.abs(g["alpha"].astype(np.float64) - o["alpha"])
    within = done & (dT <= 0.5) & (da <= 1e-3 * np.maximum(o["alpha"], 1e-4))
    pool = ident & stable
    print(f"variant {variant}: LM-identifiable {ident.sum()}, stable under the probe {stable.sum()}, "
          f"both {pool.sum()}; GPU within the bar on the pool {within[pool].mean():.5f} "
          f"({np.sum(pool & ~within)} misses), on all stable {within[stable].mean():.4f}, "
          f"on identifiable but unstable {within[ident & ~stable].mean():.3f}; "
          f"max |dE[T]| on the pool {np.nanmax(dT[pool]):.3g} K")
    assert pool.sum() >= 500
    assert within[pool].sum() >= 0.999 * pool.sum()


def test_adam_batch_graph_and_static_equal_the_single_fit(fr, torch, c1):
    t, tr, L = c1
    ctx = fr.Context(t, fr.default_config(solver="adam"))
    Ld = torch.from_numpy(L).cuda()
    wd = torch.from_numpy(tr.wv_bin.astype(np.int16)).cuda()
    ref = {k: v.cpu().numpy() for k, v in ctx.retrieve(Ld, wd).items()}
    half = tr.n_pix // 2
    scenes = [(Ld[:half].contiguous(), wd[:half].contiguous()), (Ld[half:].contiguous(), wd[half:].contiguous())]
    outs = ctx.retrieve_batch(scenes)
    static = {k: v.cpu().numpy() for k, v in ctx.retrieve_static(Ld[:half].contiguous(),
                                                                 wd[:half].contiguous()).items()}
    torch.cuda.synchronize()
    for k in ("state", "ET", "alpha", "cov", "cost", "status", "iters"):
        got = np.concatenate([outs[0][k].cpu().numpy(), outs[1][k].cpu().numpy()])
        assert np.array_equal(got, ref[k], equal_nan=True), k
        assert np.array_equal(static[k], ref[k][:half], equal_nan=True), k


def test_adam_config_is_validated(fr, torch, c1):
    t, _, _ = c1
    for bad in (dict(solver=2), dict(solver="adam", adam_lr1=-1.0), dict(solver="adam", adam_clip=0.0),
                dict(solver="adam", adam_beta2=1.0), dict(solver="adam", adam_steps2=-1)):
        with pytest.raises(fr.FireError):
            fr.Context(t, fr.default_config(**bad))
