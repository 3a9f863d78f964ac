"""Pins of the oracle's Adam solver (Sec. 2.6, Eq. adam) against values that
do not come from its own gradient code: the first two Adam steps of each
stage formed here in closed form from central differences of Eq. (loss)
evaluated with the oracle's forward model, the global-norm clip, a fixed
variable, and the box / simplex invariants after the full step counts."""
import numpy as np
import pytest

import oracle
import synth
from scenes import NOISE_ABS, NOISE_REL

K = 3
B1, B2, EPS = 0.9, 0.999, 1e-8


@pytest.fixture(scope="module")
def scene():
    t = synth.make_tables()
    tr = synth.make_config1_truth(seed=5, width=24, height=1, fire_frac=1.0)
    z = synth.noise_normals(5, np.arange(tr.n_pix), t.n_bands)
    L = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, z, NOISE_REL, NOISE_ABS)
    return t, tr, L


def _window(t, lo_hi):
    lam = np.asarray(t.wavelength_nm, np.float64)
    return np.zeros(lam.size, bool) | ((lam >= lo_hi[0]) & (lam <= lo_hi[1]))


def _loss(t, stage, L_obs, wv, xs, x, cfg):
    """Eq. (loss) of one stage, unweighted, from the oracle's forward model:
    stage 1 state [x_surf, a1, T1]; stage 2 [mu_h, s_h, mu_s, s_s, eta, a]
    with the surface fractions xs."""
    if stage == 1:
        M = oracle.forward(t, 1, x[None, :], np.array([wv]))[0]
        win = _window(t, cfg.win1)
    else:
        M = oracle.forward(t, 2, np.concatenate([xs, x])[None, :], np.array([wv]))[0]
        win = _window(t, cfg.win2h) | _window(t, cfg.win2s)
    r = L_obs.astype(np.float64) - M
    return float(np.sum(r[win] ** 2))


def _bounds(cfg, stage):
    return (np.asarray(cfg.lo1, float)[:K + 2], np.asarray(cfg.hi1, float)[:K + 2]) if stage == 1 \
        else (np.asarray(cfg.lo2, float), np.asarray(cfg.hi2, float))


def _fd_grad_z(t, stage, L_obs, wv, xs, x, cfg, h=1e-6):
    lo, hi = _bounds(cfg, stage)
    s = 0.5 * (hi - lo)
    g = np.zeros(x.size)
    for i in range(x.size):
        if not s[i] > 0:
            continue
        xp, xm = x.copy(), x.copy()
        xp[i] += s[i] * h
        xm[i] -= s[i] * h
        g[i] = (_loss(t, stage, L_obs, wv, xs, xp, cfg) - _loss(t, stage, L_obs, wv, xs, xm, cfg)) / (2 * h)
    return g


def _project_simplex(v):
    """Euclidean projection onto the unit simplex by bisection on the shift
    (an independent route to the same point as the sort-based rule)."""
    lo, hi = v.min() - 1.0, v.max()
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.maximum(v - mid, 0).sum() > 1.0:
            lo = mid
        else:
            hi = mid
    return np.maximum(v - 0.5 * (lo + hi), 0.0)


def _adam_steps(t, stage, L_obs, wv, xs, x0, cfg, n, lr):
    """n Adam steps of Eq. (adam) on the FD gradient (test-side closed form)."""
    lo, hi = _bounds(cfg, stage)
    s = 0.5 * (hi - lo)
    x = x0.copy()
    m = np.zeros(x.size)
    v = np.zeros(x.size)
    for k in range(1, n + 1):
        g = _fd_grad_z(t, stage, L_obs, wv, xs, x, cfg)
        nrm = np.linalg.norm(g)
        g = g * min(1.0, cfg.adam_clip / nrm) if nrm > 0 else g
        m = B1 * m + (1 - B1) * g
        v = B2 * v + (1 - B2) * g * g
        z = np.where(s > 0, (x - lo) / np.where(s > 0, s, 1) - 1, 0.0)
        z = np.clip(z - lr * (m / (1 - B1 ** k)) / (np.sqrt(v / (1 - B2 ** k)) + EPS), -1, 1)
        x = np.where(s > 0, lo + s * (z + 1), x)
        if stage == 1:
            x[:K] = _project_simplex(x[:K])
    return x, g


def _start(tr, i):
    """A start inside the boxes, away from the truth: fractions 0.5/0.3/0.2,
    alpha1 0.02, T1 900 K; mixture 1200/150/600/80, eta 0.6, alpha 0.02."""
    return np.array([0.5, 0.3, 0.2, 0.02, 900.0, 1200.0, 150.0, 600.0, 80.0, 0.6, 0.02])


@pytest.mark.parametrize("n_steps", [1, 2])
def test_stage1_adam_steps_match_closed_form(scene, n_steps):
    t, tr, L = scene
    cfg = oracle.Config(n_endm=K, solver="adam", adam_steps1=n_steps, adam_steps2=0)
    idx = np.arange(6)
    init = np.stack([_start(tr, i) for i in idx])
    o = oracle.retrieve(t, L[idx], tr.wv_bin[idx], cfg=cfg, init_state=init)
    for j, i in enumerate(idx):
        x_exp, g = _adam_steps(t, 1, L[i], tr.wv_bin[i], None, init[j, :K + 2].copy(), cfg, n_steps,
                               cfg.adam_lr1)
        assert np.all(np.abs(g) > 1e-9), g      # every sign resolved by the differences
        assert np.allclose(o["state"][j, :K + 2], x_exp, rtol=0, atol=1e-7 * np.array([1, 1, 1, 1, 1000])), \
            (i, o["state"][j, :K + 2], x_exp)
        assert o["it1"][j] == n_steps


@pytest.mark.parametrize("n_steps", [1, 2])
def test_stage2_adam_steps_match_closed_form(scene, n_steps):
    t, tr, L = scene
    cfg = oracle.Config(n_endm=K, solver="adam", adam_steps1=0, adam_steps2=n_steps)
    idx = np.arange(6, 12)
    init = np.stack([_start(tr, i) for i in idx])
    o = oracle.retrieve(t, L[idx], tr.wv_bin[idx], cfg=cfg, init_state=init)
    for j, i in enumerate(idx):
        xs = o["state"][j, :K]                   # stage 1 took no step: the projected start
        assert np.allclose(xs, _project_simplex(init[j, :K]), atol=1e-12)
        x_exp, _ = _adam_steps(t, 2, L[i], tr.wv_bin[i], xs, init[j, K + 2:].copy(), cfg, n_steps,
                               cfg.adam_lr2)
        scale = np.array([1000, 100, 1000, 100, 1, 1]) * 1e-7
        assert np.all(np.abs(o["state"][j, K + 2:] - x_exp) <= scale), (i, o["state"][j, K + 2:], x_exp)
        assert o["it2"][j] == n_steps


def test_first_step_is_lr_times_the_gradient_sign(scene):
    """At t = 1 the bias-corrected ratio is g / (|g| + eps): every free
    coordinate moves by lr in z against its gradient's sign (before the
    projection), whatever the gradient's size."""
    t, tr, L = scene
    cfg = oracle.Config(n_endm=K, solver="adam", adam_steps1=1, adam_steps2=0)
    lo, hi = _bounds(cfg, 1)
    i = 3
    x0 = _start(tr, i)[:K + 2]
    g = _fd_grad_z(t, 1, L[i], tr.wv_bin[i], None, x0, cfg)
    o = oracle.retrieve(t, L[i:i + 1], tr.wv_bin[i:i + 1], cfg=cfg, init_state=_start(tr, i)[None])
    z0 = 2 * (x0 - lo) / (hi - lo) - 1
    z1 = 2 * (o["state"][0, :K + 2] - lo) / (hi - lo) - 1
    gc = g * min(1.0, cfg.adam_clip / np.linalg.norm(g))
    # alpha1 and T1 are not projected: -lr gc / (|gc| + eps), i.e. -lr sign(g)
    # to within eps / |gc|
    assert np.allclose((z1 - z0)[K:], -cfg.adam_lr1 * gc[K:] / (np.abs(gc[K:]) + EPS), atol=1e-9)
    assert np.allclose(np.abs(z1 - z0)[K:], cfg.adam_lr1, rtol=1e-3)


@pytest.mark.parametrize("clip", [1e-30, 2e-8, 1.0, 1e30])
def test_global_norm_clip_scales_the_gradient_before_the_moments(scene, clip):
    """The clip rescales the whole gradient to norm <= clip before the
    moments, so the first step of a coordinate is lr gc / (|gc| + eps) with
    gc = g min(1, clip / ||g||): nothing moves at a clip far below eps, the
    step shrinks where |gc| is comparable to eps, and a huge clip is no clip."""
    t, tr, L = scene
    i = 1
    cfg = oracle.Config(n_endm=K, solver="adam", adam_steps1=1, adam_steps2=0, adam_clip=clip)
    lo, hi = _bounds(cfg, 1)
    x0 = _start(tr, i)[:K + 2]
    g = _fd_grad_z(t, 1, L[i], tr.wv_bin[i], None, x0, cfg)
    o = oracle.retrieve(t, L[i:i + 1], tr.wv_bin[i:i + 1], cfg=cfg, init_state=_start(tr, i)[None])
    z0 = 2 * (x0 - lo) / (hi - lo) - 1
    z1 = 2 * (o["state"][0, :K + 2] - lo) / (hi - lo) - 1
    gc = g * min(1.0, clip / np.linalg.norm(g))
    expect = -cfg.adam_lr1 * gc[K:] / (np.abs(gc[K:]) + EPS)
    assert np.allclose((z1 - z0)[K:], expect, rtol=1e-6, atol=1e-12), ((z1 - z0)[K:], expect)
    if clip == 1e-30:
        assert np.all(np.abs(z1 - z0) < 1e-12)


def test_fixed_variable_does_not_move_and_box_and_simplex_hold(scene):
    t, tr, L = scene
    cfg = oracle.Config(n_endm=K, solver="adam")
    cfg.lo1 = cfg.lo1.copy()
    cfg.hi1 = cfg.hi1.copy()
    cfg.lo1[K + 1] = cfg.hi1[K + 1] = cfg.init_T1    # T1 held at its start, 800 K
    o = oracle.retrieve(t, L, tr.wv_bin, cfg=cfg)
    ok = (o["status"] & 7) == 0
    assert ok.all()
    assert np.all(o["state"][:, K + 1] == cfg.init_T1)
    assert np.all(o["it1"] == cfg.adam_steps1) and np.all(o["it2"] == cfg.adam_steps2)
    full = oracle.retrieve(t, L, tr.wv_bin, cfg=oracle.Config(n_endm=K, solver="adam"))
    st = full["state"]
    assert np.allclose(st[:, :K].sum(1), 1.0, atol=1e-12) and np.all(st[:, :K] >= 0)
    lo2, hi2 = np.asarray(oracle.Config(n_endm=K).lo2), np.asarray(oracle.Config(n_endm=K).hi2)
    assert np.all(st[:, K + 2:] >= lo2 - 1e-9) and np.all(st[:, K + 2:] <= hi2 + 1e-9)
    assert np.all((st[:, K] >= 0) & (st[:, K] <= 1)) and np.all((st[:, K + 1] >= 350) & (st[:, K + 1] <= 2200))


def test_adam_ignores_the_prior(scene):
    """The paper's Adam minimises Eq. (loss) as printed: the prior
    precisions change nothing."""
    t, tr, L = scene
    a = oracle.retrieve(t, L[:4], tr.wv_bin[:4], cfg=oracle.Config(n_endm=K, solver="adam"))
    b = oracle.retrieve(t, L[:4], tr.wv_bin[:4],
                        cfg=oracle.Config(n_endm=K, solver="adam", prior_prec_T1=50.0,
                                          prior_prec_mix=50.0, prior_prec_alpha=50.0))
    for k in ("state", "ET", "cost", "var_ET"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_rounding_probe_is_seeded_and_off_by_default(scene):
    """The sensitivity probe used by the GPU tests: off at 0, deterministic
    for a seed, different for another seed, and small (a relative 1e-5 of
    the model values moves the first stage-1 step of alpha1 and T1 by less
    than lr / 100 in z)."""
    t, tr, L = scene
    base = oracle.retrieve(t, L[:6], tr.wv_bin[:6], cfg=oracle.Config(n_endm=K, solver="adam"))
    off = oracle.retrieve(t, L[:6], tr.wv_bin[:6], cfg=oracle.Config(n_endm=K, solver="adam", adam_gnoise=0.0,
                                                                     adam_gseed=7))
    assert np.array_equal(base["state"], off["state"])
    p1 = [oracle.retrieve(t, L[:6], tr.wv_bin[:6], cfg=oracle.Config(
        n_endm=K, solver="adam", adam_gnoise=1e-5, adam_gseed=s)) for s in (1, 1, 2)]
    assert np.array_equal(p1[0]["state"], p1[1]["state"])
    assert not np.array_equal(p1[0]["state"], p1[2]["state"])
    one = dict(n_endm=K, solver="adam", adam_steps1=1, adam_steps2=0)
    a = oracle.retrieve(t, L[:6], tr.wv_bin[:6], cfg=oracle.Config(**one))
    b = oracle.retrieve(t, L[:6], tr.wv_bin[:6], cfg=oracle.Config(**one, adam_gnoise=1e-5, adam_gseed=3))
    lo, hi = _bounds(oracle.Config(n_endm=K), 1)
    dz = 2 * np.abs(a["state"][:, :K + 2] - b["state"][:, :K + 2]) / (hi - lo)
    assert np.all(dz[:, K:] < oracle.Config().adam_lr1 / 100)
