"""Pins of the FP64 oracle against facts that do not come from the oracle:
closed forms (Stefan-Boltzmann, Wien, the Rayleigh-Jeans and Wien limits),
numerical integration of the mixture density, brute force (simplex
projection, simplex-constrained least squares), library routines used as
independent references (numpy Cholesky), finite differences of the
oracle's own forward model, and noise-free recovery of injected states."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

SIGMA_SB = 5.670374419e-8          # W m^-2 K^-4 (CODATA 2018, derived exact)
WIEN_B = 2.897771955e-3            # m K
H, C, KB = 6.62607015e-34, 299792458.0, 1.380649e-23
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


# ------------------------------------------------------------- Planck ----
@pytest.mark.parametrize("T", [350.0, 800.0, 1500.0, 2200.0, 5778.0])
def test_planck_integral_is_stefan_boltzmann(T):
    """Integral of B over wavelength equals sigma T^4 / pi (W m^-2 sr^-1)."""
    lnlam = np.linspace(np.log(10.0), np.log(1e9), 800001)      # 10 nm - 1 m, in nm
    lam = np.exp(lnlam)
    integral = np.trapezoid(oracle.planck(lam, T) * lam, lnlam)
    # tails: below 10 nm exp(-x) with x > 240; beyond 1 m the Rayleigh-Jeans
    # tail 2 c k T / (3 lambda^3) is below 1e-10 W m^-2 sr^-1
    tail = 2.0 * C * KB * T / 3.0
    expect = SIGMA_SB * T ** 4 / math.pi
    assert abs(integral + tail - expect) / expect < 1e-6


@pytest.mark.parametrize("T", [500.0, 1000.0, 2200.0])
def test_planck_wien_peak(T):
    lam = np.linspace(0.5 * WIEN_B / T * 1e9, 2.0 * WIEN_B / T * 1e9, 200001)
    B = oracle.planck(lam, T)
    step = lam[1] - lam[0]
    assert abs(lam[np.argmax(B)] - WIEN_B / T * 1e9) <= step


def test_planck_rayleigh_jeans_and_wien_limits():
    T = 1000.0
    for x in (1e-3, 1e-4):
        lam_m = H * C / (x * KB * T)
        rj = 2.0 * C * KB * T / lam_m ** 4 * (1 - x / 2 + x * x / 12) * 1e-9
        assert abs(oracle.planck(lam_m * 1e9, T) / rj - 1) < 1e-9
    for x in (40.0, 80.0):
        lam_m = H * C / (x * KB * T)
        wien = 2.0 * H * C ** 2 / lam_m ** 5 * math.exp(-x) * (1 + math.exp(-x)) * 1e-9
        assert abs(oracle.planck(lam_m * 1e9, T) / wien - 1) < 1e-12


def test_planck_no_overflow():
    T = 1000.0
    x = np.logspace(-3, np.log10(800.0), 2000)
    lam = H * C / (x * KB * T) * 1e9
    B = oracle.planck(lam, T)
    assert np.all(np.isfinite(B)) and np.all(B >= 0)


def test_planck_dT_matches_finite_difference():
    for lam in (900.0, 1600.0, 2400.0):
        for T in (400.0, 900.0, 2000.0):
            h = 1e-5 * T
            fd = (oracle.planck(lam, T + h) - oracle.planck(lam, T - h)) / (2 * h)
            assert abs(oracle.planck_dT(lam, T) / fd - 1) < 1e-6


# --------------------------------------------------- moment matching ----
def test_moments_equal_numerical_integration_of_mixture():
    rng = np.random.default_rng(3)
    T = np.linspace(-3000, 6000, 900001)
    for _ in range(20):
        mh, ms = rng.uniform(900, 2000), rng.uniform(400, 1000)
        sh, ss = rng.uniform(20, 400), rng.uniform(20, 400)
        eta = rng.uniform(0, 1)
        p = (eta * np.exp(-0.5 * ((T - mh) / sh) ** 2) / (sh * math.sqrt(2 * math.pi))
             + (1 - eta) * np.exp(-0.5 * ((T - ms) / ss) ** 2) / (ss * math.sqrt(2 * math.pi)))
        m1 = np.trapezoid(T * p, T)
        m2 = np.trapezoid((T - m1) ** 2 * p, T)
        E, V = oracle.moments([mh, sh, ms, ss, eta, 0.1])
        assert abs(E - m1) < 1e-6 and abs(V - m2) / m2 < 1e-7


def test_discrete_grid_moments_match_away_from_edges():
    """With sigma >= grid step and the components well inside [350, 2200] K the
    normalised grid weights have the continuous moments (aliasing ~e^-20)."""
    Tg = np.linspace(350.0, 2200.0, 64)
    dT = Tg[1] - Tg[0]
    rng = np.random.default_rng(4)
    for _ in range(20):
        sh, ss = rng.uniform(dT, 120), rng.uniform(dT, 120)
        mh = rng.uniform(350 + 7 * sh, 2200 - 7 * sh)
        ms = rng.uniform(350 + 7 * ss, 2200 - 7 * ss)
        eta = rng.uniform(0, 1)
        wh = np.exp(-0.5 * ((Tg - mh) / sh) ** 2); wh /= wh.sum()
        ws = np.exp(-0.5 * ((Tg - ms) / ss) ** 2); ws /= ws.sum()
        p = eta * wh + (1 - eta) * ws
        m1 = (p * Tg).sum()
        m2 = (p * (Tg - m1) ** 2).sum()
        E, V = oracle.moments([mh, sh, ms, ss, eta, 0.1])
        assert abs(E - m1) < 1e-6 and abs(math.sqrt(V) - math.sqrt(m2)) < 1e-6


# -------------------------------------------------- simplex projection ---
def _brute_simplex_projection(v):
    """Enumerate supports S: projection onto {x_S >= 0, sum = 1, x_notS = 0}
    is x_S = v_S - (sum v_S - 1)/|S|; keep the feasible point closest to v."""
    K = v.size
    best, bd = None, np.inf
    for r in range(1, K + 1):
        for S in itertools.combinations(range(K), r):
            S = list(S)
            x = np.zeros(K)
            x[S] = v[S] - (v[S].sum() - 1.0) / len(S)
            if np.all(x >= -1e-15):
                d = np.sum((x - v) ** 2)
                if d < bd:
                    best, bd = x, d
    return best


def test_simplex_projection_matches_brute_force():
    rng = np.random.default_rng(5)
    for _ in range(10000):
        K = int(rng.integers(1, 5))
        v = rng.normal(0.3, 0.8, K)
        assert np.max(np.abs(oracle.simplex_project(v) - _brute_simplex_projection(v))) < 1e-12


# ------------------------------------------------------------ Cholesky ---
def test_cholesky_matches_numpy():
    rng = np.random.default_rng(6)
    for n in range(1, 10):
        A = rng.normal(size=(n, n))
        A = A @ A.T + n * np.eye(n)
        L = oracle.cholesky(A)
        assert np.allclose(np.tril(L), np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
        b = rng.normal(size=n)
        assert np.allclose(oracle.chol_solve(L, b), np.linalg.solve(A, b), rtol=1e-10)
    assert oracle.cholesky(-np.eye(3)) is None


# ------------------------------------------------------ forward model ----
@pytest.fixture(scope="module")
def tables():
    return synth.make_tables(path_reflectance=True)


def test_mixture_collapses_to_single_temperature(tables):
    """A component much narrower than the grid step centred on a node is the
    single-temperature Planck term of stage 1 (two independent code paths)."""
    Tg = np.linspace(350.0, 2200.0, 64)
    xs = np.array([0.2, 0.5, 0.3])
    for j in (5, 20, 40):
        st1 = np.concatenate([xs, [0.05, Tg[j]]])[None]
        st2 = np.concatenate([xs, [Tg[j], 3.0, Tg[j], 3.0, 1.0, 0.05]])[None]
        L1 = oracle.forward(tables, 1, st1, [3])
        L2 = oracle.forward(tables, 2, st2, [3])
        assert np.max(np.abs(L2 / L1 - 1)) < 1e-12


def test_mixture_component_symmetry(tables):
    xs = np.array([0.2, 0.5, 0.3])
    a = np.concatenate([xs, [1200.0, 80.0, 600.0, 50.0, 0.3, 0.02]])
    b = np.concatenate([xs, [600.0, 50.0, 1200.0, 80.0, 0.7, 0.02]])
    La, Lb = oracle.forward(tables, 2, np.stack([a, b]), [2, 2])
    assert np.max(np.abs(La / Lb - 1)) < 1e-13


def test_solar_term_limits(tables):
    """With alpha = 0 the model is the solar term alone: linear in the
    fractions when S = 0, and rho_atm alone when the surface is black."""
    t0 = synth.make_tables()   # rho_atm = S = 0
    e = np.eye(3)
    pure = oracle.forward(t0, 1, np.column_stack([e, np.zeros(3), np.full(3, 800.0)]), [1, 1, 1])
    x = np.array([0.2, 0.5, 0.3])
    mixed = oracle.forward(t0, 1, np.concatenate([x, [0.0, 800.0]])[None], [1])[0]
    assert np.max(np.abs(mixed / (x @ pure) - 1)) < 1e-13
    black = oracle.forward(tables, 1, np.array([[0.0, 0.0, 0.0, 0.0, 800.0]]), [1])[0]
    A = tables.solar_irr.astype(np.float64) * tables.cos_sza / math.pi
    assert np.max(np.abs(black / (A * tables.rho_atm[1]) - 1)) < 1e-6


def _fd_jac(tables, stage, xs, x, w, h):
    cols = []
    for i in range(x.size):
        xp, xm = x.copy(), x.copy()
        xp[i] += h[i]
        xm[i] -= h[i]
        Lp, _ = oracle.stage_jacobian(tables, stage, xs, xp, w)
        Lm, _ = oracle.stage_jacobian(tables, stage, xs, xm, w)
        cols.append((Lp - Lm) / (2 * h[i]))
    return np.stack(cols, 1)


def test_stage1_jacobian_matches_finite_differences(tables):
    rng = np.random.default_rng(7)
    for _ in range(200):
        xs = rng.dirichlet(np.ones(3))
        x = np.concatenate([xs, [10 ** rng.uniform(-3, -0.5), rng.uniform(450, 2100)]])
        w = int(rng.integers(16))
        _, J = oracle.stage_jacobian(tables, 1, None, x, w)
        Jfd = _fd_jac(tables, 1, None, x, w, np.r_[[1e-6] * 3, 1e-9, 1e-3])
        scale = np.max(np.abs(J), 0) + 1e-300
        assert np.max(np.abs(J - Jfd) / scale) < 1e-6


def test_stage2_jacobian_matches_finite_differences(tables):
    rng = np.random.default_rng(8)
    for _ in range(200):
        xs = rng.dirichlet(np.ones(3))
        x = np.array([rng.uniform(950, 2100), rng.uniform(35, 450), rng.uniform(380, 950),
                      rng.uniform(35, 450), rng.uniform(0.05, 0.95), 10 ** rng.uniform(-3, -0.5)])
        w = int(rng.integers(16))
        _, J = oracle.stage_jacobian(tables, 2, xs, x, w)
        Jfd = _fd_jac(tables, 2, xs, x, w, np.array([1e-3, 1e-3, 1e-3, 1e-3, 1e-6, 1e-9]))
        scale = np.max(np.abs(J), 0) + 1e-300
        assert np.max(np.abs(J - Jfd) / scale) < 1e-6


# --------------------------------------------------------- HFDI --------
def test_hfdi_definition():
    t = synth.make_tables()
    lam = t.wavelength_nm
    L = np.ones(t.n_bands, np.float32)
    assert oracle.hfdi(t, L) == 0.0
    L[np.argmin(np.abs(lam - 2430))] = 3.0
    assert abs(oracle.hfdi(t, L) - 0.5) < 1e-12


# ---------------------------------------------------------- LM fits ----
def _noprior(K=3, **kw):
    return oracle.Config(n_endm=K, prior_prec_T1=0.0, prior_prec_mix=0.0, prior_prec_alpha=0.0, **kw)


def test_stage1_noise_free_recovery():
    t = synth.make_tables()
    tr = synth.make_config1_truth(seed=11, width=64, height=1, fire_frac=1.0,
                                  alpha_range=(1e-2, 0.5))
    L = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, None)
    o = oracle.retrieve(t, L, tr.wv_bin, _noprior())
    T1, a1 = o["state"][:, 4], o["state"][:, 3]
    ok = np.abs(T1 - tr.single[:, 1]) < 1e-2
    assert ok.mean() >= 0.98
    assert np.all(np.abs(a1[ok] / tr.single[ok, 0] - 1) < 1e-4)
    assert np.all(np.abs(o["state"][ok, :3] - tr.x_surf[ok]) < 1e-5)


def _stage2_case(seed, n):
    t = synth.make_tables()
    rng = np.random.default_rng(seed)
    dT = 1850 / 63
    xs = rng.dirichlet(np.ones(3), n)
    ms = rng.uniform(500, 800, n)
    mh = ms + rng.uniform(300, 800, n)
    x2 = np.column_stack([mh, rng.uniform(2 * dT, 150, n), ms, rng.uniform(2 * dT, 150, n),
                          rng.uniform(0.2, 0.8, n), 10 ** rng.uniform(-2, -0.5, n)])
    wv = rng.integers(0, 16, n).astype(np.uint16)
    return t, rng, xs, x2, wv


def test_stage2_single_gaussian_noise_free_recovery():
    """Well-posed sub-case of stage 2: eta = 1 held fixed (lo = hi), so p(T) is
    one Gaussian on the grid. From a perturbed start with the true surface
    (stage 1 given zero iterations) the fit recovers (mu_h, s_h, alpha)."""
    t, rng, xs, x2, wv = _stage2_case(12, 24)
    x2[:, 4] = 1.0
    x2[:, 0] = rng.uniform(950, 1700, x2.shape[0])
    L = oracle.synth_radiance(t, 2, np.column_stack([xs, x2]), wv, None)
    cfg = _noprior(max_it1=0, max_it2=200)
    cfg.lo2[4] = cfg.hi2[4] = 1.0
    pert = x2.copy()
    pert[:, 0] += rng.uniform(-80, 80, len(pert))
    pert[:, 1] *= rng.uniform(0.7, 1.3, len(pert))
    pert[:, 5] *= rng.uniform(0.7, 1.3, len(pert))
    init = np.column_stack([xs, np.full(len(xs), 0.01), np.full(len(xs), 800.0), pert])
    o = oracle.retrieve(t, L, wv, cfg, init_state=init)
    st = o["state"][:, 5:]
    assert np.max(np.abs(st[:, 0] - x2[:, 0])) < 1e-3
    assert np.max(np.abs(st[:, 1] - x2[:, 1])) < 1e-3
    assert np.max(np.abs(st[:, 5] / x2[:, 5] - 1)) < 1e-6


def test_stage2_mixture_fit_minimises_cost():
    """Full six-parameter mixture on noise-free mixture spectra: the fit
    drives the residual to zero: relative rms below 1e-4 of the radiance,
    fifty times under the 0.5 % noise of the configs."""
    t, rng, xs, x2, wv = _stage2_case(14, 16)
    L = oracle.synth_radiance(t, 2, np.column_stack([xs, x2]), wv, None)
    cfg = _noprior(max_it1=0, max_it2=400)
    pert = x2 * (1 + 0.05 * rng.normal(size=x2.shape))
    pert[:, 4] = np.clip(pert[:, 4], 0, 1)
    init = np.column_stack([xs, np.full(len(xs), 0.01), np.full(len(xs), 800.0), pert])
    o = oracle.retrieve(t, L, wv, cfg, init_state=init)
    lam = t.wavelength_nm
    win = (lam >= 900) & (lam <= 2500)
    scale = np.sqrt(np.mean(L[:, win].astype(np.float64) ** 2, 1))
    assert np.all(o["rms"] / scale < 1e-4)


def _brute_simplex_ls(A, y):
    """min ||A x - y||^2 over the simplex by enumerating supports and solving
    the equality-constrained normal equations (KKT) on each."""
    K = A.shape[1]
    best, bc = None, np.inf
    for r in range(1, K + 1):
        for S in itertools.combinations(range(K), r):
            S = list(S)
            As = A[:, S]
            M = np.zeros((r + 1, r + 1))
            M[:r, :r] = 2 * As.T @ As
            M[:r, r] = 1
            M[r, :r] = 1
            rhs = np.r_[2 * As.T @ y, 1.0]
            sol = np.linalg.lstsq(M, rhs, rcond=None)[0]
            x = np.zeros(K)
            x[S] = sol[:r]
            if np.all(x >= -1e-12):
                c = np.sum((A @ x - y) ** 2)
                if c < bc:
                    best, bc = x, c
    return best


def test_stage1_linear_subproblem_matches_simplex_least_squares():
    """With S = 0 and no fire the stage-1 fit of the fractions is a linear
    least-squares problem on the simplex; the constrained optimum is found by
    brute force over supports."""
    t = synth.make_tables()
    rng = np.random.default_rng(13)
    e = np.eye(3)
    basis = oracle.forward(t, 1, np.column_stack([e, np.zeros(3), np.full(3, 800.0)]), [4, 4, 4])
    win = (t.wavelength_nm >= 350) & (t.wavelength_nm <= 2500)
    A = basis.T[win]
    cfg = _noprior(max_it1=200, tol_g=1e-13, tol_x=1e-15, tol_f=0.0)
    cfg.lo1[3] = cfg.hi1[3] = 0.0             # alpha1 held at 0: no thermal term
    for _ in range(12):
        xt = rng.normal(0.33, 0.6, 3)          # off the simplex: constraints bind
        y = basis.T @ xt
        L = y[None].astype(np.float32)
        o = oracle.retrieve(t, L, [4], cfg)
        xb = _brute_simplex_ls(A, L[0].astype(np.float64)[win])
        assert np.max(np.abs(o["state"][0, :3] - xb)) < 1e-9


def test_covariance_matches_inverse_fd_hessian():
    """At a zero-residual optimum with the noise-weighted loss, the Laplace
    covariance equals the inverse of half the finite-difference Hessian of
    the cost (Gauss-Newton is exact there). Single-Gaussian case (eta = 1
    held fixed) with the true surface, so the free block (mu_h, s_h, alpha)
    is well conditioned."""
    t = synth.make_tables()
    cfg = _noprior(weighted=True, max_it1=0, max_it2=300)
    cfg.lo2[4] = cfg.hi2[4] = 1.0
    xs = np.array([0.3, 0.4, 0.3])
    x2 = np.array([1300.0, 90.0, 650.0, 70.0, 1.0, 0.05])
    L = oracle.synth_radiance(t, 2, np.r_[xs, x2][None], [5], None)
    init = np.r_[xs, 0.01, 800.0, x2 * np.array([1.03, 0.9, 1, 1, 1, 1.1])][None]
    o = oracle.retrieve(t, L, [5], cfg, init_state=init)
    x2f = o["state"][0, 5:]
    assert abs(x2f[0] - 1300.0) < 1e-3
    Lobs = L[0].astype(np.float64)
    lam = t.wavelength_nm
    win = (lam >= 900) & (lam <= 2500)
    w = win / (cfg.noise_rel ** 2 * Lobs ** 2 + cfg.noise_abs ** 2)
    free = [0, 1, 5]

    def half_cost(v):
        Lm, _ = oracle.stage_jacobian(t, 2, xs, v, 5)
        return 0.5 * np.sum(w * (Lobs - Lm) ** 2)

    h = np.array([0.05, 0.05, 0, 0, 0, 1e-6])
    Hs = np.zeros((3, 3))
    for a, i in enumerate(free):
        for b, j in enumerate(free):
            def f(di, dj):
                v = x2f.copy()
                v[i] += di * h[i]
                v[j] += dj * h[j]
                return half_cost(v)
            Hs[a, b] = (f(1, 1) - f(1, -1) - f(-1, 1) + f(-1, -1)) / (4 * h[i] * h[j])
    Cfd = np.linalg.inv(Hs)
    iu = np.triu_indices(6)
    C = np.zeros((6, 6))
    C[iu] = o["cov"][0]
    C = C + np.triu(C, 1).T
    Cf = C[np.ix_(free, free)]
    assert np.max(np.abs(Cf / Cfd - 1)) < 1e-3
    assert abs(o["var_ET"][0] / Cfd[0, 0] - 1) < 1e-3
    assert np.isinf(C[2, 2]) and np.isinf(C[3, 3])      # zero columns: eta = 1


def test_statuses_for_degenerate_inputs():
    t = synth.make_tables(sat_level=1e-6)
    L = np.full((2, t.n_bands), 0.05, np.float32)
    L[1, 7] = np.nan
    o = oracle.retrieve(t, L, [0, 0])
    assert o["status"][0] & 7 == oracle.ALL_MASKED
    assert o["status"][1] & 7 == oracle.NONFINITE


def test_hfdi_gate_skips_non_candidates():
    t = synth.make_tables()
    tr = synth.make_config1_truth(seed=0, width=16, height=16)
    L = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, None)
    o = oracle.retrieve(t, L, tr.wv_bin, oracle.Config(gate_hfdi=True))
    cand = o["hfdi"] >= -0.1
    assert np.all((o["status"][~cand] & 7) == oracle.NOT_CANDIDATE)
    assert np.all((o["status"][cand] & 7) != oracle.NOT_CANDIDATE)


def test_defaults_follow_paper_constants():
    g = json.load(open(GOLDEN))
    c = oracle.Config()
    assert (c.tgrid_lo, c.tgrid_hi) == tuple(g["temperature_grid_K"]["value"])
    assert c.win1 == tuple(g["window_stage1_nm"]["value"])
    assert c.win2h == tuple(g["window_stage2_hot_nm"]["value"])
    assert c.win2s == tuple(g["window_stage2_smol_nm"]["value"])
    assert c.hfdi_thresh == g["hfdi_threshold"]["value"]
    assert c.hfdi_lambdas == tuple(g["hfdi_bands_nm"]["value"])
    s1, s2 = g["stage_steps"]["value"]
    assert c.max_it1 >= s1 and c.max_it2 >= s2


def test_oracle_refuses_tables_beyond_its_work_arrays():
    """The C oracle's work arrays hold 512 bands, 8 endmembers and 256 grid
    nodes; larger tables are refused before any C code runs."""
    import pytest
    t = synth.make_tables(n_bands=520)
    with pytest.raises(ValueError):
        oracle.synth_radiance(t, 1, np.zeros((1, 5)), np.zeros(1, np.int64))


# ------------------------------------------------- the weak prior -------
def _cost(tables, stage, L, w, x, cfg):
    return oracle.normal_equations(tables, stage, L, w, x, cfg)[2]


def test_gradient_with_prior_matches_finite_differences_of_the_cost():
    """g = J^T W r - psc P (z - pm) is minus half the z-gradient of the cost
    (Eq. loss plus the weak prior), prior terms included: checked against
    central differences of the oracle's own cost, stage 2 in z = 2 (x - lo) /
    (hi - lo) - 1 and stage 1 along its reduced directions (fraction k
    against the largest fraction m, then alpha1 and T1), with the default
    priors (T1 and mixture shape at precision 1, alpha at 1e-6) and with
    every prior precision raised to 1e3 so that the prior dominates."""
    t = synth.make_tables()
    tr = synth.make_config1_truth(seed=31, width=24, height=1, fire_frac=1.0, alpha_range=(1e-2, 0.3))
    L = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, None).astype(np.float32)
    rng = np.random.default_rng(33)
    for cfg in (oracle.Config(), oracle.Config(prior_prec_T1=1e3, prior_prec_mix=1e3, prior_prec_alpha=1e3)):
        sc2 = 0.5 * (cfg.hi2 - cfg.lo2)
        sc1 = 0.5 * (cfg.hi1 - cfg.lo1)
        for j in range(8):
            w = int(tr.wv_bin[j])
            xs = rng.dirichlet(np.ones(3))
            x2 = np.array([rng.uniform(950, 2100), rng.uniform(40, 400), rng.uniform(400, 950),
                           rng.uniform(40, 400), rng.uniform(0.1, 0.9), 10 ** rng.uniform(-2.5, -0.5)])
            x = np.concatenate([xs, x2])
            _, g, _ = oracle.normal_equations(t, 2, L[j], w, x, cfg)
            h = 1e-5
            fd = np.empty(6)
            for i in range(6):
                xp, xm = x.copy(), x.copy()
                xp[3 + i] += h * sc2[i]
                xm[3 + i] -= h * sc2[i]
                fd[i] = -0.5 * (_cost(t, 2, L[j], w, xp, cfg) - _cost(t, 2, L[j], w, xm, cfg)) / (2 * h)
            assert np.max(np.abs(g - fd)) <= 1e-5 * np.max(np.abs(g)), (j, g, fd)
            # stage 1: reduced basis (k != m against m), then alpha1, T1
            x1 = np.concatenate([xs, [10 ** rng.uniform(-2.5, -0.5), rng.uniform(500, 2000)]])
            _, g1, _ = oracle.normal_equations(t, 1, L[j], w, x1, cfg)
            m = int(np.argmax(x1[:3]))
            dirs = []
            for k in range(3):
                if k != m:
                    d = np.zeros(5)
                    d[k], d[m] = sc1[k], -sc1[m]
                    dirs.append(d)
            for k in (3, 4):
                d = np.zeros(5)
                d[k] = sc1[k]
                dirs.append(d)
            fd1 = np.array([-0.5 * (_cost(t, 1, L[j], w, x1 + h * d, cfg) -
                                    _cost(t, 1, L[j], w, x1 - h * d, cfg)) / (2 * h) for d in dirs])
            assert np.max(np.abs(g1 - fd1)) <= 1e-5 * np.max(np.abs(g1)), (j, g1, fd1)


def test_fit_without_data_lands_on_the_prior_means():
    """With every band weight ~0 (a per-band noise sd of 1e15: weights 1e-30)
    the cost is the prior alone, so the fit must end on the prior means: T1
    at the centre of its box, the mixture shape (mu_h, s_h, mu_s, s_s, eta)
    at the centre of theirs, alpha1 and alpha at 0 (their prior mean z = -1).
    A dropped prior term, a wrong sign or a wrong scale fails this."""
    t = synth.make_tables()
    tr = synth.make_config1_truth(seed=35, width=6, height=1, fire_frac=0.5)
    L = oracle.synth_radiance(t, 1, tr.state1(), tr.wv_bin, None).astype(np.float32)
    cfg = oracle.Config(noise_sd=np.full(t.n_bands, 1e15, np.float32))
    o = oracle.retrieve(t, L, tr.wv_bin, cfg)
    assert np.all((o["status"] & 7) == oracle.CONVERGED)
    centre1 = 0.5 * (cfg.lo1[4] + cfg.hi1[4])
    centre2 = 0.5 * (cfg.lo2 + cfg.hi2)
    assert np.max(np.abs(o["state"][:, 4] - centre1)) < 1e-3            # T1
    assert np.max(np.abs(o["state"][:, 3])) < 1e-6                      # alpha1
    assert np.max(np.abs(o["state"][:, 5:10] - centre2[:5])) < 1e-3     # mixture shape
    assert np.max(np.abs(o["state"][:, 10])) < 1e-6                     # alpha
