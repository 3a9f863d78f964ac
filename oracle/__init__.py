"""ctypes wrapper of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY. The tests, the package smoke check and the
benchmark's CPU-baseline leg are the only callers; the product library never
imports this module. The oracle shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

MAXK = 8
NS1 = MAXK + 2

CONVERGED, MAXITER, NONFINITE, ALL_MASKED, CHOL_FAIL, NOT_CANDIDATE = range(6)
F_FP64, F_NOT_IDENT, F_MLP_FALLBACK, F_S1_MAXITER = 8, 16, 32, 64


def build(force=False):
    """Compile liboracle.so with gcc (FP64, IEEE semantics, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               "-Wall", "-o", _LIB, _SRC, "-lm"])
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        dp, fp = C.POINTER(C.c_double), C.POINTER(C.c_float)
        _lib.orc_planck.restype = C.c_double
        _lib.orc_planck.argtypes = [C.c_double, C.c_double]
        _lib.orc_planck_dT.restype = C.c_double
        _lib.orc_planck_dT.argtypes = [C.c_double, C.c_double]
        _lib.orc_hfdi.restype = C.c_double
        _lib.orc_hfdi.argtypes = [C.c_void_p, C.c_void_p, fp]
        _lib.orc_cholesky.restype = C.c_int
        _lib.orc_cholesky.argtypes = [dp, C.c_int]
        _lib.orc_chol_solve.argtypes = [dp, C.c_int, dp]
        _lib.orc_simplex_project.argtypes = [dp, C.c_int]
        _lib.orc_moments.argtypes = [dp, dp, dp]
        _lib.orc_planck_array.argtypes = [C.c_int64, dp, dp, dp]
    return _lib


class Tables_t(C.Structure):
    _fields_ = [("n_bands", C.c_int32), ("n_wv", C.c_int32), ("n_endm", C.c_int32),
                ("n_tgrid", C.c_int32),
                ("wavelength_nm", C.c_void_p), ("solar_irr", C.c_void_p), ("cos_sza", C.c_double),
                ("tau_down", C.c_void_p), ("tau_up", C.c_void_p), ("rho_atm", C.c_void_p),
                ("sph_alb", C.c_void_p), ("endmembers", C.c_void_p), ("sat_level", C.c_void_p),
                ("tgrid_lo", C.c_double), ("tgrid_hi", C.c_double)]


class Config_t(C.Structure):
    _fields_ = [("win1_lo", C.c_double), ("win1_hi", C.c_double),
                ("win2h_lo", C.c_double), ("win2h_hi", C.c_double),
                ("win2s_lo", C.c_double), ("win2s_hi", C.c_double),
                ("lo1", C.c_double * NS1), ("hi1", C.c_double * NS1),
                ("lo2", C.c_double * 6), ("hi2", C.c_double * 6),
                ("pm1", C.c_double * NS1), ("pp1", C.c_double * NS1),
                ("pm2", C.c_double * 6), ("pp2", C.c_double * 6),
                ("init_alpha1", C.c_double), ("init_T1", C.c_double), ("init_sigma", C.c_double),
                ("init_mu_h_floor", C.c_double), ("init_mu_s_ceil", C.c_double),
                ("init_eta_lo", C.c_double), ("init_eta_hi", C.c_double),
                ("max_it1", C.c_int32), ("max_it2", C.c_int32),
                ("tau0", C.c_double), ("tol_g", C.c_double), ("tol_x", C.c_double),
                ("tol_f", C.c_double), ("kappa_max", C.c_double), ("dfloor", C.c_double),
                ("noise_rel", C.c_double), ("noise_abs", C.c_double), ("weighted", C.c_int32),
                ("gate_hfdi", C.c_int32), ("hfdi_thresh", C.c_double),
                ("hfdi_lambda_hi", C.c_double), ("hfdi_lambda_lo", C.c_double),
                ("ident_sd_et", C.c_double), ("ident_alpha_snr", C.c_double),
                ("noise_sd", C.c_void_p),
                ("solver", C.c_int32), ("adam_steps1", C.c_int32), ("adam_steps2", C.c_int32),
                ("adam_lr1", C.c_double), ("adam_lr2", C.c_double), ("adam_clip", C.c_double),
                ("adam_beta1", C.c_double), ("adam_beta2", C.c_double), ("adam_eps", C.c_double),
                ("adam_gnoise", C.c_double), ("adam_gseed", C.c_uint64)]


class Outputs_t(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in (
        "state", "ET", "sdT", "alpha", "var_ET", "cost", "rms", "hfdi", "cost1", "kappa",
        "cov", "status", "it1", "it2", "n_used")]


@dataclasses.dataclass
class Config:
    """Retrieval constants. Windows: Sec. 2.3 and 2.6 (Omega_1 = [350, 2500] nm,
    Omega_2^hot ~ [900, 1800], Omega_2^smol ~ [1500, 2500]); HFDI gate -0.1
    at 2430/2061 nm (Sec. 2.1); everything else is the build's stated choice
    (the paper prints no LM constants and no bounds). The iteration caps
    100/400 lie well above what the damped iteration needs, so that a fit
    stops on a convergence test; the weak prior pulls T1 and the mixture
    shape towards the box centre (precision 1) and alpha towards 0 only at
    1e-6 (regularising J^T J where alpha vanishes)."""
    n_endm: int = 3
    n_tgrid: int = 64
    tgrid_lo: float = 350.0
    tgrid_hi: float = 2200.0
    win1: tuple = (350.0, 2500.0)
    win2h: tuple = (900.0, 1800.0)
    win2s: tuple = (1500.0, 2500.0)
    init_alpha1: float = 0.0
    init_T1: float = 800.0
    init_sigma: float = 100.0
    init_mu_h_floor: float = 1000.0
    init_mu_s_ceil: float = 700.0
    init_eta: tuple = (0.05, 0.95)
    max_it1: int = 100
    max_it2: int = 400
    tau0: float = 1.0
    tol_g: float = 1e-8
    tol_x: float = 1e-7
    tol_f: float = 1e-10
    kappa_max: float = 1e6
    dfloor: float = 1e-12
    noise_rel: float = 0.005
    noise_abs: float = 1e-4
    weighted: bool = False
    prior_prec_T1: float = 1.0
    prior_prec_mix: float = 1.0
    prior_prec_alpha: float = 1e-6
    gate_hfdi: bool = False
    hfdi_thresh: float = -0.1
    hfdi_lambdas: tuple = (2430.0, 2061.0)
    ident_sd_et: float = 100.0
    ident_alpha_snr: float = 3.0
    noise_sd: np.ndarray = None      # per-band noise sd [n_bands]: weights 1 / sd^2
    # solver: "lm" (damped Gauss-Newton, the default) or "adam", the paper's
    # optimiser (Sec. 2.6, Eq. adam): 30 steps at lr 0.03 (stage 1), 100 at
    # 0.015 (stage 2), beta (0.9, 0.999), eps 1e-8, global-norm clip (its
    # value is garbled in the paper: 1.0 here), no prior
    solver: str = "lm"
    adam_steps1: int = 30
    adam_steps2: int = 100
    adam_lr1: float = 0.03
    adam_lr2: float = 0.015
    adam_clip: float = 1.0
    adam_beta1: float = 0.9
    adam_beta2: float = 0.999
    adam_eps: float = 1e-8
    # sensitivity probe for tests (not part of the method): each Adam
    # gradient formed as if every band's model value were off by a relative
    # adam_gnoise times a seeded standard normal (0 = off)
    adam_gnoise: float = 0.0
    adam_gseed: int = 0
    lo1: np.ndarray = None
    hi1: np.ndarray = None
    lo2: np.ndarray = None
    hi2: np.ndarray = None
    pm1: np.ndarray = None
    pp1: np.ndarray = None
    pm2: np.ndarray = None
    pp2: np.ndarray = None

    def __post_init__(self):
        K = self.n_endm
        dT = (self.tgrid_hi - self.tgrid_lo) / (self.n_tgrid - 1)
        if self.lo1 is None:
            self.lo1 = np.array([0.0] * K + [0.0, self.tgrid_lo])
            self.hi1 = np.array([1.0] * K + [1.0, self.tgrid_hi])
        if self.lo2 is None:
            self.lo2 = np.array([900.0, dT, self.tgrid_lo, dT, 0.0, 0.0])
            self.hi2 = np.array([self.tgrid_hi, 500.0, 1000.0, 500.0, 1.0, 1.0])
        # weak Gaussian prior in z (precision in units of one band's noise
        # variance): box centre for T1 and the mixture shape, alpha = 0 for
        # the two thermal scalings; no prior on the surface fractions
        if self.pm1 is None:
            self.pm1 = np.zeros(K + 2)
            self.pm1[K] = -1.0
        if self.pm2 is None:
            self.pm2 = np.array([0.0] * 5 + [-1.0])
        if self.pp1 is None:
            self.pp1 = np.zeros(K + 2)
            self.pp1[K] = self.prior_prec_alpha
            self.pp1[K + 1] = self.prior_prec_T1
        if self.pp2 is None:
            self.pp2 = np.array([self.prior_prec_mix] * 5 + [self.prior_prec_alpha])

    def to_c(self):
        c = Config_t()
        c.win1_lo, c.win1_hi = self.win1
        c.win2h_lo, c.win2h_hi = self.win2h
        c.win2s_lo, c.win2s_hi = self.win2s
        for name in ("lo1", "hi1", "pm1", "pp1", "lo2", "hi2", "pm2", "pp2"):
            arr = getattr(c, name)
            v = np.asarray(getattr(self, name), dtype=np.float64)
            for i in range(len(arr)):
                arr[i] = v[i] if i < v.size else 0.0
        c.init_alpha1, c.init_T1, c.init_sigma = self.init_alpha1, self.init_T1, self.init_sigma
        c.init_mu_h_floor, c.init_mu_s_ceil = self.init_mu_h_floor, self.init_mu_s_ceil
        c.init_eta_lo, c.init_eta_hi = self.init_eta
        c.max_it1, c.max_it2 = self.max_it1, self.max_it2
        c.tau0, c.tol_g, c.tol_x, c.tol_f = self.tau0, self.tol_g, self.tol_x, self.tol_f
        c.kappa_max, c.dfloor = self.kappa_max, self.dfloor
        c.noise_rel, c.noise_abs, c.weighted = self.noise_rel, self.noise_abs, int(self.weighted)
        c.gate_hfdi, c.hfdi_thresh = int(self.gate_hfdi), self.hfdi_thresh
        c.hfdi_lambda_hi, c.hfdi_lambda_lo = self.hfdi_lambdas
        c.ident_sd_et, c.ident_alpha_snr = self.ident_sd_et, self.ident_alpha_snr
        if self.solver not in ("lm", "adam"):
            raise ValueError(f"unknown solver {self.solver!r}")
        c.solver = 1 if self.solver == "adam" else 0
        c.adam_steps1, c.adam_steps2 = self.adam_steps1, self.adam_steps2
        c.adam_lr1, c.adam_lr2, c.adam_clip = self.adam_lr1, self.adam_lr2, self.adam_clip
        c.adam_beta1, c.adam_beta2, c.adam_eps = self.adam_beta1, self.adam_beta2, self.adam_eps
        c.adam_gnoise, c.adam_gseed = self.adam_gnoise, self.adam_gseed
        if self.noise_sd is not None:
            # the C struct points into this array: keep it alive with the struct
            c._noise_sd = np.ascontiguousarray(self.noise_sd, dtype=np.float32)
            c.noise_sd = c._noise_sd.ctypes.data
        return c


def _ptr(a):
    return None if a is None else a.ctypes.data


MAX_BANDS, MAX_ENDM, MAX_TGRID = 512, 8, 256   # ORC_MAXB, ORC_MAXK, ORC_MAXT of oracle.h


class _TablesHolder:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, t, tgrid=(350.0, 2200.0)):
        # the C code's per-band, per-endmember and per-node work arrays have
        # fixed sizes (oracle.h): larger tables are refused here
        if not (0 < t.n_bands <= MAX_BANDS and 0 < t.n_endm <= MAX_ENDM and 0 < t.n_tgrid <= MAX_TGRID):
            raise ValueError(f"oracle tables limited to {MAX_BANDS} bands, {MAX_ENDM} endmembers, "
                             f"{MAX_TGRID} grid nodes")
        f = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)  # noqa
        self.arrs = [f(t.wavelength_nm), f(t.solar_irr), f(t.tau_down), f(t.tau_up),
                     f(t.rho_atm), f(t.sph_alb), f(t.endmembers), f(t.sat_level)]
        a = self.arrs
        self.c = Tables_t(t.n_bands, t.n_wv, t.n_endm, t.n_tgrid, _ptr(a[0]), _ptr(a[1]),
                          float(t.cos_sza), _ptr(a[2]), _ptr(a[3]), _ptr(a[4]), _ptr(a[5]),
                          _ptr(a[6]), _ptr(a[7]), float(tgrid[0]), float(tgrid[1]))


def planck(lambda_nm, T):
    lam = np.ascontiguousarray(np.broadcast_to(np.asarray(lambda_nm, np.float64),
                                               np.broadcast(lambda_nm, T).shape)).ravel().copy()
    TT = np.ascontiguousarray(np.broadcast_to(np.asarray(T, np.float64),
                                              np.broadcast(lambda_nm, T).shape)).ravel().copy()
    out = np.empty_like(lam)
    dp = C.POINTER(C.c_double)
    lib().orc_planck_array(lam.size, lam.ctypes.data_as(dp), TT.ctypes.data_as(dp),
                           out.ctypes.data_as(dp))
    return out.reshape(np.broadcast(lambda_nm, T).shape)


def planck_dT(lambda_nm, T):
    return lib().orc_planck_dT(float(lambda_nm), float(T))


def moments(x2):
    E, V = C.c_double(), C.c_double()
    x = np.ascontiguousarray(x2, dtype=np.float64)
    lib().orc_moments(x.ctypes.data_as(C.POINTER(C.c_double)), C.byref(E), C.byref(V))
    return E.value, V.value


def simplex_project(v):
    x = np.array(v, dtype=np.float64)
    lib().orc_simplex_project(x.ctypes.data_as(C.POINTER(C.c_double)), x.size)
    return x


def cholesky(A):
    M = np.array(A, dtype=np.float64, order="C")
    rc = lib().orc_cholesky(M.ctypes.data_as(C.POINTER(C.c_double)), M.shape[0])
    return None if rc != 0 else M


def chol_solve(Lc, b):
    y = np.array(b, dtype=np.float64)
    lib().orc_chol_solve(Lc.ctypes.data_as(C.POINTER(C.c_double)), Lc.shape[0],
                         y.ctypes.data_as(C.POINTER(C.c_double)))
    return y


def forward(tables, mode, state, wv_bin):
    """Noise-free model radiance [n, n_bands] (FP64). mode 1: state
    [x_surf, a1, T1]; mode 2: [x_surf, mu_h, s_h, mu_s, s_s, eta, a]."""
    th = _TablesHolder(tables)
    st = np.ascontiguousarray(state, dtype=np.float64)
    wv = np.ascontiguousarray(wv_bin, dtype=np.uint16)
    n = wv.size
    out = np.empty((n, tables.n_bands))
    lib().orc_forward(C.byref(th.c), C.c_int(mode), C.c_void_p(st.ctypes.data),
                      C.c_void_p(wv.ctypes.data), C.c_int64(n), C.c_void_p(out.ctypes.data))
    return out


def stage_jacobian(tables, stage, xs, x, wv_bin):
    th = _TablesHolder(tables)
    p = tables.n_endm + 2 if stage == 1 else 6
    L = np.empty(tables.n_bands)
    J = np.empty((tables.n_bands, p))
    xs_ = np.ascontiguousarray(xs if xs is not None else np.zeros(tables.n_endm), dtype=np.float64)
    x_ = np.ascontiguousarray(x, dtype=np.float64)
    lib().orc_stage_jacobian(C.byref(th.c), C.c_int(stage), C.c_void_p(xs_.ctypes.data),
                             C.c_void_p(x_.ctypes.data), C.c_int(int(wv_bin)),
                             C.c_void_p(L.ctypes.data), C.c_void_p(J.ctypes.data))
    return L, J


def synth_radiance(tables, mode, state, wv_bin, normals=None, noise_rel=0.005, noise_abs=1e-4):
    """Radiance = oracle forward model + sd(L) * normals, sd = sqrt((rel L)^2 + abs^2),
    cast to fp32 (the configs' noise model: 0.5 % + read noise)."""
    th = _TablesHolder(tables)
    st = np.ascontiguousarray(state, dtype=np.float64)
    wv = np.ascontiguousarray(wv_bin, dtype=np.uint16)
    n = wv.size
    nz = None if normals is None else np.ascontiguousarray(normals, dtype=np.float64)
    out = np.empty((n, tables.n_bands), dtype=np.float32)
    lib().orc_synth_radiance(C.byref(th.c), C.c_int(mode), C.c_void_p(st.ctypes.data),
                             C.c_void_p(wv.ctypes.data), C.c_void_p(_ptr(nz)), C.c_int64(n),
                             C.c_double(noise_rel), C.c_double(noise_abs),
                             C.c_void_p(out.ctypes.data))
    return out


def hfdi(tables, radiance_row, cfg=None):
    cfg = cfg or Config(n_endm=tables.n_endm)
    th = _TablesHolder(tables)
    c = cfg.to_c()
    L = np.ascontiguousarray(radiance_row, dtype=np.float32)
    return lib().orc_hfdi(C.byref(th.c), C.byref(c), L.ctypes.data_as(C.POINTER(C.c_float)))


def inject(tables, L_bg, wv_bin, alpha, T):
    """Eq. (inject): L_bg + alpha tau_up B(lambda, T) per pixel (fp32)."""
    th = _TablesHolder(tables)
    Lb = np.ascontiguousarray(L_bg, dtype=np.float32)
    wv = np.ascontiguousarray(wv_bin, dtype=np.uint16)
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    TT = np.ascontiguousarray(T, dtype=np.float64)
    out = np.empty_like(Lb)
    lib().orc_inject(C.byref(th.c), C.c_void_p(Lb.ctypes.data), C.c_void_p(wv.ctypes.data),
                     C.c_void_p(a.ctypes.data), C.c_void_p(TT.ctypes.data), C.c_int64(wv.size),
                     C.c_void_p(out.ctypes.data))
    return out


WV_LAMBDAS = (870.0, 940.0, 1010.0)     # shoulder, centre, shoulder of the 940 nm feature (nm)


def wv_depth_table(tables, lams=WV_LAMBDAS):
    """Depth of the 940 nm feature of each water-vapour bin of the tables
    (flat surface, two-way direct path), single precision [n_wv]."""
    th = _TablesHolder(tables)
    D = np.empty(tables.n_wv, dtype=np.float32)
    lib().orc_wv_depth_table(C.byref(th.c), C.c_double(lams[0]), C.c_double(lams[1]),
                             C.c_double(lams[2]), C.c_void_p(D.ctypes.data))
    return D


def wv_presolve(tables, radiance, width, height, block=12, lams=WV_LAMBDAS):
    """Water-vapour presolve (Sec. 2.5): per-pixel 940 nm band depth, the
    lower median of each block x block super-pixel, quantised to a bin of
    the tables. radiance [height * width, n_bands] row-major image order.
    Returns (bins [n] uint16, 0xFFFF for a block without any depth;
    depth [n] float32)."""
    th = _TablesHolder(tables)
    L = np.ascontiguousarray(radiance, dtype=np.float32)
    n = int(width) * int(height)
    assert L.shape == (n, tables.n_bands)
    bins = np.empty(n, dtype=np.uint16)
    depth = np.empty(n, dtype=np.float32)
    lib().orc_wv_presolve(C.byref(th.c), C.c_void_p(L.ctypes.data), C.c_int64(width), C.c_int64(height),
                          C.c_int(block), C.c_double(lams[0]), C.c_double(lams[1]), C.c_double(lams[2]),
                          C.c_void_p(bins.ctypes.data), C.c_void_p(depth.ctypes.data))
    return bins, depth


def retrieve(tables, radiance, wv_bin, cfg=None, init_state=None, n_threads=0):
    """Per-pixel two-stage fit of every row of radiance [n, n_bands] (fp32).
    Returns a dict of FP64 outputs (state [n, K+8], ET, sdT, alpha, cov [n, 21],
    var_ET, cost, rms, hfdi, cost1, kappa, status, it1, it2, n_used)."""
    cfg = cfg or Config(n_endm=tables.n_endm, n_tgrid=tables.n_tgrid)
    th = _TablesHolder(tables, (cfg.tgrid_lo, cfg.tgrid_hi))
    c = cfg.to_c()
    L = np.ascontiguousarray(radiance, dtype=np.float32)
    wv = np.ascontiguousarray(wv_bin, dtype=np.uint16)
    n = wv.size
    K = tables.n_endm
    out = {k: np.empty(n) for k in ("ET", "sdT", "alpha", "var_ET", "cost", "rms", "hfdi",
                                    "cost1", "kappa")}
    out["state"] = np.empty((n, K + 8))
    out["cov"] = np.empty((n, 21))
    for k in ("status", "it1", "it2", "n_used"):
        out[k] = np.empty(n, dtype=np.int32)
    o = Outputs_t(*[out[k].ctypes.data for k in (
        "state", "ET", "sdT", "alpha", "var_ET", "cost", "rms", "hfdi", "cost1", "kappa",
        "cov", "status", "it1", "it2", "n_used")])
    ini = None if init_state is None else np.ascontiguousarray(init_state, dtype=np.float64)
    lib().orc_retrieve(C.byref(th.c), C.byref(c), C.c_void_p(L.ctypes.data),
                       C.c_void_p(wv.ctypes.data), C.c_int64(n), C.c_void_p(_ptr(ini)),
                       C.byref(o), C.c_int(n_threads))
    return out


def mlp_forward(params, x):
    """FP64 forward of the proposal MLP; params = dict W1,b1,W2,b2,W3,b3."""
    W1, W2, W3 = (np.ascontiguousarray(params[k], np.float64) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (np.ascontiguousarray(params[k], np.float64) for k in ("b1", "b2", "b3"))
    x = np.ascontiguousarray(x, np.float64)
    B, Din = x.shape
    H, Dout = W1.shape[0], W3.shape[0]
    a1, a2, z = np.empty((B, H)), np.empty((B, H)), np.empty((B, Dout))
    v = C.c_void_p
    lib().orc_mlp_forward(C.c_int(B), C.c_int(Din), C.c_int(H), C.c_int(Dout),
                          *[v(a.ctypes.data) for a in (W1, b1, W2, b2, W3, b3, x, a1, a2, z)])
    return a1, a2, z


def mlp_backward(params, x, target, mask, n_out=None):
    """Loss and FP64 gradients of sum mask (z - t)^2 / (B n_out) in z-space;
    mask is per sample [B, Dout] (or per output [Dout])."""
    W1, W2, W3 = (np.ascontiguousarray(params[k], np.float64) for k in ("W1", "W2", "W3"))
    x = np.ascontiguousarray(x, np.float64)
    a1, a2, z = mlp_forward(params, x)
    t = np.ascontiguousarray(target, np.float64)
    B, Din = x.shape
    H, Dout = W1.shape[0], W3.shape[0]
    mk = np.ascontiguousarray(np.broadcast_to(np.asarray(mask, np.float64), (B, Dout)))
    if n_out is None:
        n_out = int(np.count_nonzero(np.asarray(mask).reshape(-1, Dout).max(0)))
    g = {"W1": np.empty((H, Din)), "b1": np.empty(H), "W2": np.empty((H, H)), "b2": np.empty(H),
         "W3": np.empty((Dout, H)), "b3": np.empty(Dout)}
    v = C.c_void_p
    lib().orc_mlp_backward.restype = C.c_double
    loss = lib().orc_mlp_backward(C.c_int(B), C.c_int(Din), C.c_int(H), C.c_int(Dout),
                                  C.c_int(n_out),
                                  *[v(a.ctypes.data) for a in (W1, W2, W3, x, a1, a2, z, t, mk,
                                                               g["W1"], g["b1"], g["W2"], g["b2"],
                                                               g["W3"], g["b3"])])
    return loss, g, z


def adam(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    vp = C.c_void_p
    lib().orc_adam(C.c_int64(w.size), vp(w.ctypes.data), vp(g.ctypes.data), vp(m.ctypes.data),
                   vp(v.ctypes.data), C.c_int(t), C.c_double(lr), C.c_double(b1), C.c_double(b2),
                   C.c_double(eps))


def posterior_at(tables, radiance, wv_bin, states, cfg=None):
    """The outputs that follow from given final states alone, per pixel
    (radiance [n, n_bands] fp32, states [n, K+8] in the layout of retrieve's
    state): E[T], sigma[T], stage-2 cost, rms, Laplace covariance [n, 21],
    var(E[T]) and the identifiability flag, as the fit's last step forms them."""
    cfg = cfg or Config(n_endm=tables.n_endm, n_tgrid=tables.n_tgrid)
    th = _TablesHolder(tables, (cfg.tgrid_lo, cfg.tgrid_hi))
    c = cfg.to_c()
    L = np.ascontiguousarray(radiance, dtype=np.float32)
    X = np.ascontiguousarray(states, dtype=np.float64)
    n = L.shape[0]
    out = {k: np.empty(n) for k in ("ET", "sdT", "cost", "rms", "var_ET")}
    out["cov"] = np.empty((n, 21))
    out["ident"] = np.zeros(n, dtype=bool)
    d = C.c_double
    for i in range(n):
        v = [d() for _ in range(5)]
        cv = np.empty(21)
        idf = C.c_int()
        lib().orc_posterior_at(C.byref(th.c), C.byref(c), C.c_void_p(L[i].ctypes.data),
                               C.c_int(int(wv_bin[i])), C.c_void_p(X[i].ctypes.data),
                               *[C.byref(x) for x in v[:4]], C.c_void_p(cv.ctypes.data),
                               C.byref(v[4]), C.byref(idf))
        for k, x in zip(("ET", "sdT", "cost", "rms", "var_ET"), v):
            out[k][i] = x.value
        out["cov"][i] = cv
        out["ident"][i] = bool(idf.value)
    return out


def normal_equations(tables, stage, radiance_row, wv_bin, x, cfg=None):
    """(H, g, cost) of one stage at state x in the fit's reduced z coordinates."""
    cfg = cfg or Config(n_endm=tables.n_endm, n_tgrid=tables.n_tgrid)
    th = _TablesHolder(tables, (cfg.tgrid_lo, cfg.tgrid_hi))
    c = cfg.to_c()
    K = tables.n_endm
    P = K + 1 if stage == 1 else 6
    L = np.ascontiguousarray(radiance_row, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    H = np.zeros((P, P))
    g = np.zeros(P)
    cost = C.c_double()
    lib().orc_normal_equations(C.byref(th.c), C.byref(c), C.c_int(stage), C.c_void_p(L.ctypes.data),
                               C.c_int(int(wv_bin)), C.c_void_p(xx.ctypes.data),
                               C.c_void_p(H.ctypes.data), C.c_void_p(g.ctypes.data), C.byref(cost))
    return H, g, cost.value
