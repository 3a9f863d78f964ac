"""ctypes binding of libfirert.so (include/firert.h).

Argument marshalling only: every step of the retrieval runs in the library's
CUDA kernels. Device arrays are torch CUDA tensors (torch is used for device
memory and streams); host arrays are numpy arrays. There is no CPU fallback:
if the library cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FIRERT_DEBUG=1 in the environment loads the bounds-checked build
LIB_PATH = os.path.join(_HERE, "libfirert_debug.so" if os.environ.get("FIRERT_DEBUG") == "1"
                        else "libfirert.so")

MAX_ENDM = 8
FIRE_MEM_DEVICE, FIRE_MEM_HOST = 0, 1
FIRE_INIT_DEFAULT, FIRE_INIT_GIVEN, FIRE_INIT_MLP = 0, 1, 2
FIRE_FIT_ALL, FIRE_FIT_HFDI = 0, 1
FIRE_SOLVER_LM, FIRE_SOLVER_ADAM = 0, 1
PX_CONVERGED, PX_MAXITER, PX_NONFINITE, PX_ALL_MASKED, PX_CHOL_FAIL, PX_NOT_CANDIDATE = range(6)
PX_F_FP64, PX_F_NOT_IDENT, PX_F_MLP_FALLBACK, PX_F_S1_MAXITER = 8, 16, 32, 64
STATIC_MAX_PIX = 16384           # scene limit of Context.retrieve_static

SYMBOLS = ("fire_default_config", "fire_default_priors", "fire_ctx_create", "fire_ctx_destroy",
           "fire_retrieve", "fire_forward", "fire_block_mean", "fire_get_stats",
           "fire_window_bands", "fire_status_str", "fire_normal_equations", "fire_gemm_bf16",
           "fire_mlp_create", "fire_mlp_destroy", "fire_mlp_train", "fire_mlp_infer",
           "fire_mlp_gradients", "fire_mlp_param_count", "fire_mlp_params", "fire_mlp_save",
           "fire_mlp_load", "fire_mlp_next_sample", "fire_ctx_set_mlp", "fire_retrieve_batch",
           "fire_graph_capture", "fire_graph_launch", "fire_graph_destroy", "fire_autotune",
           "fire_set_tuning", "fire_set_kernel_timing", "fire_get_kernel_times",
           "fire_retrieve_static", "fire_set_allocator", "fire_measure_peak", "fire_wv_presolve",
           "fire_wv_depth_table", "fire_inject", "fire_hfdi", "fire_build_flags", "fire_debug_word")

# device allocator hook (fire_set_allocator): alloc(bytes, user) -> ptr, free(ptr, user)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class FireError(RuntimeError):
    pass


class Tables_t(C.Structure):
    _fields_ = [("n_bands", C.c_int32), ("n_wv", C.c_int32), ("n_endm", C.c_int32),
                ("n_tgrid", C.c_int32), ("wavelength_nm", C.c_void_p), ("solar_irr", C.c_void_p),
                ("cos_sza", C.c_float), ("tau_down", C.c_void_p), ("tau_up", C.c_void_p),
                ("rho_atm", C.c_void_p), ("sph_alb", C.c_void_p), ("endmembers", C.c_void_p),
                ("sat_level", C.c_void_p), ("tgrid_lo", C.c_float), ("tgrid_hi", C.c_float)]


class Config_t(C.Structure):
    _fields_ = [("win1_lo", C.c_float), ("win1_hi", C.c_float), ("win2h_lo", C.c_float),
                ("win2h_hi", C.c_float), ("win2s_lo", C.c_float), ("win2s_hi", C.c_float),
                ("max_it1", C.c_int32), ("max_it2", C.c_int32), ("tau0", C.c_float),
                ("tol_g", C.c_float), ("tol_x", C.c_float), ("tol_f", C.c_float),
                ("kappa_max", C.c_float), ("dfloor", C.c_float), ("noise_rel", C.c_float),
                ("noise_abs", C.c_float), ("weighted", C.c_int32), ("hfdi_thresh", C.c_float),
                ("hfdi_lambda_hi", C.c_float), ("hfdi_lambda_lo", C.c_float),
                ("ident_sd_et", C.c_float), ("ident_alpha_snr", C.c_float),
                ("wait_spins", C.c_int64),
                ("solver", C.c_int32), ("adam_steps1", C.c_int32), ("adam_steps2", C.c_int32),
                ("adam_lr1", C.c_double), ("adam_lr2", C.c_double), ("adam_clip", C.c_double),
                ("adam_beta1", C.c_double), ("adam_beta2", C.c_double), ("adam_eps", C.c_double)]


class Priors_t(C.Structure):
    _fields_ = [("lo1", C.c_float * (MAX_ENDM + 2)), ("hi1", C.c_float * (MAX_ENDM + 2)),
                ("pm1", C.c_float * (MAX_ENDM + 2)), ("pp1", C.c_float * (MAX_ENDM + 2)),
                ("lo2", C.c_float * 6), ("hi2", C.c_float * 6), ("pm2", C.c_float * 6),
                ("pp2", C.c_float * 6), ("init_alpha1", C.c_float), ("init_T1", C.c_float),
                ("init_sigma", C.c_float), ("init_mu_h_floor", C.c_float),
                ("init_mu_s_ceil", C.c_float), ("init_eta_lo", C.c_float),
                ("init_eta_hi", C.c_float), ("init_mode", C.c_int32), ("init_state", C.c_void_p),
                ("noise_sd", C.c_void_p)]


class Scene_t(C.Structure):
    _fields_ = [("n_pix", C.c_int64), ("radiance", C.c_void_p), ("wv_bin", C.c_void_p),
                ("mem", C.c_int32), ("gate_mode", C.c_int32)]


OUTPUT_FIELDS = ("state", "ET", "sdT", "alpha", "cov", "var_ET", "cost", "rms", "hfdi", "status",
                 "iters", "resid_spec")


class Outputs_t(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in OUTPUT_FIELDS]


class Gemm_t(C.Structure):
    _fields_ = [("A", C.c_void_p), ("lda", C.c_int64), ("B", C.c_void_p), ("ldb", C.c_int64),
                ("M", C.c_int32), ("N", C.c_int32), ("K", C.c_int32), ("epi", C.c_int32),
                ("bias", C.c_void_p), ("mask", C.c_void_p), ("ldm", C.c_int64),
                ("Cf", C.c_void_p), ("ldc", C.c_int64), ("Cb", C.c_void_p), ("ldcb", C.c_int64),
                ("CbT", C.c_void_p), ("ldcbT", C.c_int64), ("accumulate", C.c_int32),
                ("err", C.c_void_p)]


class BatchItem_t(C.Structure):
    _fields_ = [("n_pix", C.c_int64), ("radiance", C.c_void_p), ("wv_bin", C.c_void_p),
                ("out", Outputs_t)]


class Tune_t(C.Structure):
    _fields_ = [("variant", C.c_int32), ("claim", C.c_int32), ("ms", C.c_float)]


class MlpTrain_t(C.Structure):
    _fields_ = [("steps", C.c_int64), ("batch", C.c_int32), ("lr", C.c_float),
                ("pfire", C.c_float), ("noise_rel", C.c_float), ("noise_abs", C.c_float),
                ("seed", C.c_uint64), ("sample0", C.c_int64)]


class Stats_t(C.Structure):
    _fields_ = [("n_pixels", C.c_uint64), ("sum_it1", C.c_uint64), ("sum_it2", C.c_uint64),
                ("n_fp64_pixels", C.c_uint64), ("band_evals1", C.c_uint64),
                ("band_evals2", C.c_uint64), ("node_band_evals2", C.c_uint64),
                ("solves64_1", C.c_uint64), ("solves64_2", C.c_uint64), ("mma_rounds2", C.c_uint64),
                ("status_counts", C.c_uint64 * 8), ("flops", C.c_double),
                ("flops1", C.c_double), ("flops2", C.c_double),
                ("kernel_launches", C.c_int32), ("n_post64", C.c_uint64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise FireError(f"{LIB_PATH} is missing: build it with paper_2608_07580_b300.build")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, f32, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_uint64
    lib.fire_default_config.argtypes = [C.POINTER(Config_t)]
    lib.fire_build_flags.argtypes = []
    lib.fire_build_flags.restype = C.c_int32
    lib.fire_debug_word.argtypes = [vp, C.POINTER(C.c_int32)]
    lib.fire_debug_word.restype = C.c_int
    lib.fire_default_priors.argtypes = [C.POINTER(Priors_t), i32, i32, f32, f32]
    lib.fire_ctx_create.argtypes = [C.POINTER(vp), C.POINTER(Tables_t), C.POINTER(Config_t)]
    lib.fire_ctx_create.restype = C.c_int
    lib.fire_ctx_destroy.argtypes = [vp]
    lib.fire_retrieve.argtypes = [vp, C.POINTER(Scene_t), C.POINTER(Priors_t),
                                  C.POINTER(Outputs_t), vp]
    lib.fire_retrieve.restype = C.c_int
    lib.fire_forward.argtypes = [vp, i32, vp, vp, i64, f32, f32, u64, u64, i64, vp, vp]
    lib.fire_forward.restype = C.c_int
    lib.fire_block_mean.argtypes = [vp, i32, i32, i32, i32, vp, vp]
    lib.fire_wv_presolve.argtypes = [vp, vp, i64, i64, i32, vp, vp, vp, vp]
    lib.fire_wv_presolve.restype = C.c_int
    lib.fire_wv_depth_table.argtypes = [vp, vp, vp]
    lib.fire_wv_depth_table.restype = C.c_int
    lib.fire_inject.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp]
    lib.fire_inject.restype = C.c_int
    lib.fire_hfdi.argtypes = [vp, vp, i64, vp, vp]
    lib.fire_hfdi.restype = C.c_int
    lib.fire_block_mean.restype = C.c_int
    lib.fire_get_stats.argtypes = [vp, C.POINTER(Stats_t)]
    lib.fire_get_stats.restype = C.c_int
    lib.fire_window_bands.argtypes = [vp] + [C.POINTER(C.c_int32)] * 4
    lib.fire_window_bands.restype = C.c_int
    lib.fire_normal_equations.argtypes = [vp, i32, vp, vp, vp, i64, C.POINTER(Priors_t), vp, vp,
                                          vp, vp]
    lib.fire_normal_equations.restype = C.c_int
    lib.fire_gemm_bf16.argtypes = [C.POINTER(Gemm_t), vp]
    lib.fire_gemm_bf16.restype = C.c_int
    lib.fire_mlp_create.argtypes = [C.POINTER(vp), vp, i32, u64]
    lib.fire_mlp_create.restype = C.c_int
    lib.fire_mlp_destroy.argtypes = [vp]
    lib.fire_mlp_train.argtypes = [vp, C.POINTER(MlpTrain_t), vp, vp]
    lib.fire_mlp_train.restype = C.c_int
    lib.fire_mlp_infer.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.fire_mlp_infer.restype = C.c_int
    lib.fire_mlp_gradients.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp]
    lib.fire_mlp_gradients.restype = C.c_int
    lib.fire_mlp_param_count.argtypes = [vp]
    lib.fire_mlp_param_count.restype = i64
    lib.fire_mlp_params.argtypes = [vp, vp, vp]
    lib.fire_mlp_params.restype = C.c_int
    lib.fire_mlp_save.argtypes = [vp, C.c_char_p]
    lib.fire_mlp_save.restype = C.c_int
    lib.fire_mlp_load.argtypes = [vp, C.c_char_p]
    lib.fire_mlp_load.restype = C.c_int
    lib.fire_mlp_next_sample.argtypes = [vp]
    lib.fire_mlp_next_sample.restype = i64
    lib.fire_ctx_set_mlp.argtypes = [vp, vp]
    lib.fire_ctx_set_mlp.restype = C.c_int
    lib.fire_retrieve_batch.argtypes = [vp, C.POINTER(BatchItem_t), i32, C.POINTER(Priors_t), i32, vp]
    lib.fire_retrieve_batch.restype = C.c_int
    lib.fire_graph_capture.argtypes = [vp, C.POINTER(BatchItem_t), i32, C.POINTER(Priors_t), i32,
                                       C.POINTER(vp)]
    lib.fire_graph_capture.restype = C.c_int
    lib.fire_graph_launch.argtypes = [vp, vp]
    lib.fire_graph_launch.restype = C.c_int
    lib.fire_graph_destroy.argtypes = [vp]
    lib.fire_autotune.argtypes = [vp, vp, vp, i64, C.POINTER(Tune_t), vp]
    lib.fire_autotune.restype = C.c_int
    lib.fire_retrieve_static.argtypes = [vp, C.POINTER(Scene_t), C.POINTER(Priors_t),
                                         C.POINTER(Outputs_t), vp]
    lib.fire_retrieve_static.restype = C.c_int
    lib.fire_set_kernel_timing.argtypes = [vp, i32]
    lib.fire_set_kernel_timing.restype = C.c_int
    lib.fire_get_kernel_times.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_int32)]
    lib.fire_get_kernel_times.restype = C.c_int
    lib.fire_set_tuning.argtypes = [vp, i32, i32]
    lib.fire_set_tuning.restype = C.c_int
    lib.fire_status_str.argtypes = [C.c_int]
    lib.fire_status_str.restype = C.c_char_p
    lib.fire_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
    lib.fire_set_allocator.restype = None
    lib.fire_measure_peak.argtypes = [i32, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
    lib.fire_measure_peak.restype = C.c_int
    return lib


lib = _load()


def _check(rc, what):
    if rc != 0:
        raise FireError(f"{what}: {lib.fire_status_str(rc).decode()} ({rc})")


def default_config(**overrides):
    c = Config_t()
    lib.fire_default_config(C.byref(c))
    for k, v in overrides.items():
        if k in ("win1", "win2h", "win2s"):
            setattr(c, k + "_lo", v[0])
            setattr(c, k + "_hi", v[1])
        elif k == "solver" and isinstance(v, str):
            c.solver = {"lm": FIRE_SOLVER_LM, "adam": FIRE_SOLVER_ADAM}[v]
        else:
            setattr(c, k, v)
    return c


def default_priors(n_endm, n_tgrid=64, tgrid=(350.0, 2200.0)):
    p = Priors_t()
    lib.fire_default_priors(C.byref(p), n_endm, n_tgrid, tgrid[0], tgrid[1])
    return p


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t, dtype=None):
    """Device pointer of a contiguous torch CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise FireError("device arguments must be CUDA tensors")
    if not t.is_contiguous():
        raise FireError("device arguments must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise FireError(f"expected {dtype}, got {t.dtype}")
    return t.data_ptr()


class Context:
    """A retrieval context: scene tables resident on the current CUDA device."""

    def __init__(self, tables, config=None, tgrid=(350.0, 2200.0)):
        self._keep = [_f32(tables.wavelength_nm), _f32(tables.solar_irr), _f32(tables.tau_down),
                      _f32(tables.tau_up), _f32(tables.rho_atm), _f32(tables.sph_alb),
                      _f32(tables.endmembers), _f32(getattr(tables, "sat_level", None))]
        k = self._keep
        p = lambda a: None if a is None else a.ctypes.data  # noqa: E731
        self.n_bands = int(k[0].size)
        self.n_endm = int(k[6].shape[0])
        self.n_tgrid = int(getattr(tables, "n_tgrid", 64))
        self.n_wv = int(k[3].shape[0])
        self.tgrid = tgrid
        tb = Tables_t(self.n_bands, int(k[3].shape[0]), self.n_endm, self.n_tgrid, p(k[0]),
                      p(k[1]), float(tables.cos_sza), p(k[2]), p(k[3]), p(k[4]), p(k[5]),
                      p(k[6]), p(k[7]), tgrid[0], tgrid[1])
        self.config = config if config is not None else default_config()
        h = C.c_void_p()
        _check(lib.fire_ctx_create(C.byref(h), C.byref(tb), C.byref(self.config)),
               "fire_ctx_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib.fire_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def default_priors(self):
        return default_priors(self.n_endm, self.n_tgrid, self.tgrid)

    def window_bands(self):
        v = [C.c_int32() for _ in range(4)]
        _check(lib.fire_window_bands(self._h, *[C.byref(x) for x in v]), "fire_window_bands")
        return tuple(x.value for x in v)

    def alloc_outputs(self, n, device=True, resid=False):
        """Output buffers for n pixels: torch CUDA tensors (device) or numpy
        (host); resid adds the residual spectrum [n, n_bands]."""
        ns = self.n_endm + 8
        shapes = {"state": ((n, ns), "f4"), "ET": ((n,), "f4"), "sdT": ((n,), "f4"),
                  "alpha": ((n,), "f4"), "cov": ((n, 21), "f4"), "var_ET": ((n,), "f4"),
                  "cost": ((n,), "f4"), "rms": ((n,), "f4"), "hfdi": ((n,), "f4"),
                  "status": ((n,), "u1"), "iters": ((n, 2), "u2")}
        if resid:
            shapes["resid_spec"] = ((n, self.n_bands), "f4")
        if device:
            import torch
            tm = {"f4": torch.float32, "u1": torch.uint8, "u2": torch.int16}
            return {k: torch.empty(s, dtype=tm[d], device="cuda") for k, (s, d) in shapes.items()}
        return {k: np.empty(s, dtype=d) for k, (s, d) in shapes.items()}

    def set_mlp(self, mlp):
        """Attach a trained network: retrieve(..., learned_start=True) then
        starts every pixel from its proposal (with the plain-LM fallback)."""
        _check(lib.fire_ctx_set_mlp(self._h, None if mlp is None else mlp._h), "fire_ctx_set_mlp")
        self._mlp = mlp

    def _priors(self, priors, noise_sd):
        pri = Priors_t()
        C.memmove(C.byref(pri), C.byref(priors if priors is not None else self.default_priors()),
                  C.sizeof(Priors_t))
        if noise_sd is not None:
            self._nsd = np.ascontiguousarray(noise_sd, dtype=np.float32)
            if self._nsd.shape != (self.n_bands,):
                raise FireError("noise_sd must have one value per band")
            pri.noise_sd = self._nsd.ctypes.data
        return pri

    def retrieve(self, radiance, wv_bin, priors=None, init_state=None, gate_hfdi=False,
                 outputs=None, stream=None, learned_start=False, noise_sd=None, resid=False):
        """Fit every pixel. radiance [n, n_bands] float32 and wv_bin [n] (uint16
        numpy or int16/uint16-bit torch): torch CUDA tensors for device
        scenes, numpy arrays for host scenes (staged inside the call).
        noise_sd: per-band noise sd (numpy, host) weighting the loss; resid:
        also return the residual spectrum."""
        import torch
        host = isinstance(radiance, np.ndarray)
        n = int(radiance.shape[0])
        if outputs is None:
            outputs = self.alloc_outputs(n, device=not host, resid=resid)
        pri = self._priors(priors, noise_sd)
        if learned_start:
            pri.init_mode = FIRE_INIT_MLP
        if host:
            rad = np.ascontiguousarray(radiance, dtype=np.float32)
            wv = np.ascontiguousarray(wv_bin, dtype=np.uint16)
            self._hold = [rad, wv]
            sc = Scene_t(n, rad.ctypes.data, wv.ctypes.data, FIRE_MEM_HOST, int(bool(gate_hfdi)))
            if init_state is not None:
                ini = np.ascontiguousarray(init_state, dtype=np.float32)
                self._hold.append(ini)
                pri.init_mode, pri.init_state = FIRE_INIT_GIVEN, ini.ctypes.data
            ptr = lambda k: None if outputs.get(k) is None else outputs[k].ctypes.data  # noqa
            stream_p = C.c_void_p(0)
        else:
            sc = Scene_t(n, _dptr(radiance, torch.float32), _dptr(wv_bin), FIRE_MEM_DEVICE,
                         int(bool(gate_hfdi)))
            if wv_bin.element_size() != 2:
                raise FireError("wv_bin must be a 16-bit tensor")
            if init_state is not None:
                pri.init_mode, pri.init_state = FIRE_INIT_GIVEN, _dptr(init_state, torch.float32)
            ptr = lambda k: _dptr(outputs.get(k))  # noqa: E731
            stream_p = _stream_ptr(stream)
        o = Outputs_t(*[ptr(k) for k in OUTPUT_FIELDS])
        _check(lib.fire_retrieve(self._h, C.byref(sc), C.byref(pri), C.byref(o), stream_p),
               "fire_retrieve")
        return outputs

    def retrieve_static(self, radiance, wv_bin, priors=None, init_state=None, gate_hfdi=False,
                        outputs=None, stream=None, noise_sd=None):
        """fire_retrieve_static: the plain-LM fit of a device scene (at most
        STATIC_MAX_PIX pixels) through the library's static scratch, without
        any allocation inside the call."""
        import torch
        n = int(radiance.shape[0])
        if outputs is None:
            outputs = self.alloc_outputs(n)
        pri = self._priors(priors, noise_sd)
        if wv_bin.element_size() != 2:
            raise FireError("wv_bin must be a 16-bit tensor")
        if init_state is not None:
            pri.init_mode, pri.init_state = FIRE_INIT_GIVEN, _dptr(init_state, torch.float32)
        sc = Scene_t(n, _dptr(radiance, torch.float32), _dptr(wv_bin), FIRE_MEM_DEVICE,
                     int(bool(gate_hfdi)))
        o = Outputs_t(*[_dptr(outputs.get(k)) for k in OUTPUT_FIELDS])
        _check(lib.fire_retrieve_static(self._h, C.byref(sc), C.byref(pri), C.byref(o),
                                        _stream_ptr(stream)), "fire_retrieve_static")
        return outputs

    def forward(self, mode, state, wv_bin, noise_rel=0.0, noise_abs=0.0, seed=0, stream_id=1,
                pixel_offset=0, out=None, stream=None):
        """Forward model (Eq. fm) on the device; state / wv_bin torch CUDA tensors."""
        import torch
        n = int(state.shape[0])
        if out is None:
            out = torch.empty((n, self.n_bands), dtype=torch.float32, device="cuda")
        _check(lib.fire_forward(self._h, mode, _dptr(state, torch.float32), _dptr(wv_bin), n,
                                noise_rel, noise_abs, seed, stream_id, pixel_offset,
                                _dptr(out, torch.float32), _stream_ptr(stream)), "fire_forward")
        return out

    def _items(self, scenes, outputs):
        import torch
        arr = (BatchItem_t * len(scenes))()
        for i, ((rad, wv), out) in enumerate(zip(scenes, outputs)):
            ptr = lambda k: _dptr(out.get(k))  # noqa: E731
            arr[i] = BatchItem_t(int(rad.shape[0]), _dptr(rad, torch.float32), _dptr(wv),
                                 Outputs_t(*[ptr(k) for k in OUTPUT_FIELDS]))
        return arr

    def retrieve_batch(self, scenes, outputs=None, priors=None, gate_hfdi=False, stream=None):
        """Fit several scenes [(radiance, wv_bin), ...] (device tensors) in one launch."""
        if outputs is None:
            outputs = [self.alloc_outputs(int(r.shape[0])) for r, _ in scenes]
        arr = self._items(scenes, outputs)
        pr = None if priors is None else C.byref(priors)
        _check(lib.fire_retrieve_batch(self._h, arr, len(scenes), pr, int(bool(gate_hfdi)),
                                       _stream_ptr(stream)), "fire_retrieve_batch")
        return outputs

    def capture_batch(self, scenes, outputs, priors=None, gate_hfdi=False):
        """CUDA graph of retrieve_batch over these buffers (replay with .launch())."""
        arr = self._items(scenes, outputs)
        h = C.c_void_p()
        pr = None if priors is None else C.byref(priors)
        _check(lib.fire_graph_capture(self._h, arr, len(scenes), pr, int(bool(gate_hfdi)),
                                      C.byref(h)), "fire_graph_capture")
        return BatchGraph(h, self, scenes, outputs)

    def autotune(self, radiance, wv_bin, stream=None):
        import torch
        t = Tune_t()
        _check(lib.fire_autotune(self._h, _dptr(radiance, torch.float32), _dptr(wv_bin),
                                 int(radiance.shape[0]), C.byref(t), _stream_ptr(stream)),
               "fire_autotune")
        return {"variant": t.variant, "claim": t.claim, "ms": t.ms}

    def set_kernel_timing(self, on=True):
        _check(lib.fire_set_kernel_timing(self._h, int(bool(on))), "fire_set_kernel_timing")

    def kernel_times(self):
        """Summed ms of (stage 1, stage 2, finalize) over the timed fits, and their count."""
        ms = (C.c_float * 3)()
        n = C.c_int32()
        _check(lib.fire_get_kernel_times(self._h, ms, C.byref(n)), "fire_get_kernel_times")
        return list(ms), n.value

    def set_tuning(self, variant, claim):
        _check(lib.fire_set_tuning(self._h, variant, claim), "fire_set_tuning")

    def normal_equations(self, stage, radiance, wv_bin, states, priors=None, stream=None,
                         noise_sd=None):
        """(H, g, cost) of one stage at the given states (device tensors)."""
        import torch
        n = int(states.shape[0])
        P = self.n_endm + 1 if stage == 1 else 6
        H = torch.empty((n, P, P), dtype=torch.float32, device="cuda")
        g = torch.empty((n, P), dtype=torch.float32, device="cuda")
        cost = torch.empty((n,), dtype=torch.float32, device="cuda")
        pr = C.byref(self._priors(priors, noise_sd))
        _check(lib.fire_normal_equations(self._h, stage, _dptr(radiance, torch.float32),
                                         _dptr(wv_bin), _dptr(states, torch.float32), n, pr,
                                         _dptr(H), _dptr(g), _dptr(cost), _stream_ptr(stream)),
               "fire_normal_equations")
        return H, g, cost

    def hfdi(self, radiance, out=None, stream=None):
        """fire_hfdi: the gate index of every pixel (torch CUDA tensors)."""
        import torch
        n = int(radiance.shape[0])
        if out is None:
            out = torch.empty((n,), dtype=torch.float32, device="cuda")
        _check(lib.fire_hfdi(self._h, _dptr(radiance, torch.float32), n, _dptr(out, torch.float32),
                             _stream_ptr(stream)), "fire_hfdi")
        return out

    def inject(self, radiance_bg, wv_bin, alpha, T, out=None, stream=None):
        """fire_inject (Eq. inject): radiance_bg + alpha tau_up B(lambda, T),
        all torch CUDA tensors."""
        import torch
        n = int(radiance_bg.shape[0])
        if out is None:
            out = torch.empty_like(radiance_bg)
        _check(lib.fire_inject(self._h, _dptr(radiance_bg, torch.float32), _dptr(wv_bin),
                               _dptr(alpha, torch.float32), _dptr(T, torch.float32), n,
                               _dptr(out, torch.float32), _stream_ptr(stream)), "fire_inject")
        return out

    def wv_depth_table(self, lams=None):
        """fire_wv_depth_table: the 940 nm depth of every water-vapour bin."""
        D = np.empty(self.n_wv, dtype=np.float32)
        lp = None if lams is None else np.ascontiguousarray(lams, dtype=np.float32)
        _check(lib.fire_wv_depth_table(self._h, None if lp is None else lp.ctypes.data, D.ctypes.data),
               "fire_wv_depth_table")
        return D

    def wv_presolve(self, radiance, width, height, block=12, lams=None, depth=False, out=None,
                    stream=None):
        """fire_wv_presolve: per-pixel water-vapour bins (int16 CUDA tensor
        holding the uint16 bits) from device radiance in row-major image
        order; with depth, also the per-pixel 940 nm depths."""
        import torch
        n = int(width) * int(height)
        if out is None:
            out = torch.empty((n,), dtype=torch.int16, device="cuda")
        d = torch.empty((n,), dtype=torch.float32, device="cuda") if depth else None
        lp = None if lams is None else np.ascontiguousarray(lams, dtype=np.float32)
        _check(lib.fire_wv_presolve(self._h, _dptr(radiance, torch.float32), int(width), int(height), int(block),
                                    None if lp is None else lp.ctypes.data, _dptr(out), _dptr(d),
                                    _stream_ptr(stream)), "fire_wv_presolve")
        return (out, d) if depth else out

    def stats(self):
        s = Stats_t()
        _check(lib.fire_get_stats(self._h, C.byref(s)), "fire_get_stats")
        d = {f: getattr(s, f) for f, _ in Stats_t._fields_ if f != "status_counts"}
        d["status_counts"] = list(s.status_counts)
        return d

    def debug_word(self):
        """The device error word after the last fit (fire_debug_word): 0, 1 (a
        bounded wait gave up) or 0x100 | site (a failed index check)."""
        w = C.c_int32(0)
        _check(lib.fire_debug_word(self._h, C.byref(w)), "fire_debug_word")
        return w.value


def build_flags():
    """fire_build_flags: bit 0 set in the bounds-checked build."""
    return int(lib.fire_build_flags())


PEAK_KINDS = {"fp32_fma": 0, "fp32_fma2": 1, "sfu_ex2": 2, "fp64_fma": 3}


def measure_peak(kind, stream=None):
    """Measured rate of one arithmetic unit (fire_measure_peak): flop/s for
    the FMA kinds, operations/s for the SFU's ex2."""
    r, sec = C.c_double(), C.c_double()
    _check(lib.fire_measure_peak(PEAK_KINDS[kind], C.byref(r), C.byref(sec), _stream_ptr(stream)),
           "fire_measure_peak")
    return r.value, sec.value


def block_mean(src, width, height, n_bands, block=12, stream=None):
    """Block mean of a BIP cube [height*width, n_bands] (torch CUDA) -> coarse cube."""
    import torch
    cw, ch = width // block, height // block
    dst = torch.empty((ch * cw, n_bands), dtype=torch.float32, device="cuda")
    _check(lib.fire_block_mean(_dptr(src, torch.float32), width, height, n_bands, block,
                               _dptr(dst), _stream_ptr(stream)), "fire_block_mean")
    return dst


def gemm_bf16(A, B, epi=0, bias=None, mask=None, Cf=None, Cb=None, CbT=None, accumulate=False,
              err=None, stream=None):
    """C = A B^T on the tensor cores (A [M, K], B [N, K] bf16 CUDA tensors)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    g = Gemm_t(_dptr(A, torch.bfloat16), A.stride(0), _dptr(B, torch.bfloat16), B.stride(0),
               M, N, K, epi, _dptr(bias), _dptr(mask), 0 if mask is None else mask.stride(0),
               _dptr(Cf), 0 if Cf is None else Cf.stride(0), _dptr(Cb),
               0 if Cb is None else Cb.stride(0), _dptr(CbT), 0 if CbT is None else CbT.stride(0),
               int(bool(accumulate)), _dptr(err))
    _check(lib.fire_gemm_bf16(C.byref(g), _stream_ptr(stream)), "fire_gemm_bf16")


class BatchGraph:
    """A captured batched fit; keeps its buffers alive."""

    def __init__(self, h, ctx, scenes, outputs):
        self._h, self.ctx, self._keep = h, ctx, (scenes, outputs)

    def launch(self, stream=None):
        _check(lib.fire_graph_launch(self._h, _stream_ptr(stream)), "fire_graph_launch")

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib.fire_graph_destroy(self._h)
                self._h = None
        except Exception:
            pass


class MLP:
    """The learned initial-state proposal of a context (tensor-core MLP)."""

    def __init__(self, ctx, hidden=512, seed=0):
        h = C.c_void_p()
        _check(lib.fire_mlp_create(C.byref(h), ctx._h, hidden, seed), "fire_mlp_create")
        self._h, self.ctx, self.hidden = h, ctx, hidden
        self.din = (ctx.n_bands + 15) // 16 * 16

    def close(self):
        if getattr(self, "_h", None):
            lib.fire_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def train(self, steps, batch=4096, lr=1e-3, pfire=0.5, noise_rel=0.005, noise_abs=1e-4,
              seed=0, sample0=None, stream=None):
        """Adam steps on fresh synthetic batches; returns the per-step losses."""
        if sample0 is None:
            sample0 = lib.fire_mlp_next_sample(self._h)
        cfg = MlpTrain_t(steps, batch, lr, pfire, noise_rel, noise_abs, seed, sample0)
        loss = np.zeros(max(steps, 1), dtype=np.float32)
        _check(lib.fire_mlp_train(self._h, C.byref(cfg), loss.ctypes.data, _stream_ptr(stream)),
               "fire_mlp_train")
        return loss[:steps]

    def infer(self, radiance, stream=None):
        import torch
        n = int(radiance.shape[0])
        z = torch.empty((n, 16), dtype=torch.float32, device="cuda")
        init = torch.empty((n, self.ctx.n_endm + 8), dtype=torch.float32, device="cuda")
        _check(lib.fire_mlp_infer(self._h, _dptr(radiance, torch.float32), n, _dptr(z), _dptr(init),
                                  _stream_ptr(stream)), "fire_mlp_infer")
        return z, init

    def gradients(self, x, tgt, msk, stream=None):
        """Gradients of the masked MSE at standardised inputs x [B, Din] (fp32)."""
        import torch
        B = int(x.shape[0])
        H, D = self.hidden, self.din
        n = H * D + H + H * H + H + H * 16 + 16
        g = torch.empty(n, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        _check(lib.fire_mlp_gradients(self._h, _dptr(x, torch.float32), _dptr(tgt, torch.float32),
                                      _dptr(msk, torch.float32), B, _dptr(g), _dptr(loss),
                                      _stream_ptr(stream)), "fire_mlp_gradients")
        g = g.cpu().numpy()
        o, out = 0, {}
        for k, shp in (("W1", (H, D)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                       ("W3T", (H, 16)), ("b3", (16,))):
            sz = int(np.prod(shp))
            out[k] = g[o:o + sz].reshape(shp)
            o += sz
        return out, float(loss.item())

    def params(self, set_params=None):
        """Get (and optionally set) the packed parameters as a dict of arrays."""
        H, D = self.hidden, self.din
        n = lib.fire_mlp_param_count(self._h)
        shapes = (("W1", (H, D)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (16, H)),
                  ("b3", (16,)), ("mean", (D,)), ("istd", (D,)))
        if set_params is not None:
            flat = np.concatenate([np.asarray(set_params[k], np.float32).ravel() for k, _ in shapes])
            assert flat.size == n
            _check(lib.fire_mlp_params(self._h, None, flat.ctypes.data), "fire_mlp_params")
        buf = np.empty(n, dtype=np.float32)
        _check(lib.fire_mlp_params(self._h, buf.ctypes.data, None), "fire_mlp_params")
        o, out = 0, {}
        for k, shp in shapes:
            sz = int(np.prod(shp))
            out[k] = buf[o:o + sz].reshape(shp)
            o += sz
        return out

    def save(self, path):
        _check(lib.fire_mlp_save(self._h, str(path).encode()), "fire_mlp_save")

    def load(self, path):
        _check(lib.fire_mlp_load(self._h, str(path).encode()), "fire_mlp_load")

    @property
    def next_sample(self):
        return lib.fire_mlp_next_sample(self._h)
