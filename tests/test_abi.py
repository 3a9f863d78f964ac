"""The C-ABI library loads and exports every symbol include/*.h declares;
host-side defaults and argument checks work without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(fire_\w+)\s*\(", src, re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2608_07580_b300 import build
    lib = C.CDLL(build.build())
    declared = _declared()
    assert {"fire_ctx_create", "fire_retrieve", "fire_forward"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), name


def test_binding_symbols_match_header():
    from paper_2608_07580_b300 import firert
    assert set(firert.SYMBOLS) <= _declared()


def test_defaults_match_paper_and_oracle():
    from paper_2608_07580_b300 import firert
    import oracle
    c = firert.default_config()
    o = oracle.Config()
    assert (c.win1_lo, c.win1_hi) == o.win1
    assert (c.win2h_lo, c.win2h_hi) == o.win2h and (c.win2s_lo, c.win2s_hi) == o.win2s
    # the stage-2 cap of the FP32 path is 1.5 x the oracle's (its normal
    # matrix resolves the mixture's flat directions less well); stage 1 equal
    assert c.max_it1 == o.max_it1 and c.max_it2 == 3 * o.max_it2 // 2
    for k in ("tau0", "tol_g", "tol_x", "tol_f", "kappa_max", "dfloor", "noise_rel", "noise_abs",
              "hfdi_thresh", "ident_sd_et", "ident_alpha_snr"):
        assert abs(getattr(c, k) - getattr(o, k)) <= 1e-6 * abs(getattr(o, k)), k
    p = firert.default_priors(3)
    assert np.allclose(np.array(p.lo1[:5]), o.lo1, rtol=1e-6)
    assert np.allclose(np.array(p.hi1[:5]), o.hi1, rtol=1e-6)
    assert np.allclose(np.array(p.lo2[:]), o.lo2, rtol=1e-6)
    assert np.allclose(np.array(p.hi2[:]), o.hi2, rtol=1e-6)
    assert np.allclose(np.array(p.pm1[:5]), o.pm1) and np.allclose(np.array(p.pp1[:5]), o.pp1)
    assert np.allclose(np.array(p.pm2[:]), o.pm2) and np.allclose(np.array(p.pp2[:]), o.pp2)
    assert np.allclose([p.init_alpha1, p.init_T1, p.init_sigma, p.init_mu_h_floor, p.init_mu_s_ceil,
                        p.init_eta_lo, p.init_eta_hi],
                       [o.init_alpha1, o.init_T1, o.init_sigma, o.init_mu_h_floor, o.init_mu_s_ceil,
                        *o.init_eta], rtol=1e-6)


def test_null_arguments_are_rejected_without_gpu():
    from paper_2608_07580_b300 import firert
    lib = firert.lib
    assert lib.fire_ctx_create(None, None, None) == 1
    h = C.c_void_p()
    assert lib.fire_ctx_create(C.byref(h), None, None) == 1
    assert lib.fire_retrieve(None, None, None, None, None) == 1
    assert lib.fire_status_str(4) == b"unsupported shape"


def test_allocator_hook_failure_gives_nomem_without_gpu():
    """A failing allocator installed through fire_set_allocator makes
    fire_ctx_create return FIRE_ERR_NOMEM at its first device allocation
    (no GPU needed: the hook answers before the runtime is asked)."""
    import synth
    from paper_2608_07580_b300 import firert
    calls = []

    def alloc(n, user):
        calls.append(n)
        return None

    a, f = firert.ALLOC_FN(alloc), firert.FREE_FN(lambda p, u: None)
    firert.lib.fire_set_allocator(a, f, None)
    try:
        with pytest.raises(firert.FireError, match="out of memory"):
            firert.Context(synth.make_tables())
    finally:
        firert.lib.fire_set_allocator(firert.ALLOC_FN(), firert.FREE_FN(), None)
    assert len(calls) == 1 and calls[0] > 0


def test_config_and_priors_layout_carry_the_new_fields():
    from paper_2608_07580_b300 import firert
    c = firert.default_config()
    assert c.wait_spins == 0                  # 0 = the default limit
    p = firert.default_priors(3)
    assert p.noise_sd is None                 # unweighted Eq. (loss) by default
    assert "resid_spec" in firert.OUTPUT_FIELDS


def test_bounds_checked_build_exports_every_symbol_and_says_so():
    """The FIRERT_DEBUG build (libfirert_debug.so): same ABI, build flag set;
    the release build's flag is clear."""
    from paper_2608_07580_b300 import build
    dbg = C.CDLL(build.build(debug=True))
    rel = C.CDLL(build.build())
    for name in sorted(_declared()):
        assert hasattr(dbg, name), name
    dbg.fire_build_flags.restype = rel.fire_build_flags.restype = C.c_int32
    assert dbg.fire_build_flags() & 1 == 1
    assert rel.fire_build_flags() & 1 == 0
    dbg.fire_status_str.restype = C.c_char_p
    assert b"index check" in dbg.fire_status_str(8)
