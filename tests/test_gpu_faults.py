"""Failure handling on the GPU without faulting it: a bounded device wait
made to run out (the wait limit is a config field; the wait gives up,
drains its own copies, frees its tensor memory and the call reports
FIRE_ERR_TIMEOUT, after which the device is still usable), and allocation
failure through the injectable allocator hook (FIRE_ERR_NOMEM), plus a
caller allocator that serves the library from torch's pool."""
import ctypes as C

import numpy as np
import pytest

from scenes import config1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2608_07580_b300 import firert
    return torch, firert


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def test_bounded_wait_runs_out_and_is_reported(env):
    torch, fr = env
    t, tr, L = config1(width=32, height=32)
    good = fr.Context(t)
    ref = {k: v.cpu().numpy() for k, v in good.retrieve(_dev(torch, L, torch.float32),
                                                        _dev(torch, tr.wv_bin.astype(np.int16),
                                                             torch.int16)).items()}
    for variant in (6, 3):
        ctx = fr.Context(t, fr.default_config(wait_spins=1))
        ctx.set_tuning(variant, 2)
        # host scene: the call synchronises and reports the timeout itself
        with pytest.raises(fr.FireError, match="timed out"):
            ctx.retrieve(L, tr.wv_bin)
        # device scene: the call returns; the next statistics report it
        ctx.retrieve(_dev(torch, L, torch.float32), _dev(torch, tr.wv_bin.astype(np.int16), torch.int16))
        with pytest.raises(fr.FireError, match="timed out"):
            ctx.stats()
        ctx.close()
    # the device and the library are still usable, with the same results
    torch.cuda.synchronize()
    again = {k: v.cpu().numpy() for k, v in good.retrieve(_dev(torch, L, torch.float32),
                                                          _dev(torch, tr.wv_bin.astype(np.int16),
                                                               torch.int16)).items()}
    for k in ("ET", "alpha", "status", "cov"):
        assert np.array_equal(ref[k], again[k], equal_nan=True), k
    good.stats()   # no error left behind


def test_allocation_failure_reports_nomem(env):
    torch, fr = env
    t, tr, L = config1(width=32, height=32)
    ctx = fr.Context(t)                           # made with cudaMalloc
    fail = fr.ALLOC_FN(lambda n, u: None)
    nofree = fr.FREE_FN(lambda p, u: None)
    fr.lib.fire_set_allocator(fail, nofree, None)
    try:
        with pytest.raises(fr.FireError, match="out of memory"):
            ctx.retrieve(L, tr.wv_bin)             # scratch and staging
        with pytest.raises(fr.FireError, match="out of memory"):
            fr.Context(t)
    finally:
        fr.lib.fire_set_allocator(fr.ALLOC_FN(), fr.FREE_FN(), None)
    out = ctx.retrieve(L, tr.wv_bin)               # recovers once memory is there
    assert np.isfinite(out["ET"][(out["status"] & 7) == 0]).all()
    ctx.close()                                    # earlier blocks return to cudaFree


def test_caller_allocator_serves_the_library(env):
    """A caller allocator (here torch's caching allocator) serves every
    device allocation of a context; its blocks go back to it on destroy,
    and the results equal those of the default allocator bit for bit."""
    torch, fr = env
    t, tr, L = config1(width=32, height=32)
    live = {}

    def alloc(n, user):
        p = torch.cuda.caching_allocator_alloc(int(n))
        live[p] = n
        return p

    def free(p, user):
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    a, f = fr.ALLOC_FN(alloc), fr.FREE_FN(free)
    fr.lib.fire_set_allocator(a, f, None)
    try:
        ctx = fr.Context(t)
        got = ctx.retrieve(L, tr.wv_bin)
        assert len(live) >= 5
    finally:
        fr.lib.fire_set_allocator(fr.ALLOC_FN(), fr.FREE_FN(), None)
    ref = fr.Context(t).retrieve(L, tr.wv_bin)
    for k in ("ET", "alpha", "state", "status"):
        assert np.array_equal(got[k], ref[k], equal_nan=True), k
    ctx.close()
    assert not live                                # every block returned to its allocator
