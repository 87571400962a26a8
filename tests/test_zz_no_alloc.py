"""ctqw_propagate_taylor_noalloc: the per-term Taylor propagation for callers
that cannot allocate device memory (in loops that must not synchronize the
device through cudaMalloc, or as a plugin of a host program that owns the
memory budget).  Its scratch is a fixed 48 MiB array
inside the library.  Checked through the C ABI against the entry point that
takes a caller-provided workspace, on two different calls in a row (so the
second call runs on a scratch array the first one has filled), and
against the FP64 oracle.

This file is named to be collected last, so that a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import ctqw_workloads as cw
from gpu_helpers import TOL_FP32, TOL_FP64, TOL_NORM_DRIFT, energy_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctqw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_00746_gb300 import build, ctqw as c

    build.build()
    lib = c.load()
    f = lib.ctqw_propagate_taylor_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [vp, ctypes.c_int32, vp, ctypes.c_double, ctypes.c_int32, ctypes.c_int64,
                  ctypes.c_int32, vp, vp, vp, vp]
    f.restype = ctypes.c_int
    return c


def _run(ctqw, w, noalloc):
    h = ctqw.build_for_workload(w)
    psi = h.new_state(w.dtype)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), w.dtype)
    n_obs = h.n_obs(w.n_steps, w.obs_every)
    P = torch.empty((n_obs, h.p_width), dtype=torch.float64, device="cuda")
    nr = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    en = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    if noalloc:
        st = ctqw.load().ctqw_propagate_taylor_noalloc(h.handle, w.dtype, ptr(psi), w.dt, w.K,
                                                      w.n_steps, w.obs_every, ptr(P), ptr(nr),
                                                      ptr(en), stream)
        assert st == ctqw.CTQW_OK, ctqw.load().ctqw_last_error()
    else:
        ws = h.workspace(w.dtype, ctqw.TAYLOR, ctqw.FLAG_PLAIN)
        ctqw.ctqw_propagate_taylor(h, psi, w.dtype, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en,
                                   ctqw.FLAG_PLAIN, ws)
    ctqw.ctqw_check_status(h)
    out = [psi.cpu().numpy(), P.cpu().numpy(), nr.cpu().numpy(), en.cpu().numpy()]
    h.close()
    return out


def test_noalloc_matches_workspace_entry_point_on_two_calls(ctqw):
    """Two calls in a row, each against the workspace entry point and against
    the FP64 oracle (P, norm and energy), so that a fault both entry points
    share cannot pass unseen."""
    import oracle

    first = cw.get("bosons_small").with_(dtype=cw.C128, R=4, n_steps=40, obs_every=10)
    second = cw.get("ring3_small").with_(dtype=cw.C64, N=9, R=2, n_steps=30, obs_every=15)
    for w, tol in ((first, TOL_FP64), (second, TOL_FP32)):
        ref = _run(ctqw, w, noalloc=False)
        got = _run(ctqw, w, noalloc=True)
        for a, b in zip(got, ref):
            assert a.shape == b.shape
            assert np.max(np.abs(a - b)) <= tol
        o = oracle.ensemble_run(w)
        e_tol = 1e-10 if w.dtype == cw.C128 else energy_tol(w)
        assert np.max(np.abs(got[1] - o["P_mean"])) <= tol
        assert np.max(np.abs(got[2] - o["norm"].T)) <= (1e-12 if w.dtype == cw.C128 else TOL_NORM_DRIFT)
        assert np.max(np.abs(got[3] - o["energy"].T)) <= e_tol


def test_noalloc_rejects_a_handle_of_another_device(ctqw):
    """The scratch address is per device, so the call wants the handle's
    device current.  With one GPU the check is seen through a second device
    ordinal only when there is one; here it must at least accept the
    handle's own device."""
    w = cw.get("bosons_small").with_(dtype=cw.C128, R=1, n_steps=2, obs_every=1)
    got = _run(ctqw, w, noalloc=True)
    assert np.isfinite(got[2]).all()
    if torch.cuda.device_count() > 1:
        h = ctqw.build_for_workload(w)
        psi = h.new_state(cw.C128)
        with torch.cuda.device(1):
            st = ctqw.load().ctqw_propagate_taylor_noalloc(
                h.handle, cw.C128, ctypes.c_void_p(psi.data_ptr()), w.dt, w.K, 1, 0, None, None, None, None)
        assert st == ctqw.CTQW_EINVAL and b"device" in ctqw.load().ctqw_last_error()
        h.close()


def test_noalloc_rejects_states_beyond_its_scratch(ctqw):
    w = cw.get("bosons_small").with_(dtype=cw.C128, N=1100, R=1, n_steps=1, obs_every=0)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C128)
    lib = ctqw.load()
    st = lib.ctqw_propagate_taylor_noalloc(h.handle, cw.C128, ctypes.c_void_p(psi.data_ptr()),
                                           w.dt, w.K, 1, 0, None, None, None,
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == ctqw.CTQW_EINVAL
    assert b"scratch" in lib.ctqw_last_error()
    h.close()
