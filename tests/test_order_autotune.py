"""The order autotuner (Sec. 2.3 truncation bound; the order is the smallest
that keeps the summed remainder of the run within a tenth of the tolerance).

Host-only checks through the C ABI (ctqw_taylor_order needs no device),
against the oracle's remainder bound and norm bound searched by brute force.
"""
import math

import pytest

import oracle

CTQW_OK, CTQW_EINVAL, CTQW_EUNSUPPORTED = 0, 1, 4


@pytest.fixture(scope="module")
def ctqw():
    from paper_1612_00746_gb300 import build, ctqw as c

    build.build()
    c.load()
    return c


def brute_force_order(h_dt, n_steps, tol, K_min, K_max):
    for K in range(K_min, K_max + 1):
        if max(n_steps, 1) * oracle.taylor_truncation_bound(h_dt, K) <= tol / 10:
            return K
    return None


@pytest.mark.parametrize("h_dt,n_steps,tol", [
    (0.05, 1000, 1e-11), (0.18, 2500, 2e-6), (0.16, 1000, 2e-6), (0.088, 1000, 2e-6),
    (0.15, 1000, 2e-6), (0.4, 10, 1e-11), (1e-3, 1, 2e-6), (0.0, 5, 2e-6),
])
def test_order_matches_brute_force_search_of_the_bound(ctqw, h_dt, n_steps, tol):
    K, bound = ctqw.ctqw_taylor_order(h_dt, n_steps, tol, 1, 30)
    assert K == brute_force_order(h_dt, n_steps, tol, 1, 30)
    assert bound <= tol / 10
    assert bound == pytest.approx(max(n_steps, 1) * oracle.taylor_truncation_bound(h_dt, K), rel=1e-12)
    if K > 1:   # one order less would not do
        assert max(n_steps, 1) * oracle.taylor_truncation_bound(h_dt, K - 1) > tol / 10


def test_ragged_batch_order_in_its_range(ctqw):
    # ragged batch: 2 particles, eps ~ U[-1,1], J = 1 + U[-0.25,0.25], U = 1, dt = 0.02, 1000 steps
    h_dt = oracle.hamiltonian_norm_bound(2, 1.0, 1.25, 1.0) * 0.02
    assert h_dt == pytest.approx(0.16)
    assert ctqw.ctqw_taylor_order(h_dt, 1000, 2e-6, 8, 20)[0] == 8
    assert ctqw.ctqw_taylor_order(h_dt, 1000, 2e-6, 1, 30)[0] == 7
    # the FP64 tolerance needs more terms
    assert ctqw.ctqw_taylor_order(h_dt, 1000, 1e-11, 1, 30)[0] == brute_force_order(h_dt, 1000, 1e-11, 1, 30)


def test_no_order_in_range(ctqw):
    lib = ctqw.load()
    import ctypes

    K = ctypes.c_int32()
    b = ctypes.c_double()
    st = lib.ctqw_taylor_order(2.0, 1000, 1e-11, 1, 5, ctypes.byref(K), ctypes.byref(b))
    assert st == CTQW_EUNSUPPORTED
    assert K.value == 5
    assert b.value == pytest.approx(1000 * oracle.taylor_truncation_bound(2.0, 5))


@pytest.mark.parametrize("args", [(-0.1, 10, 1e-6, 1, 30), (0.1, -1, 1e-6, 1, 30), (0.1, 10, 0.0, 1, 30),
                                  (0.1, 10, 1e-6, 0, 30), (0.1, 10, 1e-6, 5, 31), (0.1, 10, 1e-6, 9, 8),
                                  (math.inf, 10, 1e-6, 1, 30)])
def test_bad_arguments(ctqw, args):
    import ctypes

    K = ctypes.c_int32()
    assert ctqw.load().ctqw_taylor_order(*args, ctypes.byref(K), None) == CTQW_EINVAL


def test_order_grows_with_run_length_and_step(ctqw):
    prev = 0
    for n in (1, 10, 100, 1000, 10000):
        K = ctqw.ctqw_taylor_order(0.16, n, 2e-6)[0]
        assert K >= prev
        prev = K
    prev = 0
    for h in (0.01, 0.05, 0.1, 0.2, 0.4):
        K = ctqw.ctqw_taylor_order(h, 1000, 2e-6)[0]
        assert K >= prev
        prev = K
