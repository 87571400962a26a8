"""Parity of the temporally blocked tiled kernels (D Horner stages per launch
on tiles with halos; the iterate in shared memory, shape 0, or in registers,
shapes 1..6; the library's default picks its depth from K) with the FP64
oracle, through the C ABI.

Cases: every compiled depth, lattice sides that are not multiples of the
tile and smaller than one region, open chains and rings, K not a multiple
of D and K < D, ragged batches, bosons with U, distinguishable walkers.
"""
import numpy as np
import pytest

import ctqw_workloads as cw
import oracle
from gpu_helpers import TOL_FP32, TOL_NORM_DRIFT, energy_tol, per_realization_P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctqw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_00746_gb300 import build, ctqw as c

    build.build()
    c.load()
    return c


def _check(got, ref, w):
    dP = np.max(np.abs(got["P_mean"] - ref["P_mean"]))
    dn = np.max(np.abs(got["norm"] - ref["norm"].T))
    de = np.max(np.abs(got["energy"] - ref["energy"].T))
    assert dP <= TOL_FP32, f"max|dP| = {dP:.3e}"
    assert dn <= TOL_NORM_DRIFT, f"max|dnorm| = {dn:.3e}"
    assert de <= energy_tol(w), f"max|dE| = {de:.3e}"


@pytest.mark.parametrize("shape", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("N,periodic,K", [(40, False, 16), (100, True, 9), (130, False, 3),
                                          (256, False, 16), (17, True, 5)])
def test_tiled_bosons_against_oracle(ctqw, shape, N, periodic, K):
    w = cw.get("bosons_n256_u2").with_(N=N, R=2, periodic=periodic, K=K, n_steps=24, obs_every=8,
                                       sites=(N // 2 - 1, N // 2))
    got = ctqw.run_workload(w, flags=ctqw.FLAG_TILED(shape))
    ref = oracle.ensemble_run(w)
    _check(got, ref, w)
    P = per_realization_P(got["psi"], got["st_off"], got["sizes"], 2)
    for r in range(w.R):
        assert np.max(np.abs(P[r] - ref["P"][r][-1])) <= TOL_FP32


@pytest.mark.parametrize("shape", [0, 2, 3, 4])
def test_tiled_ragged_batch(ctqw, shape):
    w = cw.get("ragged_n128_1024").with_(R=5, ragged_sizes=(64, 130, 200), n_steps=16, obs_every=8)
    got = ctqw.run_workload(w, flags=ctqw.FLAG_TILED(shape))
    ref = oracle.ensemble_run(w)
    _check(got, ref, w)


def test_tiled_distinguishable_long_run(ctqw):
    w = cw.get("fp64_plain_small").with_(dtype=cw.C64, N=64, n_steps=300, obs_every=50)
    got = ctqw.run_workload(w, flags=ctqw.FLAG_TILED(0))
    ref = oracle.ensemble_run(w)
    _check(got, ref, w)


def test_tiled_agrees_with_fused_kernel_at_n256(ctqw):
    w = cw.get("bosons_n256_u2").with_(R=32, n_steps=200, obs_every=50)
    a = ctqw.run_workload(w, flags=ctqw.FLAG_TILED(0))
    b = ctqw.run_workload(w)
    assert np.max(np.abs(a["P_mean"] - b["P_mean"])) <= TOL_FP32
    assert np.max(np.abs(a["norm"] - 1.0)) <= TOL_NORM_DRIFT


def test_tiled_rejects_unknown_shape_and_short_workspace(ctqw):
    w = cw.get("bosons_small").with_(R=1, n_steps=2)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C64)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C64)
    with pytest.raises(ctqw.CtqwError, match="shape"):
        ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, 2, 0, None, None, None,
                                   ctqw.FUSED_SHAPE(7), None)
    with pytest.raises(ctqw.CtqwError, match="workspace"):
        ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, 2, 0, None, None, None,
                                   ctqw.FLAG_TILED(0), torch.empty(8, dtype=torch.uint8, device="cuda"))
    with pytest.raises(ctqw.CtqwError, match="tiled"):
        ctqw.ctqw_propagate_taylor(h, psi, cw.C128, w.dt, w.K, 2, 0, None, None, None,
                                   ctqw.FLAG_TILED(0), h.workspace(cw.C128, ctqw.TAYLOR, ctqw.FLAG_PLAIN))
    h.close()


@pytest.mark.parametrize("K", [1, 3, 5, 6, 7, 9, 12])
def test_tiled_default_depths(ctqw, K):
    """Every register depth the default path picks (ceil(K / ceil(K / 8)))."""
    w = cw.get("bosons_n256_u2").with_(N=300, R=2, K=K, dt=0.01, n_steps=10, obs_every=5,
                                       sites=(149, 150))
    got = ctqw.run_workload(w)
    ref = oracle.ensemble_run(w)
    _check(got, ref, w)
