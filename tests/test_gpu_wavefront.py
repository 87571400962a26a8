"""Parity of the row-wavefront kernel (one warp per Taylor term, rows streamed
through a pipeline) with the FP64 oracle, through the C ABI.

Cases span one and several launches (observation points split the run),
steps pipelined back to back inside a launch, the lowest orders K = 1, 2,
every compiled row width, a ragged batch of those widths, bosons with U on
the diagonal, distinguishable walkers, and the requests the kernel refuses.
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


@pytest.mark.parametrize("N,K,n_steps,obs_every", [
    (64, 16, 40, 10),     # several launches
    (64, 12, 37, 0),      # one launch, no samples but the final state
    (128, 16, 30, 7),     # a ragged last segment
    (192, 13, 24, 8),
    (256, 16, 24, 24),
])
def test_wavefront_bosons_against_oracle(ctqw, N, K, n_steps, obs_every):
    w = cw.get("bosons_n256_u2").with_(N=N, R=3, K=K, n_steps=n_steps, obs_every=obs_every,
                                       sites=(N // 2 - 1, N // 2))
    got = ctqw.run_workload(w, flags=ctqw.FLAG_WAVEFRONT)
    ref = oracle.ensemble_run(w.with_(obs_every=obs_every if obs_every else n_steps))
    if obs_every:
        _check(got, ref, w)
    if n_steps % (obs_every or n_steps) == 0:
        # the oracle's last sample is the final state
        P = per_realization_P(got["psi"], got["st_off"], got["sizes"], 2)
        for r in range(w.R):
            assert np.max(np.abs(P[r] - ref["P"][r][-1])) <= TOL_FP32


@pytest.mark.parametrize("K", [1, 2, 5])
def test_wavefront_low_orders(ctqw, K):
    # small dt so that low orders stay accurate; the oracle uses the same K
    w = cw.get("bosons_small").with_(N=64, R=2, K=K, dt=0.002, n_steps=60, obs_every=20,
                                     sites=(31, 32))
    got = ctqw.run_workload(w, flags=ctqw.FLAG_WAVEFRONT)
    ref = oracle.ensemble_run(w)
    dP = np.max(np.abs(got["P_mean"] - ref["P_mean"]))
    assert dP <= TOL_FP32, dP


def test_wavefront_distinguishable(ctqw):
    w = cw.get("fp64_plain_small").with_(dtype=cw.C64, N=64, n_steps=200, obs_every=25)
    got = ctqw.run_workload(w, flags=ctqw.FLAG_WAVEFRONT)
    ref = oracle.ensemble_run(w)
    _check(got, ref, w)


def test_wavefront_ragged_widths(ctqw):
    w = cw.get("ragged_n128_1024").with_(R=10, ragged_sizes=(64, 128, 192, 256), K=8,
                                         n_steps=20, obs_every=10)
    got = ctqw.run_workload(w, flags=ctqw.FLAG_WAVEFRONT)
    ref = oracle.ensemble_run(w)
    _check(got, ref, w)
    P = per_realization_P(got["psi"], got["st_off"], got["sizes"], 2)
    for r in range(w.R):
        assert np.max(np.abs(P[r] - ref["P"][r][-1])) <= TOL_FP32


def test_wavefront_agrees_with_full_row_kernel(ctqw):
    """Same inputs through both fused kernels at N = 256 (64 realizations, 300 steps)."""
    w = cw.get("bosons_n256_u2").with_(R=64, n_steps=300, obs_every=50)
    a = ctqw.run_workload(w, flags=ctqw.FLAG_WAVEFRONT)
    b = ctqw.run_workload(w)
    assert np.max(np.abs(a["P_mean"] - b["P_mean"])) <= TOL_FP32
    assert np.max(np.abs(a["norm"] - 1.0)) <= TOL_NORM_DRIFT
    assert np.max(np.abs(a["energy"] - a["energy"][0])) <= energy_tol(w)


@pytest.mark.parametrize("kw", [{"periodic": True}, {"N": 96}, {"K": 17}])
def test_wavefront_refuses_unsupported(ctqw, kw):
    w = cw.get("bosons_n256_u2").with_(R=1, n_steps=2, obs_every=1, sites=(10, 11), **kw)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C64)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C64)
    lib = ctqw.load()
    with pytest.raises(RuntimeError, match="wavefront"):
        ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, 2, 0, None, None, None,
                                   ctqw.FLAG_WAVEFRONT, None)
    h.close()


def test_wavefront_rejects_short_workspace(ctqw):
    w = cw.get("bosons_small").with_(N=64, R=2, n_steps=2, obs_every=1)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C64)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C64)
    short = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError, match="workspace"):
        ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, 2, 0, None, None, None,
                                   ctqw.FLAG_WAVEFRONT, short)
    h.close()
