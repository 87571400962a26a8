"""CTQW_FLAG_RENORMALIZE against the oracle's renormalized propagation.

The norm check of Algorithms 2 and 3 with its corrective action: after
every step each state is divided by its norm.  A coarse dt makes RK4 lose
norm visibly, so the correction is exercised.
"""
import numpy as np
import pytest

import ctqw_workloads as cw
import oracle
from gpu_helpers import TOL_FP32, TOL_FP64, energy_tol

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


def _compare(got, ref, dtype, w):
    tolP = TOL_FP64 if dtype == cw.C128 else TOL_FP32
    tol_n = 1e-13 if dtype == cw.C128 else 1e-6
    tol_e = 1e-10 if dtype == cw.C128 else energy_tol(w)
    assert np.max(np.abs(got["P_mean"] - ref["P_mean"])) <= tolP
    assert np.max(np.abs(got["norm"] - 1.0)) <= tol_n
    assert np.max(np.abs(got["norm"] - ref["norm"].T)) <= tol_n
    assert np.max(np.abs(got["energy"] - ref["energy"].T)) <= tol_e


@pytest.mark.parametrize("name", ["bosons_small", "ring3_small"])
@pytest.mark.parametrize("dtype", [cw.C128, cw.C64])
@pytest.mark.parametrize("method", ["rk4", "taylor"])
def test_renormalized_runs_match_the_oracle(ctqw, name, dtype, method):
    w = cw.get(name).with_(R=3, dt=0.05, n_steps=60, obs_every=20, dtype=dtype)
    m = ctqw.RK4 if method == "rk4" else ctqw.TAYLOR
    got = ctqw.run_workload(w, method=m, K=4, flags=ctqw.FLAG_RENORMALIZE)
    ref = oracle.ensemble_run(w, method=method, K=4, renormalize=True)
    _compare(got, ref, dtype, w)


def test_rk4_without_the_flag_drifts(ctqw):
    # the same coarse RK4 run without renormalization loses norm (what the
    # flag corrects), and matches the unrenormalized oracle
    w = cw.get("bosons_small").with_(R=2, dt=0.05, n_steps=60, obs_every=20, dtype=cw.C128)
    got = ctqw.run_workload(w, method=ctqw.RK4, flags=ctqw.FLAG_PLAIN)
    ref = oracle.ensemble_run(w, method="rk4")
    assert np.max(np.abs(got["norm"][-1] - 1.0)) > 1e-6
    assert np.max(np.abs(got["norm"] - ref["norm"].T)) <= 1e-12
