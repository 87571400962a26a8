"""Full-size runs in the launch configuration bench.py times, checked against
oracle values computed one realization at a time (sampled outputs) and against
properties that hold at any size."""
import json
import os

import numpy as np
import pytest

import ctqw_workloads as cw
import oracle
from gpu_helpers import TOL_FP32, TOL_FP64, TOL_NORM_DRIFT, energy_tol, oracle_params, per_realization_P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctqw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_00746_gb300 import build, ctqw as c

    build.build()
    c.load()
    return c


def test_fp64_plain_n64_full_against_exact_product_solution(ctqw):
    """2 distinguishable walkers, U = 0: every sample of every realization against
    exp(-iH1 t) (x) exp(-iH1 t) (exact up to the order-12 truncation, ~1e-27/step)."""
    w = cw.get("fp64_plain_n64")
    got = ctqw.run_workload(w)
    params = oracle_params(w)
    times = [w.dt * s for s in range(0, w.n_steps + 1, w.obs_every)]
    P_ref = np.zeros_like(got["P_mean"])
    for eps, Jp in params:
        J = Jp[:w.N - 1]
        psi0 = oracle.initial_state(w.N, 2, w.sites, w.statistics)
        states = oracle.noninteracting_evolution(eps, J, False, 2, psi0, times)
        P_ref += np.array([oracle.site_occupation(s, w.N, 2) for s in states]) / w.R
    assert np.max(np.abs(got["P_mean"] - P_ref)) <= TOL_FP64
    assert np.max(np.abs(got["norm"] - 1.0)) <= 1e-12


def test_bosons_n256_full_size(ctqw):
    """Headline workload at full size (1024 realizations, 2500 steps, fused c64;
    the last realizations on the second stream's register tiles)."""
    golds = []
    for name in ("bosons_n256_u2_r0-3.json", "bosons_n256_u2_r1020-1023.json"):
        path = os.path.join(GOLDEN, name)
        if not os.path.exists(path):
            pytest.skip("golden fixture missing (tests/golden/make_golden.py)")
        golds.append(json.load(open(path)))
    w = cw.get("bosons_n256_u2")
    h = ctqw.build_for_workload(w)
    assert ctqw.ctqw_fused_split(h, w.K) >= 4   # realizations 1020..1023 run on the tiles
    h.close()
    got = ctqw.run_workload(w)
    # every realization conserves the norm to the FP32 bar
    assert np.max(np.abs(got["norm"] - 1.0)) <= TOL_NORM_DRIFT
    # energy conserved per realization
    assert np.max(np.abs(got["energy"] - got["energy"][0])) <= energy_tol(w)
    # the ensemble mean sums to the mean norm at every sample
    np.testing.assert_allclose(got["P_mean"].sum(axis=1), got["norm"].mean(axis=1), atol=1e-6)
    # sampled outputs: realizations 0..3 and 1020..1023 against the oracle
    P_final = per_realization_P(got["psi"], got["st_off"], got["sizes"], 2)
    for gold in golds:
        steps = gold["steps"]
        for r, g in gold["realizations"].items():
            r = int(r)
            assert np.max(np.abs(P_final[r] - np.array(g["P"][-1]))) <= TOL_FP32
            for k, s in enumerate(steps):
                assert abs(got["norm"][s // w.obs_every, r] - g["norm"][k]) <= TOL_NORM_DRIFT
                assert abs(got["energy"][s // w.obs_every, r] - g["energy"][k]) <= energy_tol(w)
