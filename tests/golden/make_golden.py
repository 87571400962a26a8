"""Write the stored expected values used by the full-size GPU parity tests.

Every value here comes from the FP64 CPU oracle (``oracle/``) and nothing
else.  The paper prints no worked example to pin against, so these fixtures
only let the GPU tests check full-size runs without re-running the slow
oracle on the GPU machine.

  python tests/golden/make_golden.py            # all fixtures
  python tests/golden/make_golden.py bosons     # one of them

bosons_n256_u2_r0-3.json: realizations 0..3 of the 2-boson N=256 workload,
full 2500 steps (t = 50), K = 16: per-realization P_r(x) at steps 500, 1250,
2500 and the norm and energy at those steps.
bosons_n256_u2_r1020-1023.json: the same for the last four realizations
(the ones the fused path runs on its second stream).
"""
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def _bosons_realization(r):
    import numpy as np

    import ctqw_workloads as cw
    import oracle

    w = cw.get("bosons_n256_u2")
    N = w.N
    ue, uj = cw.uniform_draws(w.seed, [r], [N])
    eps, J = oracle.workload_parameters(w, ue[0], uj[0], N)
    H = oracle.many_particle_hamiltonian(oracle.single_particle_hamiltonian(eps, J, w.periodic), w.m, w.U)
    psi = oracle.initial_state(N, w.m, w.initial_sites(N), w.statistics)
    marks = (500, 1250, 2500)
    out = {"P": [], "norm": [], "energy": []}
    for n in range(1, w.n_steps + 1):
        psi = oracle.taylor_step(H, psi, w.dt, w.K)
        if n in marks:
            out["P"].append(oracle.site_occupation(psi, N, w.m).tolist())
            out["norm"].append(oracle.norm(psi))
            out["energy"].append(oracle.energy(H, psi))
    out["energy0"] = oracle.energy(H, oracle.initial_state(N, w.m, w.initial_sites(N), w.statistics))
    return r, out


def make_bosons(first=0):
    reals = list(range(first, first + 4))
    ctx = mp.get_context("spawn")
    with ctx.Pool(4) as pool:
        res = dict(pool.map(_bosons_realization, reals))
    doc = {
        "what": f"oracle FP64 Taylor (K=16) on realizations {reals[0]}..{reals[-1]} of bosons_n256_u2",
        "writer": "tests/golden/make_golden.py (oracle only)",
        "steps": [500, 1250, 2500],
        "realizations": {str(r): res[r] for r in reals},
    }
    with open(os.path.join(HERE, f"bosons_n256_u2_r{reals[0]}-{reals[-1]}.json"), "w") as f:
        json.dump(doc, f)


if __name__ == "__main__":
    which = sys.argv[1:] or ["bosons", "bosons_last"]
    if "bosons" in which:
        make_bosons(0)
    if "bosons_last" in which:
        make_bosons(1020)
