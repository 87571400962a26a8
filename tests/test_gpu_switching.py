"""Switching noise (the Hamiltonian update after every step) through the C
ABI against the oracle's piecewise-constant propagation with the same
Philox4x64-10 draws: the register tiles (two particles, FP32), the per-term
paths (FP64, three particles), a ragged batch; parameters after the run
bit for bit; p = 0 equal to the static propagation."""
import numpy as np
import pytest

import ctqw_workloads as cw
import oracle
from gpu_helpers import TOL_FP32, TOL_FP64, TOL_NORM_DRIFT, energy_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 0x5EED


@pytest.fixture(scope="module")
def ctqw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_00746_gb300 import build, ctqw as c

    build.build()
    c.load()
    return c


def _run(ctqw, w, dtype, p, flags=0, seed=SEED):
    h = ctqw.build_for_workload(w)
    psi = h.new_state(dtype)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), dtype)
    n_obs = h.n_obs(w.n_steps, w.obs_every)
    P = torch.empty((n_obs, h.p_width), dtype=torch.float64, device="cuda")
    nr = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    en = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    ctqw.ctqw_propagate_taylor_switching(h, psi, dtype, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en,
                                         seed, p, flags)
    ctqw.ctqw_check_status(h)
    eps, J = h.params()
    out = {"P": P.cpu().numpy(), "norm": nr.cpu().numpy(), "energy": en.cpu().numpy(),
           "eps": eps, "J": J, "sizes": h.sizes.copy()}
    h.close()
    return out


def _oracle(w, p, seed=SEED):
    per = [oracle.propagate_switching(w, r, seed, p) for r in range(w.R)]
    sizes = w.sizes()
    groups = sorted(set(int(n) for n in sizes))
    P = []
    for g in groups:
        members = [r for r in range(w.R) if sizes[r] == g]
        P.append(sum(per[r]["P"] for r in members) / len(members))
    return per, np.concatenate(P, axis=1)


@pytest.mark.parametrize("name,kw,dtype,tol,flags", [
    ("bosons_small", {"R": 3, "n_steps": 40, "obs_every": 10}, cw.C64, TOL_FP32, 0),
    ("bosons_small", {"R": 2, "n_steps": 30, "obs_every": 10}, cw.C64, TOL_FP32, 1),
    ("fp64_plain_small", {"R": 2, "n_steps": 30, "obs_every": 10}, cw.C128, TOL_FP64, 0),
    ("ring3_small", {"R": 2, "n_steps": 20, "obs_every": 10}, cw.C64, TOL_FP32, 0),
    ("ragged_n128_1024", {"R": 5, "ragged_sizes": (30, 52, 77), "n_steps": 25, "obs_every": 5},
     cw.C64, TOL_FP32, 0),
])
def test_switching_against_oracle(ctqw, name, kw, dtype, tol, flags):
    w = cw.get(name).with_(**kw)
    got = _run(ctqw, w, dtype, 0.15, flags)
    per, P_ref = _oracle(w, 0.15)
    assert np.max(np.abs(got["P"] - P_ref)) <= tol
    norm_ref = np.array([r["norm"] for r in per]).T
    assert np.max(np.abs(got["norm"] - norm_ref)) <= (TOL_NORM_DRIFT if dtype == cw.C64 else 1e-12)
    energy_ref = np.array([r["energy"] for r in per]).T
    assert np.max(np.abs(got["energy"] - energy_ref)) <= (energy_tol(w) if dtype == cw.C64 else 1e-10)
    # the parameters after the last update, bit for bit
    off = 0
    for r in range(w.R):
        N = int(got["sizes"][r])
        assert np.array_equal(got["eps"][off:off + N], per[r]["eps"])
        nb = len(per[r]["J"])
        assert np.array_equal(got["J"][off:off + nb], per[r]["J"])
        off += N


def test_zero_probability_equals_static_and_runs_repeat(ctqw):
    w = cw.get("bosons_small").with_(N=100, R=2, sites=(49, 50), n_steps=20, obs_every=10)
    a = _run(ctqw, w, cw.C64, 0.0)
    b = ctqw.run_workload(w)   # static, same default path (register tiles for N = 100)
    assert np.max(np.abs(a["P"] - b["P_mean"])) <= 1e-12
    c1 = _run(ctqw, w, cw.C64, 0.3)
    c2 = _run(ctqw, w, cw.C64, 0.3)
    assert np.array_equal(c1["P"], c2["P"]) or np.max(np.abs(c1["P"] - c2["P"])) <= 1e-14
    assert np.max(np.abs(c1["P"] - a["P"])) > 1e-6


def test_switching_rejects_bad_probability(ctqw):
    w = cw.get("bosons_small").with_(R=1, n_steps=2, obs_every=1)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C64)
    with pytest.raises(ctqw.CtqwError, match="p_switch"):
        ctqw.ctqw_propagate_taylor_switching(h, psi, cw.C64, w.dt, w.K, 2, 0, None, None, None, 1, 1.5)
    h.close()
