"""Exact propagation by diagonalisation on the device (Algorithm 1; batched
cyclic Jacobi in FP64) against the oracle's dense eigendecomposition and
against the FP64 Taylor path: two and three particles, open chains and
rings, odd and even state dimensions."""
import numpy as np
import pytest

import ctqw_workloads as cw
import oracle
from gpu_helpers import TOL_FP64, oracle_params

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


def _workload(m, N, periodic, stats, U=2.0):
    sites = (N // 2 - 1, N // 2) if m == 2 else (0, 1, 2)
    return cw.Workload(name="exact", m=m, statistics=stats, periodic=periodic, N=N, R=4, J0=1.0, U=U,
                       eps_halfwidth=1.0, J_halfwidth=0.25, sites=sites, dt=0.05, K=16,
                       n_steps=40, obs_every=10, dtype=cw.C128, seed=21)


@pytest.mark.parametrize("m,N,periodic,stats", [(2, 8, False, 1), (2, 5, True, 0), (2, 6, False, 2),
                                                (3, 4, True, 1), (3, 3, False, 0)])
def test_exact_against_oracle_eigendecomposition(ctqw, m, N, periodic, stats):
    w = _workload(m, N, periodic, stats)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C128)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C128)
    n_obs = h.n_obs(w.n_steps, w.obs_every)
    P = torch.empty((n_obs, h.p_width), dtype=torch.float64, device="cuda")
    nr = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    en = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    sweeps = ctqw.ctqw_propagate_exact(h, psi, w.dt, w.n_steps, w.obs_every, P, nr, en)
    assert np.all(sweeps < 40)
    got = psi.cpu().numpy()
    times = [w.dt * k for k in range(0, w.n_steps + 1, w.obs_every)]
    P_ref = np.zeros((n_obs, N))
    for r, (eps, J) in enumerate(oracle_params(w)):
        nb = N if periodic else N - 1
        H = oracle.many_particle_hamiltonian(oracle.single_particle_hamiltonian(eps, J[:nb], periodic), m, w.U)
        psi0 = oracle.initial_state(N, m, w.sites, stats)
        ref = oracle.exact_evolution(H, psi0, times)
        assert np.max(np.abs(got[h.st_off[r]:h.st_off[r + 1]] - ref[-1])) <= TOL_FP64
        for k in range(n_obs):
            P_ref[k] += oracle.site_occupation(ref[k], N, m) / w.R
    assert np.max(np.abs(P.cpu().numpy() - P_ref)) <= TOL_FP64
    assert np.max(np.abs(nr.cpu().numpy() - 1.0)) <= 1e-12
    h.close()


def test_exact_agrees_with_fp64_taylor_path(ctqw):
    w = _workload(2, 8, False, 1).with_(K=20, n_steps=60, obs_every=20)
    a = ctqw.run_workload(w, dtype=cw.C128, flags=ctqw.FLAG_PLAIN)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C128)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C128)
    P = torch.empty((h.n_obs(w.n_steps, w.obs_every), h.p_width), dtype=torch.float64, device="cuda")
    ctqw.ctqw_propagate_exact(h, psi, w.dt, w.n_steps, w.obs_every, P)
    assert np.max(np.abs(P.cpu().numpy() - a["P_mean"])) <= TOL_FP64
    assert np.max(np.abs(psi.cpu().numpy() - a["psi"])) <= TOL_FP64
    h.close()


def test_exact_refuses_fp32_and_large_states(ctqw):
    for kw, dtype in (({"N": 8}, cw.C64), ({"N": 9}, cw.C128)):
        w = _workload(2, 8, False, 0).with_(**kw)
        h = ctqw.build_for_workload(w)
        psi = h.new_state(cw.C128)
        lib = ctqw.load()
        import ctypes

        st = lib.ctqw_propagate_exact(h.handle, dtype, ctypes.c_void_p(psi.data_ptr()), w.dt, 2, 0, None,
                                      None, None, None, None)
        assert st == ctqw.CTQW_EUNSUPPORTED
        h.close()
