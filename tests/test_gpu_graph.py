"""Parity of the graph path (Sec. 2: q-dimensional lattices and general
graphs) with the FP64 oracle, through the C ABI.

Small workloads: 2-D and 3-D lattices, open and periodic, m = 2 and 3, all
three statistics, and a ring with random chords (variable degree, repeated
links).  Each spans several 256-thread blocks with a ragged tail.  The full
15 x 15 workload runs at its bench size with sampled realizations checked
one by one.
"""
import numpy as np
import pytest

import ctqw_workloads as cw
import oracle
from gpu_helpers import TOL_FP32, TOL_FP64, TOL_NORM_DRIFT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = ["lattice2d_small", "lattice2d_open_small", "lattice3d_small", "lattice2d_m3_small", "graph_small"]


@pytest.fixture(scope="module")
def ctqw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_00746_gb300 import build, ctqw as c

    build.build()
    c.load()
    return c


def _run(ctqw, w, dtype, method="taylor", realizations=None, n_steps=None, obs_every=None, K=None,
         edges=None, chunk=0):
    dev = torch.device("cuda", 0)
    if edges is None:
        g = ctqw.Graph.from_workload(w, realizations)
    else:
        ue, uj = _custom_draws(w, len(edges[0]))
        g = ctqw.Graph(w.m, w.statistics, w.n_nodes(), edges[0], edges[1], ue.shape[0], w.J0, w.U,
                       w.eps_halfwidth, w.J_halfwidth, ue, uj)
    n_steps = w.n_steps if n_steps is None else n_steps
    obs_every = w.obs_every if obs_every is None else obs_every
    K = w.K if K is None else K
    if chunk:
        ctqw.ctqw_graph_set_chunk(g, chunk)
    psi = g.new_state(dtype, dev)
    ctqw.ctqw_graph_init_state(g, psi, w.sites, dtype)
    n_obs = g.n_obs(n_steps, obs_every)
    P = torch.empty((n_obs, g.N), dtype=torch.float64, device=dev)
    nr = torch.empty((n_obs, g.R), dtype=torch.float64, device=dev)
    en = torch.empty((n_obs, g.R), dtype=torch.float64, device=dev)
    if method == "taylor":
        ctqw.ctqw_graph_propagate_taylor(g, psi, dtype, w.dt, K, n_steps, obs_every, P, nr, en)
    else:
        ctqw.ctqw_graph_propagate_rk4(g, psi, dtype, w.dt, n_steps, obs_every, P, nr, en)
    torch.cuda.synchronize()
    out = {"P": P.cpu().numpy(), "norm": nr.cpu().numpy(), "energy": en.cpu().numpy(),
           "psi": g.states(psi).cpu().numpy().astype(np.complex128)}
    g.close()
    return out


def _check(got, ref, dtype):
    tolP = TOL_FP64 if dtype == cw.C128 else TOL_FP32
    tol_n = 1e-12 if dtype == cw.C128 else TOL_NORM_DRIFT
    tol_e = 1e-10 if dtype == cw.C128 else 2e-5
    tol_psi = 1e-10 if dtype == cw.C128 else 2e-5
    dP = np.max(np.abs(got["P"] - ref["P"]), initial=0.0)
    assert dP <= tolP, f"max|dP| = {dP:.3e}"
    assert np.max(np.abs(got["norm"] - ref["norm"]), initial=0.0) <= tol_n
    assert np.max(np.abs(got["energy"] - ref["energy"]), initial=0.0) <= tol_e
    dpsi = max(np.max(np.abs(a - b)) for a, b in zip(got["psi"], ref["psi"]))
    assert dpsi <= tol_psi, f"max|dpsi| = {dpsi:.3e}"


@pytest.mark.parametrize("name", SMALL)
def test_graph_params_bit_exact(ctqw, name):
    w = cw.get_graph(name)
    g = ctqw.Graph.from_workload(w)
    eps, J = g.params()
    ue, uj = cw.graph_draws(w)
    for r in range(w.R):
        e_ref, j_ref = oracle.graph_parameters(ue[r], uj[r], w.eps_halfwidth, w.J0, w.J_halfwidth)
        assert np.array_equal(eps[r], e_ref), r
        assert np.array_equal(J[r], j_ref), r
    g.close()


@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("dtype", [cw.C128, cw.C64])
def test_graph_taylor_matches_oracle(ctqw, name, dtype):
    w = cw.get_graph(name)
    got = _run(ctqw, w, dtype)
    ref = oracle.graph_ensemble_run(w)
    _check(got, ref, dtype)


@pytest.mark.parametrize("chunk", [1, 3, 32])
@pytest.mark.parametrize("dtype", [cw.C128, cw.C64])
def test_graph_chunks_give_the_same_result(ctqw, chunk, dtype):
    # passes over 1, 3 or 32 realizations at a time (7 realizations: a ragged
    # last pass) against the oracle, for Taylor and RK4
    w = cw.get_graph("lattice2d_small").with_(R=7, n_steps=30)
    for method in ("taylor", "rk4"):
        got = _run(ctqw, w, dtype, method=method, chunk=chunk)
        ref = oracle.graph_ensemble_run(w, method=method)
        _check(got, ref, dtype)


@pytest.mark.parametrize("dtype", [cw.C128, cw.C64])
def test_graph_rk4_matches_oracle(ctqw, dtype):
    w = cw.get_graph("lattice2d_small").with_(n_steps=60)
    got = _run(ctqw, w, dtype, method="rk4")
    ref = oracle.graph_ensemble_run(w, method="rk4")
    _check(got, ref, dtype)


@pytest.mark.parametrize("K,n_steps,obs_every", [(1, 7, 1), (2, 5, 5), (30, 3, 1), (16, 0, 1), (16, 9, 0)])
def test_graph_orders_and_sampling(ctqw, K, n_steps, obs_every):
    w = cw.get_graph("graph_small").with_(R=2, dt=0.01)
    got = _run(ctqw, w, cw.C128, K=K, n_steps=n_steps, obs_every=obs_every)
    ref = oracle.graph_ensemble_run(w, K=K, n_steps=n_steps, obs_every=obs_every)
    if obs_every == 0:
        ref["P"] = np.zeros((0, w.n_nodes()))
        ref["norm"] = ref["energy"] = np.zeros((0, 2))
    _check(got, ref, cw.C128)


@pytest.mark.parametrize("dtype", [cw.C128, cw.C64])
def test_graph_without_links_and_with_isolated_node_and_repeated_link(ctqw, dtype):
    # no links at all: H is diagonal
    w = cw.get_graph("graph_small").with_(ring_nodes=6, chords=0, R=3, sites=(1, 4), n_steps=40)
    none = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    got = _run(ctqw, w, dtype, edges=none)
    ref = _oracle_custom(w, none)
    _check(got, ref, dtype)
    # node 5 isolated, link (0, 1) twice (entries add), a node of degree 3
    links = (np.array([0, 0, 1, 2, 3, 1], np.int32), np.array([1, 1, 2, 3, 4, 3], np.int32))
    w2 = w.with_(statistics=cw.BOSONS, sites=(1, 1))
    got = _run(ctqw, w2, dtype, edges=links)
    ref = _oracle_custom(w2, links)
    _check(got, ref, dtype)


def _custom_draws(w, E):
    """Draws for a custom link list: the workload's streams, E from the list."""
    n = w.n_nodes()
    ue = np.zeros((w.R, n))
    uj = np.zeros((w.R, E))
    for r in range(w.R):
        gen = np.random.Generator(np.random.Philox(np.random.SeedSequence([int(w.seed), int(r), 0x62])))
        ue[r] = gen.random(n)
        uj[r] = gen.random(E)
    return ue, uj


def _oracle_custom(w, edges):
    n = w.n_nodes()
    ue, uj = _custom_draws(w, len(edges[0]))
    P, norms, energies, finals = None, [], [], []
    for r in range(w.R):
        eps, J = oracle.graph_parameters(ue[r], uj[r], w.eps_halfwidth, w.J0, w.J_halfwidth)
        H = oracle.many_particle_hamiltonian(
            oracle.graph_single_particle_hamiltonian(n, edges[0], edges[1], eps, J), w.m, w.U)
        out = oracle.propagate(H, oracle.initial_state(n, w.m, w.sites, w.statistics), n, w.m, w.dt,
                               w.n_steps, w.obs_every, "taylor", w.K)
        P = out["P"] if P is None else P + out["P"]
        norms.append(out["norm"])
        energies.append(out["energy"])
        finals.append(out["psi"])
    return {"P": P / w.R, "norm": np.array(norms).T, "energy": np.array(energies).T, "psi": finals}


@pytest.mark.parametrize("stats,sites", [(0, (3, 3)), (1, (3, 3)), (1, (2, 7)), (2, (2, 7))])
def test_graph_initial_states(ctqw, stats, sites):
    w = cw.get_graph("lattice2d_small").with_(statistics=stats, sites=sites, R=2)
    g = ctqw.Graph.from_workload(w)
    psi = g.new_state(cw.C128, torch.device("cuda", 0))
    ctqw.ctqw_graph_init_state(g, psi, sites, cw.C128)
    got = g.states(psi).cpu().numpy()
    ref = oracle.initial_state(w.n_nodes(), 2, sites, stats)
    assert np.array_equal(got[0], ref) and np.array_equal(got[1], ref)
    g.close()


def test_graph_fermions_on_one_node_rejected(ctqw):
    w = cw.get_graph("lattice2d_small").with_(statistics=cw.FERMIONS, R=1)
    g = ctqw.Graph.from_workload(w)
    psi = g.new_state(cw.C64, torch.device("cuda", 0))
    with pytest.raises(ctqw.CtqwError):
        ctqw.ctqw_graph_init_state(g, psi, (4, 4), cw.C64)
    g.close()


def test_graph_full_size_sampled_realizations(ctqw):
    # the 15 x 15 workload at its full ensemble (1000 realizations, FP32, the
    # launch configuration of the bench), 200 steps; realizations 0, 517 and
    # 999 checked one by one against the oracle
    w = cw.get_graph("lattice2d_15x15_m2").with_(n_steps=200, obs_every=50)
    got = _run(ctqw, w, cw.C64)
    picks = [0, 517, 999]
    ref = oracle.graph_ensemble_run(w, realizations=picks)
    assert np.max(np.abs(got["norm"][:, picks] - ref["norm"])) <= TOL_NORM_DRIFT
    assert np.max(np.abs(got["energy"][:, picks] - ref["energy"])) <= 2e-5
    for k, r in enumerate(picks):
        assert np.max(np.abs(got["psi"][r] - ref["psi"][k])) <= 2e-5, r
    # the ensemble mean of P sums to the mean norm at every sample
    np.testing.assert_allclose(got["P"].sum(axis=1), got["norm"].mean(axis=1), atol=1e-9)
