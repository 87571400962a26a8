"""Pins of the oracle's q-dimensional lattices and general graphs (Sec. 2).

Each test checks the graph part of the oracle against something that does not
come from it: the chain Hamiltonian (pinned on its own elsewhere), closed-form
spectra of tori and open grids, the filling factor (mk + 1) / N^m that Sec. 2
states for a regular lattice, the Kronecker factorisation of a separable
lattice propagated with scipy's matrix exponential, and conservation laws.
"""
import numpy as np
import pytest
import scipy.linalg

import ctqw_workloads as cw
import oracle as O


def _graph_h1(shape, periodic, eps, J):
    u, v = cw.lattice_edges(shape, periodic)
    return O.graph_single_particle_hamiltonian(int(np.prod(shape)), u, v, eps, J)


@pytest.mark.parametrize("N", [2, 3, 7])
@pytest.mark.parametrize("periodic", [False, True])
def test_graph_of_a_chain_is_the_chain(N, periodic):
    rng = np.random.default_rng(N + 10 * periodic)
    nb = N if periodic else N - 1
    eps, J = rng.uniform(-1, 1, N), 1.0 + rng.uniform(-0.25, 0.25, nb)
    u, v = cw.lattice_edges((N,), periodic)
    assert len(u) == nb
    H_graph = O.graph_single_particle_hamiltonian(N, u, v, eps, J)
    np.testing.assert_array_equal(H_graph, O.single_particle_hamiltonian(eps, J, periodic))


def _spectrum_many(H1_eigs, m):
    tot = np.zeros(1)
    for _ in range(m):
        tot = (tot[:, None] + H1_eigs[None, :]).reshape(-1)
    return np.sort(tot)


def test_torus_spectrum_closed_form():
    # 3 x 4 torus, uniform hopping J: one-particle energies
    # -2J (cos(2 pi a / 3) + cos(2 pi b / 4)); two free particles add them
    J = 0.7
    shape = (3, 4)
    n_links = len(cw.lattice_edges(shape, True)[0])
    H1 = _graph_h1(shape, True, np.zeros(12), np.full(n_links, J))
    lam = np.array([-2 * J * (np.cos(2 * np.pi * a / 3) + np.cos(2 * np.pi * b / 4))
                    for a in range(3) for b in range(4)])
    H = O.many_particle_hamiltonian(H1, 2, 0.0).toarray()
    np.testing.assert_allclose(np.linalg.eigvalsh(H), _spectrum_many(lam, 2), atol=1e-12)


def test_open_grid_spectrum_closed_form():
    # open 3 x 5 grid: -2J (cos(pi a / 4) + cos(pi b / 6)), a = 1..3, b = 1..5
    J = 1.3
    shape = (3, 5)
    n_links = len(cw.lattice_edges(shape, False)[0])
    assert n_links == 2 * 5 + 3 * 4
    H1 = _graph_h1(shape, False, np.zeros(15), np.full(n_links, J))
    lam = np.sort([-2 * J * (np.cos(np.pi * a / 4) + np.cos(np.pi * b / 6))
                   for a in range(1, 4) for b in range(1, 6)])
    np.testing.assert_allclose(np.linalg.eigvalsh(H1), lam, atol=1e-12)


def test_three_dim_lattice_with_extent_two_adds_both_links():
    # a periodic direction of extent 2 carries two links between the same
    # nodes; their entries add, -2J (cos(pi a) + ...) for that direction
    J = 0.9
    shape = (2, 3, 3)
    n_links = len(cw.lattice_edges(shape, True)[0])
    assert n_links == 3 * 18
    H1 = _graph_h1(shape, True, np.zeros(18), np.full(n_links, J))
    lam = np.sort([-2 * J * (np.cos(np.pi * a) + np.cos(2 * np.pi * b / 3) + np.cos(2 * np.pi * c / 3))
                   for a in range(2) for b in range(3) for c in range(3)])
    np.testing.assert_allclose(np.linalg.eigvalsh(H1), lam, atol=1e-12)


@pytest.mark.parametrize("m", [2, 3])
def test_filling_factor_of_a_regular_lattice(m):
    # Sec. 2: at most m k + 1 non-null entries per row, k = sum_i 2 k_i = 2q
    # for nearest neighbours; with noisy energies every row reaches it
    shape = (4, 5) if m == 2 else (3, 4)
    rng = np.random.default_rng(m)
    n = int(np.prod(shape))
    n_links = len(cw.lattice_edges(shape, True)[0])
    H1 = _graph_h1(shape, True, rng.uniform(0.1, 1.0, n), 1.0 + rng.uniform(-0.2, 0.2, n_links))
    H = O.many_particle_hamiltonian(H1, m, 1.5).tocsr()
    H.eliminate_zeros()
    nnz_per_row = np.diff(H.indptr)
    assert np.all(nnz_per_row == m * 4 + 1)


def test_separable_lattice_factorises_into_chains():
    # eps(i, j) = ex_i + ey_j, hopping along direction 0 depending on i only,
    # along direction 1 on j only: H1 = hx (x) I + I (x) hy with chain
    # matrices hx, hy, so exp(-i H t) = exp(-i hx t) (x) exp(-i hy t) per
    # particle; two distinguishable free particles propagate as a product
    rng = np.random.default_rng(5)
    n0, n1 = 4, 3
    ex, ey = rng.uniform(-1, 1, n0), rng.uniform(-1, 1, n1)
    Jx, Jy = 1 + rng.uniform(-0.3, 0.3, n0 - 1), 1 + rng.uniform(-0.3, 0.3, n1 - 1)
    u, v = cw.lattice_edges((n0, n1), False)
    J = np.empty(len(u))
    for e in range(len(u)):
        i0, j0 = divmod(int(u[e]), n1)
        i1, j1 = divmod(int(v[e]), n1)
        J[e] = Jx[i0] if i1 != i0 else Jy[j0]
    eps = (ex[:, None] + ey[None, :]).reshape(-1)
    H1 = O.graph_single_particle_hamiltonian(n0 * n1, u, v, eps, J)
    hx = O.single_particle_hamiltonian(ex, Jx, False)
    hy = O.single_particle_hamiltonian(ey, Jy, False)
    np.testing.assert_allclose(H1, np.kron(hx, np.eye(n1)) + np.kron(np.eye(n0), hy), atol=1e-15)

    n = n0 * n1
    H = O.many_particle_hamiltonian(H1, 2, 0.0)
    psi0 = O.initial_state(n, 2, (1, 10), 0)
    dt, steps = 0.05, 40
    out = O.propagate(H, psi0, n, 2, dt, steps, 0, "taylor", 16)
    t = dt * steps
    G = np.kron(scipy.linalg.expm(-1j * hx * t), scipy.linalg.expm(-1j * hy * t))
    expect = np.kron(G[:, 1], G[:, 10])
    np.testing.assert_allclose(out["psi"], expect, atol=1e-11)


def test_graph_parameters_law():
    # eps = w (2u - 1), J = J0 + w_J (2u - 1), rounded to float32
    u = np.array([0.0, 0.5, 0.75])
    eps, J = O.graph_parameters(u, u, 1.0, 1.0, 0.25)
    np.testing.assert_array_equal(eps, [-1.0, 0.0, 0.5])
    np.testing.assert_array_equal(J, [0.75, 1.0, 1.125])
    eps, _ = O.graph_parameters(np.array([0.1]), np.array([0.1]), 1.0, 1.0, 0.25)
    assert eps[0] == float(np.float32(-0.8))


def test_self_loop_rejected():
    with pytest.raises(ValueError):
        O.graph_single_particle_hamiltonian(3, np.array([0, 1]), np.array([1, 1]), np.zeros(3), np.ones(2))


@pytest.mark.parametrize("name", ["graph_small", "lattice2d_open_small"])
def test_graph_ensemble_conserves_norm_energy_and_symmetry(name):
    w = cw.get_graph(name).with_(R=2, n_steps=60)
    out = O.graph_ensemble_run(w)
    np.testing.assert_allclose(out["norm"], 1.0, atol=1e-12)
    np.testing.assert_allclose(out["energy"], np.broadcast_to(out["energy"][0], out["energy"].shape), atol=1e-11)
    np.testing.assert_allclose(out["P"].sum(axis=1), 1.0, atol=1e-12)
    N = w.n_nodes()
    for psi in out["psi"]:
        t = psi.reshape(N, N)
        sign = {0: None, 1: 1.0, 2: -1.0}[w.statistics]
        if sign is not None:
            np.testing.assert_allclose(t, sign * t.T, atol=1e-13)


def test_graph_taylor_matches_exact_evolution():
    # Algorithm 3 on a general graph against Eq. (evolPsi) by diagonalisation
    w = cw.get_graph("graph_small").with_(R=1, n_steps=50, obs_every=50)
    out = O.graph_ensemble_run(w)
    ue, uj = cw.graph_draws(w, [0])
    eu, ev = w.edges()
    eps, J = O.graph_parameters(ue[0], uj[0], w.eps_halfwidth, w.J0, w.J_halfwidth)
    N = w.n_nodes()
    H = O.many_particle_hamiltonian(O.graph_single_particle_hamiltonian(N, eu, ev, eps, J), w.m, w.U)
    psi0 = O.initial_state(N, w.m, w.sites, w.statistics)
    exact = O.exact_evolution(H, psi0, [w.dt * w.n_steps])[0]
    np.testing.assert_allclose(out["psi"][0], exact, atol=1e-11)
