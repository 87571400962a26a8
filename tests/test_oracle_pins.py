"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, a brute-force construction
written independently here, a library routine for a special case that reduces
to it, or an invariant the mathematics fixes.  Together they are chosen so that
a dropped term, a wrong sign, a wrong index or a transposed operand anywhere in
the oracle fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.special

import ctqw_workloads as cw
import oracle as O


def _rand_params(rng, N, periodic, eps_w=1.0, J0=1.0, J_w=0.25):
    nb = N if periodic else N - 1
    eps = rng.uniform(-eps_w, eps_w, N)
    J = J0 + rng.uniform(-J_w, J_w, nb)
    return eps, J


def _brute_force_hamiltonian(eps, J, periodic, m, U):
    """Matrix elements of the many-particle Hamiltonian from its definition.

    Basis: all tuples (x_1..x_m), row-major.  Diagonal: sum_j eps[x_j] + U per
    coinciding pair.  Off-diagonal: particle j hops across bond b = (b, b+1 mod N)
    with amplitude -J_b in either direction.
    """
    N = len(eps)
    basis = list(itertools.product(range(N), repeat=m))
    index = {s: k for k, s in enumerate(basis)}
    H = np.zeros((len(basis), len(basis)))
    for s in basis:
        a = index[s]
        H[a, a] += sum(eps[x] for x in s)
        H[a, a] += U * sum(1 for j in range(m) for l in range(j + 1, m) if s[j] == s[l])
        for j in range(m):
            for b in range(len(J)):
                i, k = b, (b + 1) % N
                if s[j] == i:
                    t = list(s); t[j] = k
                    H[index[tuple(t)], a] += -J[b]
                if s[j] == k:
                    t = list(s); t[j] = i
                    H[index[tuple(t)], a] += -J[b]
    return H


@pytest.mark.parametrize("m,N,periodic,U", [(2, 5, False, 2.0), (2, 4, True, -1.5),
                                            (3, 4, False, 2.0), (3, 3, True, 1.0),
                                            (2, 2, True, 0.7)])
def test_hamiltonian_matches_brute_force_definition(m, N, periodic, U):
    rng = np.random.default_rng(1 + m * 10 + N)
    eps, J = _rand_params(rng, N, periodic)
    H = O.many_particle_hamiltonian(O.single_particle_hamiltonian(eps, J, periodic), m, U)
    Hb = _brute_force_hamiltonian(eps, J, periodic, m, U)
    np.testing.assert_allclose(H.toarray(), Hb, rtol=0, atol=1e-14)


def test_free_walk_bessel_closed_form():
    """U=0, clean, long open chain: each walker has amplitude i^|n| J_|n|(2Jt).

    (Jacobi-Anger expansion of exp(2iJt cos k); valid while the wave has not
    reached the chain ends.)  Two distinguishable walkers: the product.
    """
    N, a, b, t, J0 = 64, 31, 33, 3.0, 1.0
    eps, J = np.zeros(N), np.full(N - 1, J0)
    H = O.many_particle_hamiltonian(O.single_particle_hamiltonian(eps, J, False), 2, 0.0)
    psi0 = O.initial_state(N, 2, (a, b), 0)
    dt, n = 0.05, 60
    psi = psi0.copy()
    for _ in range(n):
        psi = O.taylor_step(H, psi, dt, 16)
    x = np.arange(N)
    amp = lambda s: (1j ** np.abs(x - s)) * scipy.special.jv(np.abs(x - s), 2 * J0 * t)
    expect = np.outer(amp(a), amp(b)).reshape(-1)
    assert np.max(np.abs(psi - expect)) < 1e-12


def test_clean_open_chain_sine_basis_any_time():
    """Clean open chain: eigenvectors sqrt(2/(N+1)) sin(pi k (i+1)/(N+1)),
    energies -2J cos(pi k/(N+1)); two walkers at U=0 evolve as the product."""
    N, J0, t = 7, 1.3, 13.7
    k = np.arange(1, N + 1)
    i = np.arange(N)
    V = np.sqrt(2.0 / (N + 1)) * np.sin(np.pi * np.outer(i + 1, k) / (N + 1))
    E = -2 * J0 * np.cos(np.pi * k / (N + 1))
    G = V @ np.diag(np.exp(-1j * E * t)) @ V.T   # single-particle propagator
    a, b = 1, 5
    expect = np.outer(G[:, a], G[:, b]).reshape(-1)
    H = O.many_particle_hamiltonian(
        O.single_particle_hamiltonian(np.zeros(N), np.full(N - 1, J0), False), 2, 0.0)
    got = O.exact_evolution(H, O.initial_state(N, 2, (a, b), 0), [t])[0]
    assert np.max(np.abs(got - expect)) < 1e-13
    psi = O.initial_state(N, 2, (a, b), 0)
    steps = 1370
    for _ in range(steps):
        psi = O.taylor_step(H, psi, t / steps, 14)
    assert np.max(np.abs(psi - expect)) < 1e-11


def test_clean_ring_plane_waves():
    """Clean ring: E_k = -2J cos(2 pi k / N), plane-wave eigenvectors."""
    N, J0, t = 6, 0.8, 4.2
    x = np.arange(N)
    G = sum(np.exp(-1j * (-2 * J0 * np.cos(2 * np.pi * q / N)) * t)
            * np.outer(np.exp(2j * np.pi * q * x / N), np.exp(-2j * np.pi * q * x / N)) / N
            for q in range(N))
    H = O.many_particle_hamiltonian(
        O.single_particle_hamiltonian(np.zeros(N), np.full(N, J0), True), 2, 0.0)
    got = O.exact_evolution(H, O.initial_state(N, 2, (0, 2), 0), [t])[0]
    expect = np.outer(G[:, 0], G[:, 2]).reshape(-1)
    assert np.max(np.abs(got - expect)) < 1e-13


def test_disordered_noninteracting_is_kronecker_product_of_expm():
    """U=0 with disorder: exp(-iHt) = exp(-iH1 t) (x) exp(-iH1 t) (scipy expm)."""
    rng = np.random.default_rng(7)
    N, t = 9, 2.5
    eps, J = _rand_params(rng, N, False)
    H1 = O.single_particle_hamiltonian(eps, J, False)
    G = scipy.linalg.expm(-1j * H1 * t)
    H = O.many_particle_hamiltonian(H1, 2, 0.0)
    psi = O.initial_state(N, 2, (3, 4), 0)
    dt = 0.02
    for _ in range(round(t / dt)):
        psi = O.taylor_step(H, psi, dt, 16)
    expect = np.outer(G[:, 3], G[:, 4]).reshape(-1)
    assert np.max(np.abs(psi - expect)) < 1e-12


def test_two_site_hubbard_two_bosons_closed_form():
    """Two bosons on two sites: symmetric-sector energies U and
    (U +- sqrt(U^2 + 16 J^2))/2; evolve |0,0> in closed form."""
    J0, U, t = 0.9, 2.3, 3.1
    H = O.many_particle_hamiltonian(
        O.single_particle_hamiltonian(np.zeros(2), np.array([J0]), False), 2, U)
    Hd = H.toarray()
    # spectrum of the symmetric sector (|00>, |11>, (|01>+|10>)/sqrt2)
    S = np.array([[1, 0, 0, 0], [0, 0, 0, 1], [0, 1 / np.sqrt(2), 1 / np.sqrt(2), 0]])
    ev = np.sort(np.linalg.eigvalsh(S @ Hd @ S.T))
    root = np.sqrt(U ** 2 + 16 * J0 ** 2)
    np.testing.assert_allclose(ev, np.sort([U, (U + root) / 2, (U - root) / 2]), atol=1e-14)
    # closed-form evolution of |0,0>
    Om = root / 2
    ph = np.exp(-1j * U * t / 2)
    plus = ph * (np.cos(Om * t) - 1j * (U / 2) / Om * np.sin(Om * t)) / np.sqrt(2)
    sym = ph * (1j * 2 * J0 / Om * np.sin(Om * t)) / np.sqrt(2)
    minus = np.exp(-1j * U * t) / np.sqrt(2)
    expect = np.array([(plus + minus) / np.sqrt(2), sym / np.sqrt(2), sym / np.sqrt(2),
                       (plus - minus) / np.sqrt(2)])
    psi = O.initial_state(2, 2, (0, 0), 1)
    dt = 0.01
    for _ in range(310):
        psi = O.taylor_step(H, psi, dt, 16)
    assert np.max(np.abs(psi - expect)) < 1e-12
    np.testing.assert_allclose(O.exact_evolution(H, O.initial_state(2, 2, (0, 0), 0), [t])[0],
                               expect, atol=1e-13)


def test_hong_ou_mandel_statistics():
    """Balanced two-site coupler (J t = pi/4), U=0: bosons bunch (no coincidences),
    fermions antibunch (no double occupancy), distinguishable: coincidence 1/2."""
    J0 = 1.0
    t = np.pi / 4
    H = O.many_particle_hamiltonian(
        O.single_particle_hamiltonian(np.zeros(2), np.array([J0]), False), 2, 0.0)
    out = {}
    for stat in (0, 1, 2):
        psi = O.exact_evolution(H, O.initial_state(2, 2, (0, 1), stat), [t])[0]
        out[stat] = O.pair_correlation(psi, 2)
    assert out[1][0, 1] + out[1][1, 0] < 1e-28
    assert out[2][0, 0] + out[2][1, 1] < 1e-28
    assert abs(out[0][0, 1] + out[0][1, 0] - 0.5) < 1e-14


def test_rk4_equals_fourth_order_taylor():
    """Sec. 2.3: for the exponential, order-n RK and order-n Taylor coincide."""
    rng = np.random.default_rng(3)
    N = 5
    eps, J = _rand_params(rng, N, True)
    H = O.many_particle_hamiltonian(O.single_particle_hamiltonian(eps, J, True), 2, 1.7)
    psi = rng.normal(size=N * N) + 1j * rng.normal(size=N * N)
    for dt in (0.01, 0.2):
        a = O.rk4_step(H, psi, dt)
        b = O.taylor_step(H, psi, dt, 4)
        assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(psi))
        c = O.taylor_step(H, psi, dt, 5)
        assert np.max(np.abs(a - c)) > 1e-12 * (dt / 0.2) ** 5


@pytest.mark.parametrize("m,N,periodic", [(2, 6, False), (3, 4, True)])
def test_taylor_within_truncation_bound_of_exact(m, N, periodic):
    rng = np.random.default_rng(11)
    eps, J = _rand_params(rng, N, periodic)
    U = 2.0
    H = O.many_particle_hamiltonian(O.single_particle_hamiltonian(eps, J, periodic), m, U)
    psi0 = O.initial_state(N, m, tuple(range(m)), 1)
    hn = O.hamiltonian_norm_bound(m, np.max(np.abs(eps)), np.max(J), U)
    Hn = np.linalg.norm(H.toarray(), 2)
    assert Hn <= hn + 1e-12
    for dt, K, steps in ((0.1, 6, 40), (0.05, 12, 80)):
        psi = psi0.copy()
        for _ in range(steps):
            psi = O.taylor_step(H, psi, dt, K)
        ex = O.exact_evolution(H, psi0, [dt * steps])[0]
        bound = steps * O.taylor_truncation_bound(Hn * dt, K)
        err = np.linalg.norm(psi - ex)
        assert err <= bound * 1.01 + 1e-13
    # K too small must visibly fail (the bound is not vacuous)
    psi = psi0.copy()
    for _ in range(40):
        psi = O.taylor_step(H, psi, 0.1, 2)
    assert np.linalg.norm(psi - O.exact_evolution(H, psi0, [4.0])[0]) > 1e-4


def test_conservation_and_symmetries():
    w = cw.get("bosons_small").with_(n_steps=200, obs_every=50, R=2)
    res = O.ensemble_run(w)
    for r in range(2):
        assert np.max(np.abs(res["norm"][r] - 1.0)) < 1e-12
        assert np.max(np.abs(res["energy"][r] - res["energy"][r][0])) < 1e-11
        # sum_x P(x) equals the norm
        np.testing.assert_allclose(res["P"][r].sum(axis=1), res["norm"][r], atol=1e-13)
        psi = res["psi"][r].reshape(w.N, w.N)
        assert np.max(np.abs(psi - psi.T)) < 1e-14      # bosons stay symmetric
    # fermions stay antisymmetric, with an empty diagonal
    wf = w.with_(statistics=cw.FERMIONS, R=1)
    psi = O.ensemble_run(wf)["psi"][0].reshape(w.N, w.N)
    assert np.max(np.abs(psi + psi.T)) < 1e-14
    assert np.max(np.abs(np.diag(psi))) < 1e-14


def test_mirror_symmetry_clean_chain():
    """Clean open chain, mirror-symmetric start: P(x) = P(N-1-x) for all t."""
    N = 10
    H = O.many_particle_hamiltonian(
        O.single_particle_hamiltonian(np.zeros(N), np.full(N - 1, 1.0), False), 2, 3.0)
    psi0 = O.initial_state(N, 2, (4, 5), 1)
    res = O.propagate(H, psi0, N, 2, 0.05, 200, 20, "taylor", 12)
    for P in res["P"]:
        np.testing.assert_allclose(P, P[::-1], atol=1e-13)


def test_ring_translation_covariance():
    N = 8
    H = O.many_particle_hamiltonian(
        O.single_particle_hamiltonian(np.zeros(N), np.full(N, 1.0), True), 2, 1.5)
    a = O.propagate(H, O.initial_state(N, 2, (1, 2), 1), N, 2, 0.05, 60, 60, "taylor", 12)
    b = O.propagate(H, O.initial_state(N, 2, (4, 5), 1), N, 2, 0.05, 60, 60, "taylor", 12)
    np.testing.assert_allclose(np.roll(a["P"][-1], 3), b["P"][-1], atol=1e-13)


def test_site_occupation_definition():
    # product state: P = (delta_a + delta_b)/2
    N = 5
    P = O.site_occupation(O.initial_state(N, 2, (1, 3), 0), N, 2)
    np.testing.assert_allclose(P, [0, 0.5, 0, 0.5, 0])
    # hand-computed 2x2 tile: |psi|^2 = [[a, b], [c, d]]
    psi = np.sqrt(np.array([0.1, 0.2, 0.3, 0.4])).astype(complex)
    # site 0: (row 0 sum + col 0 sum)/2 = ((0.1+0.2) + (0.1+0.3))/2
    np.testing.assert_allclose(O.site_occupation(psi, 2, 2), [0.35, 0.65], atol=1e-15)
    # three particles: site counts weighted 1/3 per particle
    psi3 = O.initial_state(3, 3, (0, 0, 2), 0)
    np.testing.assert_allclose(O.site_occupation(psi3, 3, 3), [2 / 3, 0, 1 / 3], atol=1e-15)
    # bosonic symmetrised 3-particle state is normalised and symmetric
    b3 = O.initial_state(4, 3, (0, 1, 1), 1).reshape(4, 4, 4)
    assert abs(np.sum(np.abs(b3) ** 2) - 1) < 1e-15
    for perm in itertools.permutations(range(3)):
        assert np.max(np.abs(b3 - np.transpose(b3, perm))) < 1e-15


def test_lattice_parameters_transform_and_rounding():
    u = np.array([0.0, 0.25, 0.5, 0.999])
    eps, J = O.lattice_parameters(u, u, 4, False, 0.0, 1.0, 1.0, 0.25)
    np.testing.assert_array_equal(eps, np.float32([-1.0, -0.5, 0.0, 0.998]).astype(np.float64))
    assert len(J) == 3
    np.testing.assert_array_equal(J, np.float32([0.75, 0.875, 1.0]).astype(np.float64))
    _, Jr = O.lattice_parameters(u, u, 4, True, 0.0, 1.0, 1.0, 0.25)
    assert len(Jr) == 4


def test_ensemble_mean_groups_ragged_sizes():
    w = cw.get("ragged_n128_1024").with_(ragged_sizes=(6, 8), R=5, n_steps=20, obs_every=10,
                                         sites=(-1, 0))
    res = O.ensemble_run(w)
    sizes = res["sizes"]
    assert res["groups"] == sorted(set(sizes))
    off = 0
    for g in res["groups"]:
        members = [k for k in range(5) if sizes[k] == g]
        np.testing.assert_allclose(res["P_mean"][:, off:off + g],
                                   np.mean([res["P"][k] for k in members], axis=0), atol=1e-15)
        off += g


def _loss(eps_list, J_list, N, m, periodic, U, psi0, dt, K, steps, target):
    finals = []
    for eps, J in zip(eps_list, J_list):
        H = O.many_particle_hamiltonian(O.single_particle_hamiltonian(eps, J, periodic), m, U)
        psi = psi0.copy()
        for _ in range(steps):
            psi = O.taylor_step(H, psi, dt, K)
        finals.append(psi)
    Pbar = sum(O.site_occupation(p, N, m) for p in finals) / len(finals)
    return float(np.sum((Pbar - target) ** 2))


def test_adjoint_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    N, m, periodic, U, dt, K, steps, R = 5, 2, False, 1.0, 0.05, 8, 12, 2
    eps_list, J_list = zip(*[_rand_params(rng, N, periodic, 0.5, 1.0, 0.2) for _ in range(R)])
    psi0 = O.initial_state(N, m, (1, 3), 0)
    target = rng.dirichlet(np.ones(N))
    loss, ge, gJ = O.loss_and_adjoint_gradient(list(eps_list), list(J_list), N, m, periodic, U,
                                               psi0, dt, K, steps, target)
    h = 1e-4
    for r in range(R):
        for i in range(N):
            ep = [e.copy() for e in eps_list]; em = [e.copy() for e in eps_list]
            ep[r][i] += h; em[r][i] -= h
            fd = (_loss(ep, J_list, N, m, periodic, U, psi0, dt, K, steps, target)
                  - _loss(em, J_list, N, m, periodic, U, psi0, dt, K, steps, target)) / (2 * h)
            assert abs(fd - ge[r, i]) < 1e-8 * max(1.0, abs(fd))
        for b in range(N - 1):
            jp = [j.copy() for j in J_list]; jm = [j.copy() for j in J_list]
            jp[r][b] += h; jm[r][b] -= h
            fd = (_loss(eps_list, jp, N, m, periodic, U, psi0, dt, K, steps, target)
                  - _loss(eps_list, jm, N, m, periodic, U, psi0, dt, K, steps, target)) / (2 * h)
            assert abs(fd - gJ[r, b]) < 1e-8 * max(1.0, abs(fd))
    assert abs(loss - _loss(eps_list, J_list, N, m, periodic, U, psi0, dt, K, steps, target)) < 1e-15


def test_adjoint_gradient_matches_eigenbasis_derivative():
    """Daleckii-Krein: d exp(-iHT) = W (F o (W^T dH W)) W^T with the divided
    differences F_ab = (e^{-iE_a T} - e^{-iE_b T})/(E_a - E_b), F_aa = -iT e^{-iE_a T}.
    The discrete Taylor gradient agrees to the truncation bound."""
    rng = np.random.default_rng(9)
    N, m, periodic, U, dt, K, steps = 4, 2, True, 1.3, 0.05, 14, 20
    eps, J = _rand_params(rng, N, periodic, 0.5, 1.0, 0.2)
    psi0 = O.initial_state(N, m, (0, 1), 1)
    target = rng.dirichlet(np.ones(N))
    _, ge, gJ = O.loss_and_adjoint_gradient([eps], [J], N, m, periodic, U, psi0, dt, K, steps, target)
    T = dt * steps
    H = O.many_particle_hamiltonian(O.single_particle_hamiltonian(eps, J, periodic), m, U).toarray()
    E, W = np.linalg.eigh(H)
    ph = np.exp(-1j * E * T)
    dE = E[:, None] - E[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        F = np.where(np.abs(dE) > 1e-9, (ph[:, None] - ph[None, :]) / np.where(dE == 0, 1, dE),
                     -1j * T * ph[:, None])
    psiT = W @ (ph * (W.T @ psi0))
    P = O.site_occupation(psiT, N, m)
    grids = np.indices((N, N)).reshape(2, -1)
    g = (2 * (P - target)[grids[0]] + 2 * (P - target)[grids[1]]) / 2

    def grad(dH):
        dpsi = W @ (F * (W.T @ dH @ W)) @ (W.T @ psi0)
        return float(np.sum(g * 2 * np.real(np.conj(psiT) * dpsi)))

    for i in range(N):
        d1 = np.zeros((N, N)); d1[i, i] = 1
        dH = O.many_particle_hamiltonian(d1, m, 0.0).toarray()
        assert abs(grad(dH) - ge[0, i]) < 1e-10
    for b in range(N):
        d1 = np.zeros((N, N)); d1[b, (b + 1) % N] -= 1; d1[(b + 1) % N, b] -= 1
        dH = O.many_particle_hamiltonian(d1, m, 0.0).toarray()
        assert abs(grad(dH) - gJ[0, b]) < 1e-10


@pytest.mark.parametrize("m,periodic,stats", [(2, False, 0), (2, True, 1), (3, False, 1), (3, True, 2)])
def test_noninteracting_evolution_matches_dense_exact_and_taylor(m, periodic, stats):
    rng = np.random.default_rng(21 + m)
    N = 5
    eps, J = _rand_params(rng, N, periodic)
    psi0 = O.initial_state(N, m, tuple(range(m)), stats)
    H = O.many_particle_hamiltonian(O.single_particle_hamiltonian(eps, J, periodic), m, 0.0)
    t = [0.0, 0.7, 3.3]
    a = O.noninteracting_evolution(eps, J, periodic, m, psi0, t)
    b = O.exact_evolution(H, psi0, t)
    assert np.max(np.abs(a - b)) < 1e-13
    psi = psi0.copy()
    for _ in range(330):
        psi = O.taylor_step(H, psi, 0.01, 14)
    assert np.max(np.abs(a[2] - psi)) < 1e-12


# ---------------------------------------------------------------- one-body density matrix
def _random_unit(N, rng):
    v = rng.normal(size=N) + 1j * rng.normal(size=N)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("m,N", [(2, 7), (3, 5)])
def test_one_body_density_diagonal_trace_hermitian(m, N):
    rng = np.random.default_rng(11)
    psi = rng.normal(size=N ** m) + 1j * rng.normal(size=N ** m)
    rho = O.one_body_density(psi, N, m)
    assert np.allclose(np.diag(rho).real, O.site_occupation(psi, N, m), rtol=0, atol=1e-12)
    assert np.allclose(np.diag(rho).imag, 0.0, atol=1e-13)
    assert abs(np.trace(rho).real - O.norm(psi)) <= 1e-11
    assert np.allclose(rho, rho.conj().T, atol=1e-13)
    assert np.min(np.linalg.eigvalsh(rho)) >= -1e-12


def test_one_body_density_of_product_states_closed_form():
    """|phi> x |chi> (x |eta>): rho1 = the mean of the one-particle projectors;
    the same for the symmetrised state of two orthogonal modes."""
    rng = np.random.default_rng(12)
    N = 6
    phi, chi, eta = (_random_unit(N, rng) for _ in range(3))
    proj = lambda v: np.outer(v, v.conj())
    rho2 = O.one_body_density(np.kron(phi, chi), N, 2)
    assert np.allclose(rho2, (proj(phi) + proj(chi)) / 2, atol=1e-14)
    rho3 = O.one_body_density(np.kron(np.kron(phi, chi), eta), N, 3)
    assert np.allclose(rho3, (proj(phi) + proj(chi) + proj(eta)) / 3, atol=1e-14)
    # two orthogonal modes, bosonic symmetrisation
    chi_o = chi - phi * np.vdot(phi, chi)
    chi_o /= np.linalg.norm(chi_o)
    sym = (np.kron(phi, chi_o) + np.kron(chi_o, phi)) / np.sqrt(2)
    assert np.allclose(O.one_body_density(sym, N, 2), (proj(phi) + proj(chi_o)) / 2, atol=1e-14)


def test_one_body_density_of_localized_state():
    """|a, b> (distinguishable): rho1 = (|a><a| + |b><b|) / 2 exactly."""
    N = 9
    psi = O.initial_state(N, 2, (2, 6), 0)
    rho = O.one_body_density(psi, N, 2)
    want = np.zeros((N, N))
    want[2, 2] = want[6, 6] = 0.5
    assert np.array_equal(rho, want)


# ---------------------------------------------------------------- switching noise
@pytest.mark.parametrize("ctr,key", [((7, 3, 2, 0), (0x1234, 0x5678)), ((0, 0, 0, 0), (0, 0)),
                                     ((2 ** 64 - 5, 11, 0, 9), (2 ** 63, 17))])
def test_philox_matches_numpy_bit_generator(ctr, key):
    """numpy's Philox (4x64-10) emits the block of counter + 1 first."""
    # the 256-bit counter minus one (word 0 least significant)
    v = sum(int(c) << (64 * i) for i, c in enumerate(ctr))
    v = (v - 1) % 2 ** 256
    prev = [(v >> (64 * i)) & (2 ** 64 - 1) for i in range(4)]
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(prev, dtype=np.uint64))
    assert [int(x) for x in bg.random_raw(4)] == O.philox4x64(ctr, key)


def test_switching_probability_and_range():
    N, p = 400, 0.2
    eps0 = np.zeros(N)
    J0 = np.ones(N - 1)
    switched_e, switched_j = 0, 0
    for step in range(10):
        e, j = O.switch_parameters(eps0, J0, 3, step, 99, p, N, False, 0.0, 1.0, 1.0, 0.25,
                                   round_to_f32=False)
        switched_e += np.count_nonzero(e != eps0)
        switched_j += np.count_nonzero(j != J0)
        assert np.all(np.abs(e) <= 1.0) and np.all(np.abs(j - 1.0) <= 0.25)
    n = 10 * N
    for k in (switched_e, switched_j * N / (N - 1)):
        assert abs(k / n - p) <= 5 * math.sqrt(p * (1 - p) / n)   # binomial, 5 sigma


def test_switching_with_zero_probability_is_static():
    w = cw.get("bosons_small").with_(N=10, R=1, sites=(4, 5), n_steps=20, obs_every=5, K=10)
    a = O.propagate_switching(w, 0, seed=5, p=0.0)
    b = O.ensemble_run(w)
    assert np.max(np.abs(a["P"] - b["P"][0])) <= 1e-15
    assert np.max(np.abs(a["psi"] - b["psi"][0])) <= 1e-15


def test_switching_conserves_norm_and_keeps_bosonic_symmetry():
    w = cw.get("bosons_small").with_(N=8, R=1, sites=(3, 4), n_steps=60, obs_every=10, K=14,
                                     dt=0.02)
    res = O.propagate_switching(w, 0, seed=7, p=0.3)
    assert np.max(np.abs(res["norm"] - 1.0)) <= 1e-12
    psi = res["psi"].reshape(8, 8)
    assert np.max(np.abs(psi - psi.T)) <= 1e-13
    # the parameters did switch, within their ranges
    static = O.ensemble_run(w)
    assert np.max(np.abs(res["P"][-1] - static["P"][0][-1])) > 1e-6
    assert np.all(np.abs(res["eps"]) <= w.eps_halfwidth)


@pytest.mark.parametrize("method", ["rk4", "taylor"])
def test_renormalized_propagation_is_the_state_over_its_norm(method):
    # H is linear, so dividing by the norm after every step gives the
    # unrenormalized state divided by its norm (closed form); a coarse dt
    # makes RK4 lose norm visibly first
    rng = np.random.default_rng(11)
    N, m, dt, steps = 9, 2, 0.3, 40
    eps, J = _rand_params(rng, N, False)
    H = O.many_particle_hamiltonian(O.single_particle_hamiltonian(eps, J, False), m, 1.5)
    psi0 = O.initial_state(N, m, (3, 5), 1)
    raw = O.propagate(H, psi0, N, m, dt, steps, 1, method, 4, keep_states=True)
    ren = O.propagate(H, psi0, N, m, dt, steps, 1, method, 4, keep_states=True, renormalize=True)
    assert abs(raw["norm"][-1] - 1.0) > 1e-6          # the correction has something to correct
    np.testing.assert_allclose(ren["norm"], 1.0, atol=1e-13)
    for a, b in zip(raw["states"], ren["states"]):
        np.testing.assert_allclose(b, a / np.sqrt(O.norm(a)), atol=1e-13)
    np.testing.assert_allclose(ren["P"], raw["P"] / raw["norm"][:, None], atol=1e-13)


# ---------------------------------------------------------------- energy values
# The pins above fix energy only through its conservation, which a wrong
# functional (the imaginary part, a constant factor, the diagonal only) would
# also satisfy.  These fix its value: <Psi|H|Psi> on states whose energy is
# known in closed form.

@pytest.mark.parametrize("m,sites,periodic", [(2, (1, 4), False), (2, (3, 3), False),
                                              (2, (0, 6), True), (3, (2, 2, 5), False),
                                              (3, (1, 1, 1), True)])
def test_energy_of_localised_states(m, sites, periodic):
    """|x_1..x_m> has E = sum_j eps_{x_j} + U #{j<l: x_j = x_l}: hops move
    amplitude off the site and contribute nothing to the expectation."""
    N, U = 7, 1.7
    rng = np.random.default_rng(7 + m)
    eps, J = _rand_params(rng, N, periodic)
    H = O.many_particle_hamiltonian(O.single_particle_hamiltonian(eps, J, periodic), m, U)
    psi = O.initial_state(N, m, sites, 0)
    pairs = sum(1 for j in range(m) for l in range(j + 1, m) if sites[j] == sites[l])
    expect = sum(eps[x] for x in sites) + U * pairs
    assert abs(O.energy(H, psi) - expect) < 1e-14
    # the same value from the sampled energies of a propagation (conserved)
    res = O.propagate(H, psi, N, m, 0.02, 30, 10, "taylor", 16)
    np.testing.assert_allclose(res["energy"], expect, atol=1e-12)


def test_energy_of_two_site_hubbard_eigenstates():
    """Two bosons on two sites: in the basis |+> = (|00> + |11>)/sqrt2,
    |s> = (|01> + |10>)/sqrt2 the Hamiltonian is [[U, -2J], [-2J, 0]], so
    (lam |+> - 2J |s>) / sqrt(lam^2 + 4J^2) has energy lam = (U +- sqrt(U^2 + 16 J^2))/2;
    (|00> - |11>)/sqrt2 has energy U.  A complex global phase leaves E unchanged."""
    J0, U = 0.8, 2.6
    H = O.many_particle_hamiltonian(
        O.single_particle_hamiltonian(np.zeros(2), np.array([J0]), False), 2, U)
    root = np.sqrt(U ** 2 + 16 * J0 ** 2)
    s2 = 1 / np.sqrt(2)
    plus = np.array([s2, 0, 0, s2])
    sym = np.array([0, s2, s2, 0])
    for lam in ((U + root) / 2, (U - root) / 2):
        v = (lam * plus - 2 * J0 * sym) / np.sqrt(lam ** 2 + 4 * J0 ** 2)
        assert abs(O.energy(H, np.exp(0.7j) * v.astype(complex)) - lam) < 1e-14
    minus = np.array([s2, 0, 0, -s2], dtype=complex)
    assert abs(O.energy(H, 1j * minus) - U) < 1e-14


@pytest.mark.parametrize("k1,k2,U", [(1, 1, 0.0), (2, 5, 0.0), (3, 7, 1.3)])
def test_energy_of_clean_chain_sine_mode_products(k1, k2, U):
    """Clean open chain: phi_k(i) = sqrt(2/(N+1)) sin(pi k (i+1)/(N+1)) has
    E_k = -2J cos(pi k/(N+1)).  The product phi_k1 x phi_k2 has energy
    E_k1 + E_k2 + U sum_x phi_k1(x)^2 phi_k2(x)^2 (the interaction acts on
    the diagonal x1 = x2 only)."""
    N, J0 = 9, 1.1
    H = O.many_particle_hamiltonian(
        O.single_particle_hamiltonian(np.zeros(N), np.full(N - 1, J0), False), 2, U)
    i = np.arange(N)
    phi = lambda k: np.sqrt(2 / (N + 1)) * np.sin(np.pi * k * (i + 1) / (N + 1))
    Ek = lambda k: -2 * J0 * np.cos(np.pi * k / (N + 1))
    psi = np.kron(phi(k1), phi(k2)).astype(complex)
    expect = Ek(k1) + Ek(k2) + U * np.sum(phi(k1) ** 2 * phi(k2) ** 2)
    assert abs(O.energy(H, psi) - expect) < 1e-13


def test_energy_of_ring_plane_waves():
    """Clean ring: e^{i q x}/sqrt(N) with q = 2 pi k / N has E = -2J cos q
    per particle; the energy of a complex state is real and uses both parts."""
    N, J0 = 8, 0.9
    H = O.many_particle_hamiltonian(
        O.single_particle_hamiltonian(np.zeros(N), np.full(N, J0), True), 2, 0.0)
    x = np.arange(N)
    for k1, k2 in ((1, 0), (3, 2), (1, 6)):
        q1, q2 = 2 * np.pi * k1 / N, 2 * np.pi * k2 / N
        psi = np.kron(np.exp(1j * q1 * x), np.exp(1j * q2 * x)) / N
        expect = -2 * J0 * (np.cos(q1) + np.cos(q2))
        assert abs(O.energy(H, psi) - expect) < 1e-14
