"""FP64 reference implementation of the CTQW hot path (test infrastructure).

Written from the paper's Sec. 2 (arXiv:1612.00746), in its order and notation:

* Eq. (Hij) / Sec. 2: the Hamiltonian of m particles on an N-site lattice is
  an N^m x N^m sparse matrix; diagonal entries are on-site energies, entries
  between connected nodes are (noisy) tunnelling amplitudes.  Readings taken
  here: hbar = 1; a bond carries -J (so the free walk is the Bessel walk);
  particles interact only on-site with energy U per pair; the many-particle
  matrix is the Kronecker sum of the single-particle matrix over the m
  particles plus diag(U * number of coinciding pairs).
* Eq. (Schroedinger) and Eq. (evolPsi), Algorithm 1: exact evolution by
  diagonalisation, used here as the plain definition exp(-i H t) psi.
* Algorithm 2: fourth-order Runge-Kutta step.
* Sec. 2.3 / Algorithm 3: truncated Taylor series of the evolution operator,
  Phi^(0) = Psi, Phi^(j) = -(i dt / j) H Phi^(j-1), Psi(t+dt) = sum_j Phi^(j).
* Sec. 2, q-dimensional lattices and general graphs: the one-particle matrix
  of a link list (graph_single_particle_hamiltonian), the same Kronecker sum
  over particles, noise per node and per link (graph_parameters).
* Sec. 2, density matrix <rho> = (1/R) sum_i |Psi_i><Psi_i|: its diagonal
  gives the site occupations P(x) averaged over realizations; its one-body
  reduction (partial trace over all particles but one) is one_body_density.

Everything is numpy / scipy in float64 / complex128, one realization at a time,
with no blocking, fusion or reordering beyond the algorithms themselves.
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, List, Optional, Sequence

import numpy as np
import scipy.sparse as sp

__all__ = [
    "round_f32", "lattice_parameters", "single_particle_hamiltonian",
    "many_particle_hamiltonian", "initial_state", "taylor_step", "rk4_step",
    "exact_evolution", "site_occupation", "pair_correlation", "norm", "energy",
    "propagate", "ensemble_run", "workload_parameters", "n_samples",
    "taylor_truncation_bound", "hamiltonian_norm_bound", "loss_and_adjoint_gradient",
    "occupation_weights", "noninteracting_evolution", "one_body_density",
    "philox4x64", "unit_double", "switch_parameters", "propagate_switching",
    "graph_parameters", "graph_single_particle_hamiltonian", "graph_ensemble_run",
]


# ---------------------------------------------------------------- parameters
def round_f32(x):
    """Nearest float32-representable value, returned as float64.

    Reading (the paper is silent on input precision): every disorder value is
    rounded to float32 so that FP32 and FP64 paths see identical inputs.
    """
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def lattice_parameters(u_eps, u_J, N, periodic, eps_mean, eps_halfwidth, J_mean,
                       J_halfwidth, round_to_f32=True):
    """On-site energies and hoppings of one realization (Eq. (Hij), c + xi).

    eps_i = c_ii + xi_ii with xi ~ Uniform[-w, w] drawn as w(2u - 1); the same
    for the hopping of bond b = (b, b+1 mod N).  Open chains have N-1 bonds,
    rings N.  ``eps_mean`` / ``J_mean`` are scalars or per-site / per-bond
    arrays (the deterministic part c of Eq. (Hij)).
    """
    n_bonds = N if periodic else N - 1
    u_eps = np.asarray(u_eps, dtype=np.float64)[:N]
    u_J = np.asarray(u_J, dtype=np.float64)[:n_bonds]
    eps = np.broadcast_to(np.asarray(eps_mean, dtype=np.float64), (N,)) + eps_halfwidth * (2.0 * u_eps - 1.0)
    J = np.broadcast_to(np.asarray(J_mean, dtype=np.float64), (n_bonds,)) + J_halfwidth * (2.0 * u_J - 1.0)
    if round_to_f32:
        eps, J = round_f32(eps), round_f32(J)
    return np.array(eps), np.array(J)


def single_particle_hamiltonian(eps, J, periodic):
    """Dense N x N one-particle matrix: eps on the diagonal, -J_b on bond b.

    Sec. 2: tunnelling only between nearest neighbours; bond b joins sites b
    and (b+1) mod N.  Entries are added, so a two-site ring gets -(J_0+J_1).
    """
    N = len(eps)
    H1 = np.diag(np.asarray(eps, dtype=np.float64)).astype(np.float64)
    for b in range(len(J)):
        i, k = b, (b + 1) % N
        H1[i, k] += -J[b]
        H1[k, i] += -J[b]
    return H1


def graph_parameters(u_eps, u_J, eps_halfwidth, J_mean, J_halfwidth, round_to_f32=True):
    """On-site energies of the nodes and hoppings of the links of a graph.

    Sec. 2 allows a q-dimensional lattice or a general graph; the disorder
    law is that of lattice_parameters (Eq. (Hij), c + xi with xi drawn as
    w(2u - 1)), one draw per node and one per link, zero mean on the nodes.
    """
    u_eps = np.asarray(u_eps, dtype=np.float64)
    u_J = np.asarray(u_J, dtype=np.float64)
    eps = 0.0 + eps_halfwidth * (2.0 * u_eps - 1.0)
    J = J_mean + J_halfwidth * (2.0 * u_J - 1.0)
    if round_to_f32:
        eps, J = round_f32(eps), round_f32(J)
    return np.array(eps, dtype=np.float64), np.array(J, dtype=np.float64)


def graph_single_particle_hamiltonian(n_nodes, edge_u, edge_v, eps, J):
    """Dense one-particle matrix of a graph: eps on the diagonal, -J_e on both
    entries of link e = (edge_u[e], edge_v[e]) (Sec. 2: tunnelling along the
    links of the topology, the same topology for every realization).  Entries
    add, so repeated links sum their hoppings.
    """
    H1 = np.diag(np.asarray(eps, dtype=np.float64)[:n_nodes]).astype(np.float64)
    for e in range(len(edge_u)):
        i, k = int(edge_u[e]), int(edge_v[e])
        if i == k:
            raise ValueError("a link must join two different nodes")
        H1[i, k] += -J[e]
        H1[k, i] += -J[e]
    return H1


def occupation_weights(N, m):
    """Pair-count diagonal of the interaction: #{j<l : x_j = x_l} per basis state."""
    grids = np.indices((N,) * m).reshape(m, -1)
    pairs = np.zeros(N ** m, dtype=np.float64)
    for j in range(m):
        for l in range(j + 1, m):
            pairs += (grids[j] == grids[l])
    return pairs


def many_particle_hamiltonian(H1, m, U):
    """N^m x N^m sparse matrix of m particles on the lattice of H1 (Sec. 2).

    H = sum_j I x ... x H1 (slot j) x ... x I + U * diag(#coinciding pairs),
    basis |x_1, ..., x_m> in row-major order (x_m fastest).
    """
    N = H1.shape[0]
    H1s = sp.csr_matrix(H1)
    I = sp.identity(N, format="csr", dtype=np.float64)
    H = sp.csr_matrix((N ** m, N ** m), dtype=np.float64)
    for j in range(m):
        term = None
        for slot in range(m):
            f = H1s if slot == j else I
            term = f if term is None else sp.kron(term, f, format="csr")
        H = H + term
    if U != 0.0:
        H = H + sp.diags(U * occupation_weights(N, m), format="csr")
    return sp.csr_matrix(H)


def initial_state(N, m, sites, statistics):
    """Localised initial state on ``sites`` (len m), complex128 of length N^m.

    0 = distinguishable |x_1..x_m>; 1 = bosons, the normalised sum over all
    permutations; 2 = fermions, the normalised signed sum (sites distinct).
    """
    psi = np.zeros((N,) * m, dtype=np.complex128)
    sites = tuple(int(s) for s in sites)
    if statistics == 0:
        psi[sites] = 1.0
    else:
        for perm in itertools.permutations(range(m)):
            sign = 1.0
            if statistics == 2:
                sign = _perm_sign(perm)
            psi[tuple(sites[p] for p in perm)] += sign
        nrm = np.sqrt(np.sum(np.abs(psi) ** 2))
        if nrm == 0.0:
            raise ValueError("fermions on a repeated site: the antisymmetric state vanishes")
        psi /= nrm
    return psi.reshape(-1)


def _perm_sign(perm):
    sign, seen = 1.0, list(perm)
    for i in range(len(seen)):
        while seen[i] != i:
            j = seen[i]
            seen[i], seen[j] = seen[j], seen[i]
            sign = -sign
    return sign


# ---------------------------------------------------------------- propagators
def taylor_step(H, psi, dt, K):
    """One step of Algorithm 3 (Sec. 2.3), in the paper's order.

    Phi^(0) <- Psi;  Psi(t+dt) <- Psi;  for j = 1..K:
    Phi^(j) <- -(1/j)(i dt) H Phi^(j-1);  Psi(t+dt) <- Psi(t+dt) + Phi^(j).
    """
    phi = psi.copy()
    out = psi.copy()
    for j in range(1, K + 1):
        phi = (-1j * dt / j) * (H @ phi)
        out = out + phi
    return out


def rk4_step(H, psi, dt):
    """One step of Algorithm 2: classical RK4 for d psi/dt = -i H psi.

    Reading of the paper's "sum_j mu_j K^(j)": mu = dt (1/6, 1/3, 1/3, 1/6),
    added to Psi(t); stages K^(1) = f(Psi), K^(2) = f(Psi + dt/2 K^(1)),
    K^(3) = f(Psi + dt/2 K^(2)), K^(4) = f(Psi + dt K^(3)).
    """
    f = lambda v: -1j * (H @ v)
    k1 = f(psi)
    k2 = f(psi + 0.5 * dt * k1)
    k3 = f(psi + 0.5 * dt * k2)
    k4 = f(psi + dt * k3)
    return psi + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def exact_evolution(H, psi0, times):
    """exp(-i H t) psi0 by diagonalisation (Eq. (evolPsi), Algorithm 1).

    H is real symmetric, so H = W diag(E) W^T with real orthogonal W and
    psi(t) = sum_j exp(-i E_j t) w_j <w_j | psi0>.  Returns [len(times), D].
    """
    Hd = H.toarray() if sp.issparse(H) else np.asarray(H)
    E, W = np.linalg.eigh(Hd)
    c = W.T @ psi0
    return np.stack([W @ (np.exp(-1j * E * t) * c) for t in times])


def noninteracting_evolution(eps, J, periodic, m, psi0, times):
    """exp(-i H t) psi0 for U = 0, where H is the Kronecker sum of H1.

    Then exp(-iHt) = exp(-iH1 t) (x) ... (x) exp(-iH1 t), and exp(-iH1 t) comes
    from Eq. (evolPsi) applied to the N x N one-particle matrix, so any state
    of an N^m tile is propagated exactly by applying it along every axis.
    Returns [len(times), N^m].
    """
    H1 = single_particle_hamiltonian(eps, J, periodic)
    N = H1.shape[0]
    E, W = np.linalg.eigh(H1)
    psi0 = np.asarray(psi0, dtype=np.complex128).reshape((N,) * m)
    out = []
    for t in times:
        G = (W * np.exp(-1j * E * t)) @ W.T
        psi = psi0
        for axis in range(m):
            psi = np.moveaxis(np.tensordot(G, psi, axes=([1], [axis])), 0, axis)
        out.append(psi.reshape(-1))
    return np.stack(out)


# ---------------------------------------------------------------- observables
def site_occupation(psi, N, m):
    """P(x) = (1/m) sum_j sum_{basis states with x_j = x} |psi|^2.

    Reading: the paper post-processes <rho> into observables without naming
    one; the one-body site occupation normalised to the norm (its diagonal
    marginals) is the observable here.
    """
    p = (np.abs(psi) ** 2).reshape((N,) * m)
    out = np.zeros(N, dtype=np.float64)
    for j in range(m):
        axes = tuple(a for a in range(m) if a != j)
        out += p.sum(axis=axes)
    return out / m


def one_body_density(psi, N, m):
    """One-body reduced density matrix, rho1(x, x') = (1/m) sum_j
    sum_{other coordinates} psi(.., x_j = x, ..) conj(psi(.., x_j = x', ..)).

    The partial trace of |Psi><Psi| (Sec. 2) over all particles but one,
    averaged over which particle is kept, so that trace(rho1) = <Psi|Psi>
    and diag(rho1) = site_occupation.  A matrix product per particle.
    """
    t = np.asarray(psi, dtype=np.complex128).reshape((N,) * m)
    out = np.zeros((N, N), dtype=np.complex128)
    for j in range(m):
        a = np.moveaxis(t, j, 0).reshape(N, -1)
        out += a @ a.conj().T
    return out / m


def pair_correlation(psi, N):
    """Two-particle diagonal of rho: |psi(x1, x2)|^2 as an N x N array (m = 2)."""
    return (np.abs(psi) ** 2).reshape(N, N)


def norm(psi):
    """<Psi|Psi> (the norm check of Algorithms 2 and 3)."""
    return float(np.sum(np.abs(psi) ** 2))


def energy(H, psi):
    """<Psi|H|Psi> (real for Hermitian H)."""
    return float(np.real(np.vdot(psi, H @ psi)))


def n_samples(n_steps, obs_every):
    return 0 if obs_every <= 0 else n_steps // obs_every + 1


def propagate(H, psi0, N, m, dt, n_steps, obs_every, method="taylor", K=16,
              keep_states=False, renormalize=False):
    """Propagate one realization, sampling P(x), norm and energy.

    Samples are taken at steps 0, obs_every, 2*obs_every, ... <= n_steps
    (reading of "averaged every 10 steps": samples in time, not a time mean).
    With renormalize, the state is divided by its norm after every step: the
    corrective action that the norm check of Algorithms 2 and 3 calls for
    (Sec. 2.2: RK4 does not conserve the norm).
    """
    psi = np.array(psi0, dtype=np.complex128)
    P, nr, en, states = [], [], [], [psi.copy()] if keep_states else None
    for n in range(n_steps + 1):
        if obs_every > 0 and n % obs_every == 0:
            P.append(site_occupation(psi, N, m))
            nr.append(norm(psi))
            en.append(energy(H, psi))
        if n == n_steps:
            break
        if method == "taylor":
            psi = taylor_step(H, psi, dt, K)
        elif method == "rk4":
            psi = rk4_step(H, psi, dt)
        else:
            raise ValueError(method)
        if renormalize:
            psi = psi / np.sqrt(norm(psi))
        if keep_states:
            states.append(psi.copy())
    out = {"P": np.array(P), "norm": np.array(nr), "energy": np.array(en), "psi": psi}
    if keep_states:
        out["states"] = states
    return out


# ---------------------------------------------------------------- ensembles
def workload_parameters(w, u_eps, u_J, N, eps_mean=None, J_mean=None, round_to_f32=True):
    """(eps, J) of one realization of a workload from its uniform draws."""
    em = 0.0 if eps_mean is None else eps_mean
    jm = w.J0 if J_mean is None else J_mean
    return lattice_parameters(u_eps, u_J, N, w.periodic, em, w.eps_halfwidth, jm,
                              w.J_halfwidth, round_to_f32)


def ensemble_run(w, realizations=None, method="taylor", K=None, n_steps=None,
                 obs_every=None, eps_mean=None, J_mean=None, renormalize=False):
    """Propagate the listed realizations of a workload and average P(x).

    Algorithm 3 per realization, then the diagonal of <rho> = (1/R) sum_i
    |Psi_i><Psi_i| reduced to P(x).  Realizations of different sizes are
    averaged within their own size group; groups are ordered by N and the
    averaged P of all groups are concatenated (reading for ragged batches).
    Returns per-realization P [R][n_obs][N_r], norms [R][n_obs], energies
    [R][n_obs], the group sizes and the group means [n_obs][sum_g N_g].
    """
    import ctqw_workloads as cw

    K = w.K if K is None else K
    n_steps = w.n_steps if n_steps is None else n_steps
    obs_every = w.obs_every if obs_every is None else obs_every
    sizes_all = w.sizes()
    if realizations is None:
        realizations = list(range(w.R))
    realizations = list(realizations)
    sizes = [int(sizes_all[r]) for r in realizations]
    ue, uj = cw.uniform_draws(w.seed, realizations, sizes)
    per_P, per_norm, per_energy, finals = [], [], [], []
    for k, r in enumerate(realizations):
        N = sizes[k]
        eps, J = workload_parameters(w, ue[k], uj[k], N, eps_mean, J_mean)
        H = many_particle_hamiltonian(single_particle_hamiltonian(eps, J, w.periodic), w.m, w.U)
        psi0 = initial_state(N, w.m, w.initial_sites(N), w.statistics)
        res = propagate(H, psi0, N, w.m, w.dt, n_steps, obs_every, method, K,
                        renormalize=renormalize)
        per_P.append(res["P"])
        per_norm.append(res["norm"])
        per_energy.append(res["energy"])
        finals.append(res["psi"])
    groups = sorted(set(sizes))
    n_obs = n_samples(n_steps, obs_every)
    mean = np.zeros((n_obs, sum(groups)), dtype=np.float64)
    off = 0
    for g in groups:
        members = [k for k in range(len(sizes)) if sizes[k] == g]
        mean[:, off:off + g] = sum(per_P[k] for k in members) / len(members)
        off += g
    return {"P": per_P, "norm": np.array(per_norm), "energy": np.array(per_energy),
            "sizes": sizes, "groups": groups, "P_mean": mean, "psi": finals}


# ---------------------------------------------------------------- switching noise
# Sec. 2: the stochastic parts of the Hamiltonian switch between values at
# random times, and Algorithms 1-3 update the switching times and H after
# every step.  Reading (the paper gives no law): after each step every
# stochastic parameter of every realization is redrawn, independently, with
# probability p from its own Uniform[-w, w] around its mean (discrete
# telegraph noise; waiting times geometric with mean 1/p steps).  The draws
# come from the counter-based generator Philox4x64-10 (Salmon et al., SC'11),
# written out here from its definition: key (seed, 0), counter
# (step, realization, site, 0); words 0, 1 decide and redraw eps of the
# site, words 2, 3 the hopping of the bond to its right.

_PHILOX_M = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
_PHILOX_W = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)
_U64 = (1 << 64) - 1


def philox4x64(counter, key):
    """Philox4x64-10: ten rounds of two 64x64 -> 128-bit products and a key
    schedule bumped by the Weyl constants; four 64-bit output words."""
    c = [int(x) & _U64 for x in counter]
    k = [int(x) & _U64 for x in key]
    for _ in range(10):
        p0 = _PHILOX_M[0] * c[0]
        p1 = _PHILOX_M[1] * c[2]
        hi0, lo0 = p0 >> 64, p0 & _U64
        hi1, lo1 = p1 >> 64, p1 & _U64
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
        k = [(k[0] + _PHILOX_W[0]) & _U64, (k[1] + _PHILOX_W[1]) & _U64]
    return c


def unit_double(word):
    """A 64-bit word to a double in [0, 1) from its top 53 bits."""
    return (int(word) >> 11) * 2.0 ** -53


def switch_parameters(eps, J, r, step, seed, p, N, periodic, eps_mean, eps_halfwidth,
                      J_mean, J_halfwidth, round_to_f32=True):
    """The Hamiltonian update after step ``step`` of realization ``r``.

    eps and J as lattice_parameters returns them (J: N - 1 bonds on an open
    chain, N on a ring); returns updated copies.
    """
    eps = np.array(eps, dtype=np.float64)
    J = np.array(J, dtype=np.float64)
    em = np.broadcast_to(np.asarray(eps_mean, dtype=np.float64), (N,))
    jm = np.broadcast_to(np.asarray(J_mean, dtype=np.float64), (N,))
    for i in range(N):
        w = philox4x64((step, r, i, 0), (seed, 0))
        if unit_double(w[0]) < p:
            v = em[i] + eps_halfwidth * (2.0 * unit_double(w[1]) - 1.0)
            eps[i] = round_f32(v) if round_to_f32 else v
        if i < len(J) and unit_double(w[2]) < p:
            v = jm[i] + J_halfwidth * (2.0 * unit_double(w[3]) - 1.0)
            J[i] = round_f32(v) if round_to_f32 else v
    return eps, J


def propagate_switching(w, r, seed, p, n_steps=None, obs_every=None, K=None):
    """One realization with switching noise: a Taylor step (Algorithm 3) with
    the current H, then the Hamiltonian update, n_steps times."""
    import ctqw_workloads as cw

    n_steps = w.n_steps if n_steps is None else n_steps
    obs_every = w.obs_every if obs_every is None else obs_every
    K = w.K if K is None else K
    N = int(w.sizes()[r])
    ue, uj = cw.uniform_draws(w.seed, [r], [N])
    eps, J = workload_parameters(w, ue[0], uj[0], N)
    psi = initial_state(N, w.m, w.initial_sites(N), w.statistics)
    P, nr, en = [], [], []
    for n in range(n_steps + 1):
        H = many_particle_hamiltonian(single_particle_hamiltonian(eps, J, w.periodic), w.m, w.U)
        if obs_every > 0 and n % obs_every == 0:
            P.append(site_occupation(psi, N, w.m))
            nr.append(norm(psi))
            en.append(energy(H, psi))
        if n == n_steps:
            break
        psi = taylor_step(H, psi, w.dt, K)
        eps, J = switch_parameters(eps, J, r, n, seed, p, N, w.periodic, 0.0, w.eps_halfwidth,
                                   w.J0, w.J_halfwidth)
    return {"P": np.array(P), "norm": np.array(nr), "energy": np.array(en), "psi": psi,
            "eps": eps, "J": J}


# ---------------------------------------------------------------- error bounds
def hamiltonian_norm_bound(m, eps_max, J_max, U):
    """Upper bound of ||H||_2: m (max|eps| + 2 max J) + U m(m-1)/2."""
    return m * (eps_max + 2.0 * J_max) + abs(U) * m * (m - 1) / 2.0


def taylor_truncation_bound(h_dt, K):
    """Remainder of the order-K Taylor series of exp(-i H dt) for ||H dt|| = h_dt.

    ||exp(-iA) - T_K(-iA)|| <= h^(K+1)/(K+1)! * exp(h)  (Lagrange remainder).
    """
    return h_dt ** (K + 1) / math.factorial(K + 1) * math.exp(h_dt)


# ---------------------------------------------------------------- adjoint
def loss_and_adjoint_gradient(eps_list, J_list, N, m, periodic, U, psi0, dt, K, n_steps,
                              P_target):
    """Loss sum_x (Pbar(x,T) - P*(x))^2 and its exact discrete gradient.

    The forward map is n_steps applications of Algorithm 3's polynomial
    T = sum_{k<=K} c_k H^k, c_k = (-i dt)^k / k!, per realization.  With
    lambda_T = g * psi_T, g(s) = dL/d|psi(s)|^2, the gradient of the step
    psi_{n+1} = T psi_n with respect to a parameter theta of H is
    2 Re <lambda_{n+1}, dT/dtheta psi_n>, and lambda_n = T^dagger lambda_{n+1}.
    Written out term by term: dT/dtheta = sum_k c_k sum_{a<k} H^{k-1-a} dH H^a.

    eps_list / J_list hold the (eps, J) of every realization; the returned
    gradients are with respect to those per-realization values, shape [R][N]
    and [R][n_bonds] (their sums over realizations are the gradients with
    respect to shared means).
    """
    R = len(eps_list)
    Hs, finals, histories = [], [], []
    for r in range(R):
        H1 = single_particle_hamiltonian(eps_list[r], J_list[r], periodic)
        H = many_particle_hamiltonian(H1, m, U)
        Hs.append(H)
        hist = [np.array(psi0, dtype=np.complex128)]
        for _ in range(n_steps):
            hist.append(taylor_step(H, hist[-1], dt, K))
        histories.append(hist)
        finals.append(hist[-1])
    Pbar = sum(site_occupation(p, N, m) for p in finals) / R
    diff = Pbar - np.asarray(P_target, dtype=np.float64)
    loss = float(np.sum(diff ** 2))
    # g(s) = sum_x 2 diff(x) (1/R) (1/m) #{j : s_j = x}
    grids = np.indices((N,) * m).reshape(m, -1)
    g = np.zeros(N ** m)
    for j in range(m):
        g += 2.0 * diff[grids[j]] / (R * m)
    c = [(-1j * dt) ** k / math.factorial(k) for k in range(K + 1)]
    n_bonds = N if periodic else N - 1
    g_eps = np.zeros((R, N))
    g_J = np.zeros((R, n_bonds))
    dH_eps = [_dH_eps(N, m, i) for i in range(N)]
    dH_J = [_dH_J(N, m, b) for b in range(n_bonds)]
    for r in range(R):
        H = Hs[r]
        lam = g * finals[r]
        for n in range(n_steps - 1, -1, -1):
            psi_n = histories[r][n]
            # phi_a = H^a psi_n, a = 0..K-1
            phis = [psi_n]
            for a in range(1, K):
                phis.append(H @ phis[-1])
            # mu_a = sum_{k=a+1..K} conj(c_k) H^{k-1-a} lambda
            mus = [None] * K
            mus[K - 1] = np.conj(c[K]) * lam
            for a in range(K - 2, -1, -1):
                mus[a] = np.conj(c[a + 1]) * lam + H @ mus[a + 1]
            for a in range(K):
                for i in range(N):
                    g_eps[r, i] += 2.0 * np.real(np.vdot(mus[a], dH_eps[i] @ phis[a]))
                for b in range(n_bonds):
                    g_J[r, b] += 2.0 * np.real(np.vdot(mus[a], dH_J[b] @ phis[a]))
            # lambda_n = T^dagger lambda_{n+1}
            acc = lam.copy()
            term = lam.copy()
            for k in range(1, K + 1):
                term = (1j * dt / k) * (H @ term)
                acc = acc + term
            lam = acc
    return loss, g_eps, g_J


def _dH_eps(N, m, i):
    """dH/d eps_i: diagonal count of particles on site i."""
    grids = np.indices((N,) * m).reshape(m, -1)
    return sp.diags((grids == i).sum(axis=0).astype(np.float64), format="csr")


def _dH_J(N, m, b):
    """dH/dJ_b: minus the hop across bond b = (b, b+1 mod N), for every particle."""
    d1 = np.zeros((N, N))
    i, k = b, (b + 1) % N
    d1[i, k] -= 1.0
    d1[k, i] -= 1.0
    return many_particle_hamiltonian(d1, m, 0.0)


# ---------------------------------------------------------------- graphs
def graph_ensemble_run(w, realizations=None, K=None, n_steps=None, obs_every=None, method="taylor"):
    """Algorithm 3 (or Algorithm 2, method="rk4") on every listed realization
    of a graph workload.

    The many-particle matrix is many_particle_hamiltonian of the graph's
    one-particle matrix (the Kronecker sum over particles of Sec. 2, with
    the lattice replaced by the graph).  Returns the realization-averaged P
    [n_obs][N], norms and energies [n_obs][n] and the final states.
    """
    if realizations is None:
        realizations = range(w.R)
    realizations = list(realizations)
    K = w.K if K is None else K
    n_steps = w.n_steps if n_steps is None else n_steps
    obs_every = w.obs_every if obs_every is None else obs_every
    from ctqw_workloads import graph_draws
    ue, uj = graph_draws(w, realizations)
    eu, ev = w.edges()
    N = w.n_nodes()
    P, norms, energies, finals = None, [], [], []
    for k in range(len(realizations)):
        eps, J = graph_parameters(ue[k], uj[k], w.eps_halfwidth, w.J0, w.J_halfwidth)
        H = many_particle_hamiltonian(graph_single_particle_hamiltonian(N, eu, ev, eps, J), w.m, w.U)
        psi0 = initial_state(N, w.m, w.sites, w.statistics)
        out = propagate(H, psi0, N, w.m, w.dt, n_steps, obs_every, method, K)
        P = out["P"] if P is None else P + out["P"]
        norms.append(out["norm"])
        energies.append(out["energy"])
        finals.append(out["psi"])
    n = max(len(realizations), 1)
    return {"P": None if P is None else P / n, "norm": np.array(norms).T,
            "energy": np.array(energies).T, "psi": finals}
