"""Seeded synthetic workloads for the many-particle CTQW hot path.

This module is shared by the CPU oracle (``oracle/``), the CUDA path's Python
binding, the tests and ``bench.py``.  It holds *no* arithmetic of the method:
only the workload shapes (lattice size, particle number, statistics, disorder
widths, time step, Taylor order, number of steps) and the seeded uniform draws
u in [0, 1) from which each side builds its own disorder.  Turning u into
on-site energies and hoppings is done separately by each side.

The paper (Sec. 4) benchmarks a 1D chain with two particles, nearest-neighbour
hopping and noise on the couplings, R = 1000 realizations and 1500 steps; it
publishes no data set, so every input here is synthetic.  The named workloads
below restate that family at the sizes used for parity and measurement.

Random streams: realization r of a workload with seed s draws from
``numpy.random.Philox`` keyed by ``SeedSequence([s, r])``, so the draws of a
realization do not depend on how many realizations are requested (subsets of
a workload see exactly the same disorder as the full workload).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional, Sequence, Tuple

import numpy as np

DISTINGUISHABLE = 0
BOSONS = 1
FERMIONS = 2

C64 = 0
C128 = 1

# Seed of the hidden parameter set that generates the target distribution of
# the differentiation workload (never handed to the optimiser).
HIDDEN_TARGET_SEED = 0x5EED7A46


@dataclass(frozen=True)
class Workload:
    """Shape of one ensemble propagation (all fields are plain data)."""

    name: str
    m: int                      # particles (2 or 3)
    statistics: int             # DISTINGUISHABLE / BOSONS / FERMIONS
    periodic: bool              # ring (True) or open chain (False)
    N: int                      # sites; for ragged workloads, the largest size
    R: int                      # noise realizations
    J0: float                   # mean hopping
    U: float                    # on-site interaction
    eps_halfwidth: float        # on-site disorder Uniform[-w, w]
    J_halfwidth: float          # hopping disorder Uniform[-w, w] around J0
    sites: Tuple[int, ...]      # initial occupied sites (len m); for ragged, offsets from N//2
    dt: float
    K: int                      # Taylor order
    n_steps: int
    obs_every: int              # sample P(x), norm, energy every this many steps
    dtype: int                  # C64 / C128
    seed: int = 0
    ragged_sizes: Optional[Tuple[int, ...]] = None   # allowed N values (ragged batches)
    centered_sites: bool = False                     # sites are offsets from N//2

    def sizes(self) -> np.ndarray:
        """Number of sites of every realization (int64, length R)."""
        if self.ragged_sizes is None:
            return np.full(self.R, self.N, dtype=np.int64)
        g = np.random.Generator(np.random.Philox(np.random.SeedSequence([self.seed, 0xA11])))
        u = g.random(self.R)
        choices = np.asarray(self.ragged_sizes, dtype=np.int64)
        return choices[np.minimum((u * len(choices)).astype(np.int64), len(choices) - 1)]

    def initial_sites(self, n_sites: int) -> Tuple[int, ...]:
        if self.centered_sites:
            return tuple(int(n_sites // 2 + s) for s in self.sites)
        return tuple(int(s) for s in self.sites)

    def site_updates(self) -> float:
        """Amplitude-term updates of the whole job: sum_r N_r^m * K * steps."""
        n = self.sizes().astype(np.float64)
        return float(np.sum(n ** self.m)) * self.K * self.n_steps

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def uniform_draws(seed: int, realizations: Sequence[int], n_sites: Sequence[int]):
    """Uniform draws for the disorder of the listed realizations.

    Returns two lists (u_eps, u_J); entry k holds float64 arrays of length
    n_sites[k] drawn from realization ``realizations[k]``'s own stream.  The
    hopping draws always have length N (the last one is ignored on open chains).
    """
    u_eps, u_J = [], []
    for r, n in zip(realizations, n_sites):
        g = np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(r)])))
        u_eps.append(g.random(int(n)))
        u_J.append(g.random(int(n)))
    return u_eps, u_J


def packed_draws(w: Workload, realizations: Optional[Sequence[int]] = None):
    """Draws of a workload packed back to back: (u_eps, u_J, sizes, offsets).

    ``offsets[k]`` is the start of realization k inside the packed arrays
    (length len(realizations) + 1); both arrays are float64 of length sum(N_r).
    """
    sizes_all = w.sizes()
    if realizations is None:
        realizations = range(w.R)
    realizations = list(realizations)
    sizes = sizes_all[realizations]
    ue, uj = uniform_draws(w.seed, realizations, sizes)
    offsets = np.zeros(len(realizations) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    if len(realizations) == 0:
        return np.zeros(0), np.zeros(0), sizes, offsets
    return np.concatenate(ue), np.concatenate(uj), sizes, offsets


# --------------------------------------------------------------------------
# Named workloads.  Sizes and physics follow the benchmark family of the
# paper's Sec. 4 (1D chain, two particles, noisy couplings, many realizations)
# at the scales listed in the design notes; "*_small" variants keep the same
# physics at sizes the oracle finishes in seconds.
# --------------------------------------------------------------------------

WORKLOADS = {
    # Plain FP64 path: 2 distinguishable walkers, open N=64 chain, on-site
    # disorder only, no interaction.
    "fp64_plain_n64": Workload(
        name="fp64_plain_n64", m=2, statistics=DISTINGUISHABLE, periodic=False, N=64, R=8,
        J0=1.0, U=0.0, eps_halfwidth=0.5, J_halfwidth=0.0, sites=(31, 32), dt=0.01, K=12,
        n_steps=1000, obs_every=10, dtype=C128, seed=0),
    # Precision workload (the headline): 2 bosons, N=256, U=2, noisy eps and J.
    "bosons_n256_u2": Workload(
        name="bosons_n256_u2", m=2, statistics=BOSONS, periodic=False, N=256, R=1024,
        J0=1.0, U=2.0, eps_halfwidth=1.0, J_halfwidth=0.25, sites=(127, 128), dt=0.02, K=16,
        n_steps=2500, obs_every=10, dtype=C64, seed=0),
    # Ragged batch: sizes drawn from {128, 192, ..., 1024}.
    "ragged_n128_1024": Workload(
        name="ragged_n128_1024", m=2, statistics=DISTINGUISHABLE, periodic=False, N=1024,
        R=2048, J0=1.0, U=1.0, eps_halfwidth=1.0, J_halfwidth=0.25, sites=(-1, 0), dt=0.02,
        K=8, n_steps=1000, obs_every=10, dtype=C64, seed=0,
        ragged_sizes=tuple(range(128, 1025, 64)), centered_sites=True),
    # Differentiation workload: learnable means + per-realization noise.
    "adjoint_n512": Workload(
        name="adjoint_n512", m=2, statistics=DISTINGUISHABLE, periodic=False, N=512, R=256,
        J0=1.0, U=0.0, eps_halfwidth=0.2, J_halfwidth=0.2, sites=(255, 256), dt=0.02, K=14,
        n_steps=1000, obs_every=1000, dtype=C64, seed=0),
    # Three bosons on a ring.
    "ring3_n160": Workload(
        name="ring3_n160", m=3, statistics=BOSONS, periodic=True, N=160, R=64,
        J0=1.0, U=2.0, eps_halfwidth=1.0, J_halfwidth=0.0, sites=(79, 80, 81), dt=0.01, K=16,
        n_steps=1000, obs_every=10, dtype=C64, seed=0),
    # Large two-particle state in FP64 (268 MB per realization).
    "dist_n4096_c128": Workload(
        name="dist_n4096_c128", m=2, statistics=DISTINGUISHABLE, periodic=False, N=4096, R=16,
        J0=1.0, U=2.0, eps_halfwidth=1.0, J_halfwidth=0.0, sites=(2047, 2048), dt=0.01, K=16,
        n_steps=1000, obs_every=10, dtype=C128, seed=0),
}

# Same physics, sizes the oracle finishes in seconds (several tiles and a
# ragged tail for the GPU kernels).
WORKLOADS_SMALL = {
    "fp64_plain_small": WORKLOADS["fp64_plain_n64"].with_(name="fp64_plain_small", n_steps=200),
    "bosons_small": WORKLOADS["bosons_n256_u2"].with_(
        name="bosons_small", N=64, R=6, sites=(31, 32), n_steps=300),
    "ring3_small": WORKLOADS["ring3_n160"].with_(
        name="ring3_small", N=12, R=3, sites=(5, 6, 7), n_steps=200),
}


def get(name: str) -> Workload:
    if name in WORKLOADS:
        return WORKLOADS[name]
    return WORKLOADS_SMALL[name]


# --------------------------------------------------------------------------
# q-dimensional lattices and general graphs (Sec. 2: a q-dimensional lattice
# of N = prod_i N_i nodes, or a general graph where each node has its own
# number of links).  A topology is an undirected link list shared by all
# realizations; the noise is one draw per node and one per link.
# --------------------------------------------------------------------------


def lattice_edges(shape: Sequence[int], periodic: bool) -> Tuple[np.ndarray, np.ndarray]:
    """Nearest-neighbour links of a q-dimensional lattice of extents ``shape``.

    Nodes are numbered row-major (the last direction fastest).  Along each
    direction i, node c is linked to c + e_i; with ``periodic`` the last node
    of a line is linked back to the first, so a direction of extent 2 gets
    two links between the same pair of nodes and extent 1 none.  Returns
    (u, v) int32 arrays; links are ordered by direction, then by node.
    """
    shape = tuple(int(n) for n in shape)
    n_nodes = int(np.prod(shape)) if shape else 0
    idx = np.arange(n_nodes).reshape(shape)
    us, vs = [], []
    for axis, n in enumerate(shape):
        if n < 2:
            continue
        nxt = np.roll(idx, -1, axis=axis)
        src = idx
        if not periodic:
            sl = [slice(None)] * len(shape)
            sl[axis] = slice(0, n - 1)
            src, nxt = idx[tuple(sl)], nxt[tuple(sl)]
        us.append(src.reshape(-1))
        vs.append(nxt.reshape(-1))
    if not us:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    return np.concatenate(us).astype(np.int32), np.concatenate(vs).astype(np.int32)


def ring_with_chords(n_nodes: int, n_chords: int, seed: int) -> Tuple[np.ndarray, np.ndarray]:
    """A general graph: a ring of ``n_nodes`` plus ``n_chords`` random links.

    Chord endpoints are uniform over distinct node pairs; a chord may repeat
    a link (the two then add), so node degrees vary from 2 upwards.
    """
    u = np.arange(n_nodes, dtype=np.int64)
    v = (u + 1) % n_nodes
    g = np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), 0x6EA])))
    a = g.integers(0, n_nodes, size=n_chords)
    b = (a + 1 + g.integers(0, n_nodes - 1, size=n_chords)) % n_nodes
    return (np.concatenate([u, a]).astype(np.int32), np.concatenate([v, b]).astype(np.int32))


@dataclass(frozen=True)
class GraphWorkload:
    """Ensemble propagation on a q-dimensional lattice or a general graph."""

    name: str
    m: int                      # particles (2 or 3)
    statistics: int
    shape: Tuple[int, ...]      # lattice extents N_1..N_q; () for the ring-with-chords graph
    periodic: bool              # lattices: periodic in every direction
    R: int
    J0: float
    U: float
    eps_halfwidth: float
    J_halfwidth: float
    sites: Tuple[int, ...]      # initial occupied nodes (len m)
    dt: float
    K: int
    n_steps: int
    obs_every: int
    dtype: int
    seed: int = 0
    ring_nodes: int = 0         # general graph: nodes of the ring
    chords: int = 0             # general graph: random chords on top of it

    def n_nodes(self) -> int:
        return int(np.prod(self.shape)) if self.shape else self.ring_nodes

    def edges(self) -> Tuple[np.ndarray, np.ndarray]:
        if self.shape:
            return lattice_edges(self.shape, self.periodic)
        return ring_with_chords(self.ring_nodes, self.chords, self.seed)

    def site_updates(self) -> float:
        """Amplitude-term updates of the whole job: R * N^m * K * steps."""
        return float(self.R) * float(self.n_nodes()) ** self.m * self.K * self.n_steps

    def with_(self, **kw) -> "GraphWorkload":
        return replace(self, **kw)


def graph_draws(w: GraphWorkload, realizations: Optional[Sequence[int]] = None):
    """Uniform draws (u_eps [n][N], u_J [n][E]) of the listed realizations.

    Realization r draws from Philox keyed by SeedSequence([seed, r, 0x62]).
    """
    if realizations is None:
        realizations = range(w.R)
    realizations = list(realizations)
    n, e = w.n_nodes(), len(w.edges()[0])
    ue = np.zeros((len(realizations), n))
    uj = np.zeros((len(realizations), e))
    for k, r in enumerate(realizations):
        g = np.random.Generator(np.random.Philox(np.random.SeedSequence([int(w.seed), int(r), 0x62])))
        ue[k] = g.random(n)
        uj[k] = g.random(e)
    return ue, uj


GRAPH_WORKLOADS = {
    # Two bosons on a 15 x 15 periodic square lattice (q = 2, m = 2,
    # N_1 N_2 = 225: the size Sec. 3 names as the memory limit of its GPUs),
    # noisy energies and hoppings, 1000 realizations, 1500 steps.
    "lattice2d_15x15_m2": GraphWorkload(
        name="lattice2d_15x15_m2", m=2, statistics=BOSONS, shape=(15, 15), periodic=True, R=1000,
        J0=1.0, U=2.0, eps_halfwidth=1.0, J_halfwidth=0.25, sites=(112, 113), dt=0.02, K=16,
        n_steps=1500, obs_every=10, dtype=C64, seed=0),
}

GRAPH_WORKLOADS_SMALL = {
    "lattice2d_small": GRAPH_WORKLOADS["lattice2d_15x15_m2"].with_(
        name="lattice2d_small", shape=(5, 4), R=4, sites=(9, 10), n_steps=120),
    "lattice2d_open_small": GRAPH_WORKLOADS["lattice2d_15x15_m2"].with_(
        name="lattice2d_open_small", shape=(6, 5), periodic=False, statistics=FERMIONS, R=3,
        sites=(14, 15), n_steps=100),
    "lattice3d_small": GRAPH_WORKLOADS["lattice2d_15x15_m2"].with_(
        name="lattice3d_small", shape=(3, 3, 4), statistics=DISTINGUISHABLE, R=3,
        sites=(17, 18), n_steps=80),
    "lattice2d_m3_small": GRAPH_WORKLOADS["lattice2d_15x15_m2"].with_(
        name="lattice2d_m3_small", m=3, shape=(4, 3), R=2, sites=(4, 5, 6), n_steps=60),
    "graph_small": GRAPH_WORKLOADS["lattice2d_15x15_m2"].with_(
        name="graph_small", shape=(), ring_nodes=40, chords=30, R=4, sites=(0, 20),
        statistics=DISTINGUISHABLE, n_steps=100),
}


def get_graph(name: str) -> GraphWorkload:
    if name in GRAPH_WORKLOADS:
        return GRAPH_WORKLOADS[name]
    return GRAPH_WORKLOADS_SMALL[name]
