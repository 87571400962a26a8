"""Host checks of the graph topologies and draws of ctqw_workloads (no GPU)."""
import numpy as np
import pytest

import ctqw_workloads as cw


def _degrees(u, v, n):
    return np.bincount(np.concatenate([u, v]), minlength=n)


@pytest.mark.parametrize("shape", [(3, 4), (5, 5), (3, 3, 4)])
def test_periodic_lattice_is_regular(shape):
    # every node has 2q neighbours on a torus with all extents >= 3
    u, v = cw.lattice_edges(shape, True)
    n = int(np.prod(shape))
    assert len(u) == len(shape) * n
    assert np.all(_degrees(u, v, n) == 2 * len(shape))
    assert np.all(u != v)


@pytest.mark.parametrize("shape", [(3, 4), (6, 5), (2, 3, 4)])
def test_open_lattice_link_count(shape):
    # sum over directions of (N_i - 1) prod_{j != i} N_j
    u, v = cw.lattice_edges(shape, False)
    n = int(np.prod(shape))
    expect = sum((shape[i] - 1) * n // shape[i] for i in range(len(shape)))
    assert len(u) == expect
    d = _degrees(u, v, n)
    assert d.min() == len(shape) and d.max() <= 2 * len(shape)


def test_lattice_links_join_nearest_neighbours():
    # row-major numbering: a link changes one coordinate by one (mod extent)
    shape = (4, 5)
    u, v = cw.lattice_edges(shape, True)
    cu = np.array(np.unravel_index(u, shape)).T
    cv = np.array(np.unravel_index(v, shape)).T
    diff = (cv - cu) % np.array(shape)
    assert np.all((diff != 0).sum(axis=1) == 1)
    assert np.all(diff[diff != 0] == 1)


def test_ring_with_chords_is_seeded_and_has_no_self_loops():
    u1, v1 = cw.ring_with_chords(40, 30, seed=3)
    u2, v2 = cw.ring_with_chords(40, 30, seed=3)
    u3, _ = cw.ring_with_chords(40, 30, seed=4)
    assert np.array_equal(u1, u2) and np.array_equal(v1, v2)
    assert not np.array_equal(u1, u3)
    assert np.all(u1 != v1)
    assert _degrees(u1, v1, 40).min() >= 2
    assert len(u1) == 70


def test_graph_draws_depend_on_the_realization_only():
    w = cw.get_graph("graph_small").with_(R=6)
    ue, uj = cw.graph_draws(w)
    se, sj = cw.graph_draws(w, [4, 1])
    assert np.array_equal(se, ue[[4, 1]]) and np.array_equal(sj, uj[[4, 1]])
    assert ue.shape == (6, w.n_nodes()) and uj.shape == (6, len(w.edges()[0]))
    assert np.all((ue >= 0) & (ue < 1)) and np.all((uj >= 0) & (uj < 1))
