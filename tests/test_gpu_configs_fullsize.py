"""The remaining workloads at their full sizes: ragged batch (2048 realizations,
N = 128..1024), three bosons on a ring (N = 160, 4.1M amplitudes per state),
a large FP64 state (N = 4096, 16.8M amplitudes) and the adjoint on N = 512.

Each runs in full on the GPU and is checked on outputs the oracle can compute
one realization at a time (the smallest members, or the first steps of the
same configuration), and on properties that hold at any size: norm and energy
conservation, exchange symmetry, P summing to the norm.
"""
import numpy as np
import pytest

import ctqw_workloads as cw
import oracle
from gpu_helpers import TOL_FP32, TOL_FP64, TOL_NORM_DRIFT, energy_tol, per_realization_P

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


def _oracle_one(w, r, n_steps=None):
    """Oracle propagation of realization r of workload w (P samples, norm, energy, psi)."""
    N = int(w.sizes()[r])
    ue, uj = cw.uniform_draws(w.seed, [r], [N])
    eps, J = oracle.workload_parameters(w, ue[0], uj[0], N)
    H = oracle.many_particle_hamiltonian(oracle.single_particle_hamiltonian(eps, J, w.periodic), w.m, w.U)
    psi0 = oracle.initial_state(N, w.m, w.initial_sites(N), w.statistics)
    n = w.n_steps if n_steps is None else n_steps
    return oracle.propagate(H, psi0, N, w.m, w.dt, n, w.obs_every if n_steps is None else n, "taylor", w.K)


def test_ragged_batch_full_size(ctqw):
    """2048 realizations with N drawn from {128, ..., 1024}, K = 8, 1000 steps, c64."""
    w = cw.get("ragged_n128_1024")
    got = ctqw.run_workload(w)
    sizes = got["sizes"]
    assert np.max(np.abs(got["norm"] - 1.0)) <= TOL_NORM_DRIFT
    assert np.max(np.abs(got["energy"] - got["energy"][0])) <= energy_tol(w)
    # each group's mean sums to the group's mean norm
    off = 0
    for g, N in enumerate(got["group_sizes"]):
        members = np.nonzero(sizes == N)[0]
        np.testing.assert_allclose(got["P_mean"][:, off:off + N].sum(axis=1),
                                   got["norm"][:, members].mean(axis=1), atol=2e-6)
        off += N
    # the oracle on the two smallest realizations (N = 128), full 1000 steps
    P_final = per_realization_P(got["psi"], got["st_off"], sizes, 2)
    for r in [int(i) for i in np.nonzero(sizes == sizes.min())[0][:2]]:
        ref = _oracle_one(w, r)
        assert np.max(np.abs(P_final[r] - ref["P"][-1])) <= TOL_FP32
        assert abs(got["norm"][-1, r] - ref["norm"][-1]) <= TOL_NORM_DRIFT


def test_three_bosons_ring_full_size(ctqw):
    """3 bosons on a ring of N = 160 (4.1M amplitudes), 64 realizations, K = 16, 1000 steps, c64."""
    w = cw.get("ring3_n160")
    got = ctqw.run_workload(w)
    assert np.max(np.abs(got["norm"] - 1.0)) <= TOL_NORM_DRIFT
    assert np.max(np.abs(got["energy"] - got["energy"][0])) <= energy_tol(w)
    np.testing.assert_allclose(got["P_mean"].sum(axis=1), got["norm"].mean(axis=1), atol=2e-6)
    # the state of realization 0 stays symmetric under every exchange of particles
    psi = got["psi"][got["st_off"][0]:got["st_off"][1]].reshape(160, 160, 160)
    scale = np.max(np.abs(psi))
    for perm in ((1, 0, 2), (0, 2, 1), (2, 1, 0)):
        assert np.max(np.abs(psi - np.transpose(psi, perm))) <= 1e-6 * scale


def test_three_bosons_ring_first_steps_against_oracle(ctqw):
    """Same configuration, first 12 steps, realization 0 against the oracle."""
    w = cw.get("ring3_n160").with_(R=2, n_steps=12, obs_every=12)
    got = ctqw.run_workload(w)
    ref = _oracle_one(w, 0)
    assert np.max(np.abs(got["P_mean"][-1] - (ref["P"][-1] + _oracle_one(w, 1)["P"][-1]) / 2)) <= TOL_FP32


def test_large_fp64_state_full_size(ctqw):
    """2 distinguishable walkers on N = 4096 (16.8M amplitudes, 268 MB per state),
    16 realizations, K = 16, 1000 steps, FP64."""
    w = cw.get("dist_n4096_c128")
    got = ctqw.run_workload(w)
    assert np.max(np.abs(got["norm"] - 1.0)) <= 1e-11
    assert np.max(np.abs(got["energy"] - got["energy"][0])) <= 1e-10
    np.testing.assert_allclose(got["P_mean"].sum(axis=1), got["norm"].mean(axis=1), atol=1e-12)


def test_large_fp64_state_first_steps_against_oracle(ctqw):
    w = cw.get("dist_n4096_c128").with_(N=4096, R=1, n_steps=3, obs_every=3)
    got = ctqw.run_workload(w)
    ref = _oracle_one(w, 0)
    assert np.max(np.abs(got["P_mean"][-1] - ref["P"][-1])) <= TOL_FP64


def test_adjoint_full_size_against_central_differences(ctqw):
    """Differentiation workload at full size: N = 512, 256 realizations, K = 14,
    1000 steps, checkpoints every 50, FP32 states with FP64 accumulation.  The
    gradient w.r.t. shared means is checked against central differences
    (h = 1e-4) of the loss computed by the same library in FP64."""
    w = cw.get("adjoint_n512")
    rng = np.random.default_rng(0x5EED7A46)
    N = w.N
    # target: P(x, T) of a hidden parameter set
    hidden_em = rng.uniform(-0.5, 0.5, N)
    hidden_jm = 1.0 + rng.uniform(-0.2, 0.2, N)
    em = np.zeros(N)
    jm = np.ones(N)

    def adjoint(eps_mean, J_mean, target):
        h = ctqw.build_for_workload(w, eps_mean=eps_mean, J_mean=J_mean, round_to_f32=False)
        psi = h.new_state(cw.C64)
        ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C64)
        loss, _, _, Pf, gem, gJm = ctqw.ctqw_adjoint_grad(h, psi, cw.C64, w.dt, w.K, w.n_steps, 50,
                                                          torch.tensor(target), per_realization=False)
        ctqw.ctqw_check_status(h)
        out = (float(loss.item()), gem.cpu().numpy(), gJm.cpu().numpy(), Pf.cpu().numpy())
        h.close()
        return out

    def loss64(eps_mean, J_mean, target):
        """Forward-only FP64 loss on Pbar(x, T) through the same library."""
        h = ctqw.build_for_workload(w, eps_mean=eps_mean, J_mean=J_mean, round_to_f32=False)
        psi = h.new_state(cw.C128)
        ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C128)
        P = torch.empty((2, h.p_width), dtype=torch.float64, device="cuda")
        ctqw.ctqw_propagate_taylor(h, psi, cw.C128, w.dt, w.K, w.n_steps, w.n_steps, P,
                                   workspace=h.workspace(cw.C128))
        ctqw.ctqw_check_status(h)
        h.close()
        return float(np.sum((P[-1].cpu().numpy() - target) ** 2))

    _, _, _, target = adjoint(hidden_em, hidden_jm, np.zeros(N))
    loss, ge, gJ, _ = adjoint(em, jm, target)
    assert loss > 0
    assert abs(loss - loss64(em, jm, target)) <= 1e-6 * max(loss, 1e-9) + 1e-12
    hfd = 1e-4
    for kind, i in (("eps", 255), ("J", 255)):
        a, b = em.copy(), jm.copy()
        a2, b2 = em.copy(), jm.copy()
        if kind == "eps":
            a[i] += hfd
            a2[i] -= hfd
        else:
            b[i] += hfd
            b2[i] -= hfd
        fd = (loss64(a, b, target) - loss64(a2, b2, target)) / (2 * hfd)
        got = ge[i] if kind == "eps" else gJ[i]
        assert abs(got - fd) <= 1e-3 * max(abs(fd), 1e-6), (kind, i, got, fd)


def test_large_two_particle_states_on_the_tiled_path_against_oracle(ctqw):
    """The default path for two particles in FP32 beyond N = 256 (temporally
    blocked register tiles), at full batch size, first steps: N = 512
    (256 realizations) and the ragged batch's largest members (N = 1024)."""
    w = cw.get("adjoint_n512").with_(n_steps=12, obs_every=12)
    got = ctqw.run_workload(w)
    P = per_realization_P(got["psi"], got["st_off"], got["sizes"], 2)
    for r in (0, w.R - 1):
        ref = _oracle_one(w, r)
        assert np.max(np.abs(P[r] - ref["P"][-1])) <= TOL_FP32
        assert abs(got["norm"][-1, r] - ref["norm"][-1]) <= TOL_NORM_DRIFT
    wr = cw.get("ragged_n128_1024").with_(n_steps=6, obs_every=6)
    got = ctqw.run_workload(wr)
    sizes = got["sizes"]
    P = per_realization_P(got["psi"], got["st_off"], sizes, 2)
    for r in [int(i) for i in np.nonzero(sizes == sizes.max())[0][:2]]:
        ref = _oracle_one(wr, r)
        assert np.max(np.abs(P[r] - ref["P"][-1])) <= TOL_FP32
