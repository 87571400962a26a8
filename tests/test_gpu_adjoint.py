"""Adjoint gradient (ctqw_adjoint_grad) against the FP64 oracle's discrete adjoint,
against central differences of the GPU's own loss, and checkpoint invariance."""
import numpy as np
import pytest

import ctqw_workloads as cw
import oracle

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


def _workload(m=2, N=6, R=2, periodic=False, K=8, n_steps=12, dt=0.05, U=1.0, stats=0):
    sites = (1, 3) if m == 2 else (0, 1, 2)
    return cw.Workload(name="adj", m=m, statistics=stats, periodic=periodic, N=N, R=R, J0=1.0, U=U,
                       eps_halfwidth=0.5, J_halfwidth=0.2, sites=sites, dt=dt, K=K,
                       n_steps=n_steps, obs_every=0, dtype=cw.C128, seed=3)


def _gpu(ctqw, w, dtype, target, M=5, eps_mean=None, J_mean=None, round_to_f32=True):
    h = ctqw.build_for_workload(w, eps_mean=eps_mean, J_mean=J_mean, round_to_f32=round_to_f32)
    psi = h.new_state(dtype)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), dtype)
    loss, ge, gJ, Pf, _, _ = ctqw.ctqw_adjoint_grad(h, psi, dtype, w.dt, w.K, w.n_steps, M,
                                                    torch.tensor(target))
    ctqw.ctqw_check_status(h)
    eps, J = h.params()
    h.close()
    return (float(loss.item()), ge.cpu().numpy().reshape(w.R, w.N), gJ.cpu().numpy().reshape(w.R, w.N),
            Pf.cpu().numpy(), eps.reshape(w.R, w.N), J.reshape(w.R, w.N))


def _oracle(w, eps, J, target):
    nb = w.N if w.periodic else w.N - 1
    psi0 = oracle.initial_state(w.N, w.m, w.sites, w.statistics)
    return oracle.loss_and_adjoint_gradient([e for e in eps], [j[:nb] for j in J], w.N, w.m,
                                            w.periodic, w.U, psi0, w.dt, w.K, w.n_steps, target)


@pytest.mark.parametrize("m,N,periodic,K", [(2, 6, False, 8), (2, 5, True, 7), (3, 4, True, 6)])
def test_adjoint_fp64_matches_oracle(ctqw, m, N, periodic, K):
    w = _workload(m=m, N=N, periodic=periodic, K=K)
    target = np.random.default_rng(1).dirichlet(np.ones(N))
    loss, ge, gJ, Pf, eps, J = _gpu(ctqw, w, cw.C128, target)
    lo, ge_o, gJ_o = _oracle(w, eps, J, target)
    assert abs(loss - lo) <= 1e-13 * max(1.0, abs(lo))
    scale = max(np.max(np.abs(ge_o)), np.max(np.abs(gJ_o)))
    nb = N if periodic else N - 1
    assert np.max(np.abs(ge - ge_o)) <= 1e-11 * scale
    assert np.max(np.abs(gJ[:, :nb] - gJ_o)) <= 1e-11 * scale
    if not periodic:
        assert np.all(gJ[:, N - 1] == 0.0)


def test_adjoint_checkpoint_spacing_does_not_change_result(ctqw):
    w = _workload(n_steps=13)
    target = np.full(w.N, 1.0 / w.N)
    ref = _gpu(ctqw, w, cw.C128, target, M=1)
    for M in (2, 5, 13, 40):
        got = _gpu(ctqw, w, cw.C128, target, M=M)
        assert abs(got[0] - ref[0]) < 1e-15
        assert np.max(np.abs(got[1] - ref[1])) < 1e-13
        assert np.max(np.abs(got[2] - ref[2])) < 1e-13


def test_adjoint_fp32_states_fp64_accumulation(ctqw):
    w = _workload(N=8, R=3, n_steps=40, K=10)
    target = np.random.default_rng(2).dirichlet(np.ones(w.N))
    loss, ge, gJ, Pf, eps, J = _gpu(ctqw, w, cw.C64, target)
    lo, ge_o, gJ_o = _oracle(w, eps, J, target)
    scale = max(np.max(np.abs(ge_o)), np.max(np.abs(gJ_o)))
    assert abs(loss - lo) <= 1e-6 * max(1.0, lo)
    assert np.max(np.abs(ge - ge_o)) <= 1e-5 * scale
    assert np.max(np.abs(gJ[:, :w.N - 1] - gJ_o)) <= 1e-5 * scale


@pytest.mark.parametrize("N,periodic,K,n_steps", [(120, False, 14, 5), (110, True, 5, 6), (57, False, 9, 4),
                                                   (57, False, 1, 3), (57, True, 2, 3)])
def test_adjoint_fp32_register_tiles_span_several_tiles(ctqw, N, periodic, K, n_steps):
    """The c64 two-particle adjoint runs on register tiles (a 64 x 64 region,
    a tile of 64 - 2D per side): sizes that need several tiles per side and a
    ragged last tile, K that needs one and two launches per chain, both
    boundary conditions, against the FP64 oracle."""
    w = _workload(N=N, R=2, periodic=periodic, K=K, n_steps=n_steps, dt=0.03)
    target = np.random.default_rng(5).dirichlet(np.ones(N))
    loss, ge, gJ, Pf, eps, J = _gpu(ctqw, w, cw.C64, target, M=3)
    lo, ge_o, gJ_o = _oracle(w, eps, J, target)
    scale = max(np.max(np.abs(ge_o)), np.max(np.abs(gJ_o)))
    nb = N if periodic else N - 1
    assert abs(loss - lo) <= 1e-6 * max(1.0, lo)
    assert np.max(np.abs(ge - ge_o)) <= 1e-5 * scale
    assert np.max(np.abs(gJ[:, :nb] - gJ_o)) <= 1e-5 * scale
    if not periodic:
        assert np.all(gJ[:, N - 1] == 0.0)


def test_adjoint_fp32_ragged_register_tiles(ctqw):
    """Two size groups of several tiles each: per-realization gradients
    against the oracle, realization by realization."""
    w = cw.Workload(name="adj_ragged_tiles", m=2, statistics=1, periodic=True, N=104, R=3, J0=1.0,
                    U=1.0, eps_halfwidth=0.5, J_halfwidth=0.2, sites=(20, 21), dt=0.03, K=8,
                    n_steps=4, obs_every=0, dtype=cw.C64, seed=9, ragged_sizes=(56, 104))
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C64)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C64)
    groups = [int(g) for g in h.group_sizes]
    rng = np.random.default_rng(7)
    target = np.concatenate([rng.dirichlet(np.ones(g)) for g in groups])
    loss, ge, gJ, *_ = ctqw.ctqw_adjoint_grad(h, psi, cw.C64, w.dt, w.K, w.n_steps, 2, torch.tensor(target))
    ctqw.ctqw_check_status(h)
    eps, J = h.params()
    ge, gJ = ge.cpu().numpy(), gJ.cpu().numpy()
    sizes = [int(n) for n in h.sizes]
    po = np.concatenate([[0], np.cumsum(sizes)])
    h.close()
    goff = 0
    for g in groups:
        members = [r for r in range(w.R) if sizes[r] == g]
        psi0 = oracle.initial_state(g, 2, w.sites, w.statistics)
        e_l = [eps[po[r]:po[r + 1]] for r in members]
        j_l = [J[po[r]:po[r + 1]] for r in members]
        # the loss couples the realizations of a group only through its mean
        _, ge_o, gJ_o = oracle.loss_and_adjoint_gradient(e_l, j_l, g, 2, True, w.U, psi0, w.dt, w.K,
                                                         w.n_steps, target[goff:goff + g])
        scale = max(np.max(np.abs(ge_o)), np.max(np.abs(gJ_o)))
        for q, r in enumerate(members):
            assert np.max(np.abs(ge[po[r]:po[r + 1]] - ge_o[q])) <= 1e-5 * scale
            assert np.max(np.abs(gJ[po[r]:po[r + 1]] - gJ_o[q])) <= 1e-5 * scale
        goff += g


def test_adjoint_against_central_differences_of_gpu_loss(ctqw):
    """Gradient w.r.t. shared means (sum over realizations) vs central FD (h = 1e-4)
    of the GPU's own FP64 loss, without float32 rounding of the parameters."""
    w = _workload(N=6, R=2, n_steps=10, K=8)
    rng = np.random.default_rng(4)
    em = rng.uniform(-0.3, 0.3, w.N)
    jm = 1.0 + rng.uniform(-0.1, 0.1, w.N)
    target = rng.dirichlet(np.ones(w.N))
    _, ge, gJ, *_ = _gpu(ctqw, w, cw.C128, target, eps_mean=em, J_mean=jm, round_to_f32=False)
    h_fd = 1e-4
    for i in (0, 2, 5):
        ep, emn = em.copy(), em.copy()
        ep[i] += h_fd
        emn[i] -= h_fd
        fd = (_gpu(ctqw, w, cw.C128, target, eps_mean=ep, J_mean=jm, round_to_f32=False)[0] -
              _gpu(ctqw, w, cw.C128, target, eps_mean=emn, J_mean=jm, round_to_f32=False)[0]) / (2 * h_fd)
        assert abs(fd - ge[:, i].sum()) <= 1e-8 * max(1.0, abs(fd))
    for b in (0, 3):
        jp, jmn = jm.copy(), jm.copy()
        jp[b] += h_fd
        jmn[b] -= h_fd
        fd = (_gpu(ctqw, w, cw.C128, target, eps_mean=em, J_mean=jp, round_to_f32=False)[0] -
              _gpu(ctqw, w, cw.C128, target, eps_mean=em, J_mean=jmn, round_to_f32=False)[0]) / (2 * h_fd)
        assert abs(fd - gJ[:, b].sum()) <= 1e-8 * max(1.0, abs(fd))


def test_autograd_function_returns_summed_gradients(ctqw):
    """EnsembleOccupationLoss takes its gradients from the C call's sums over
    realizations; they must equal the oracle's per-realization gradients
    summed (the gradient with respect to the shared means)."""
    w = _workload(N=6, R=3, n_steps=8, K=8)
    em = torch.zeros(w.N, dtype=torch.float64, requires_grad=True)
    jm = torch.ones(w.N, dtype=torch.float64, requires_grad=True)
    target = torch.full((w.N,), 1.0 / w.N, dtype=torch.float64, device="cuda")
    loss = ctqw.EnsembleOccupationLoss.apply(em, jm, w, target, cw.C128, 4)
    loss.backward()
    eps, J = (a.reshape(w.R, w.N) for a in ctqw.build_for_workload(
        w, eps_mean=np.zeros(w.N), J_mean=np.ones(w.N)).params())
    lo, ge_o, gJ_o = _oracle(w, eps, J, target.cpu().numpy())
    assert abs(loss.item() - lo) <= 1e-13 * max(1.0, lo)
    scale = max(np.max(np.abs(ge_o)), np.max(np.abs(gJ_o)))
    np.testing.assert_allclose(em.grad.numpy(), ge_o.sum(0), atol=1e-11 * scale)
    np.testing.assert_allclose(jm.grad.numpy()[:w.N - 1], gJ_o.sum(0), atol=1e-11 * scale)
    assert jm.grad.numpy()[w.N - 1] == 0.0     # no wrap bond on an open chain


@pytest.mark.parametrize("dtype", [cw.C128, cw.C64])
def test_mean_gradients_are_group_sums_of_realization_gradients(ctqw, dtype):
    """A ragged batch (three size groups): grad_eps_mean / grad_J_mean hold,
    per group in ascending N, the sum over the group's realizations of the
    per-realization gradients, and match the oracle's sums."""
    w = cw.Workload(name="adj_ragged", m=2, statistics=0, periodic=False, N=7, R=7, J0=1.0,
                    U=1.0, eps_halfwidth=0.5, J_halfwidth=0.2, sites=(1, 3), dt=0.05, K=8,
                    n_steps=10, obs_every=0, dtype=dtype, seed=4, ragged_sizes=(5, 6, 7))
    h = ctqw.build_for_workload(w)
    psi = h.new_state(dtype)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), dtype)
    groups = [int(g) for g in h.group_sizes]
    assert groups == [5, 6, 7]
    rng = np.random.default_rng(3)
    target = np.concatenate([rng.dirichlet(np.ones(g)) for g in groups])
    loss, ge, gJ, _, gem, gJm = ctqw.ctqw_adjoint_grad(h, psi, dtype, w.dt, w.K, w.n_steps, 4,
                                                       torch.tensor(target))
    ctqw.ctqw_check_status(h)
    eps, J = h.params()
    ge, gJ, gem, gJm = (a.cpu().numpy() for a in (ge, gJ, gem, gJm))
    hsizes = [int(n) for n in h.sizes]
    h.close()
    offs = np.concatenate([[0], np.cumsum(hsizes)])
    tol = 1e-11 if dtype == cw.C128 else 1e-5
    goff = 0
    for g in groups:
        members = [r for r in range(w.R) if hsizes[r] == g]
        # the C sums are exactly the per-realization outputs summed in order
        se = sum(ge[offs[r]:offs[r] + g] for r in members)
        sj = sum(gJ[offs[r]:offs[r] + g] for r in members)
        np.testing.assert_allclose(gem[goff:goff + g], se, rtol=0, atol=1e-15 * max(1, np.abs(se).max()))
        np.testing.assert_allclose(gJm[goff:goff + g], sj, rtol=0, atol=1e-15 * max(1, np.abs(sj).max()))
        # and the oracle's gradients of this group's realizations, summed
        psi0 = oracle.initial_state(g, 2, w.initial_sites(g), 0)
        _, ge_o, gJ_o = oracle.loss_and_adjoint_gradient(
            [eps[offs[r]:offs[r] + g] for r in members], [J[offs[r]:offs[r] + g - 1] for r in members],
            g, 2, False, w.U, psi0, w.dt, w.K, w.n_steps, target[goff:goff + g])
        scale = max(np.abs(ge_o).max(), np.abs(gJ_o).max())
        assert np.max(np.abs(gem[goff:goff + g] - ge_o.sum(0))) <= tol * scale
        assert np.max(np.abs(gJm[goff:goff + g - 1] - gJ_o.sum(0))) <= tol * scale
        assert gJm[goff + g - 1] == 0.0
        goff += g
