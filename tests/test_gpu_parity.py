"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Sizes here are small enough for the oracle to finish in seconds while still
spanning several warp blocks / CTAs and, for the plain kernels, a ragged tail.
"""
import numpy as np
import pytest

import ctqw_workloads as cw
import oracle
from gpu_helpers import TOL_FP32, TOL_FP64, TOL_NORM_DRIFT, energy_tol, oracle_params, per_realization_P

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


def _compare(got, ref, tolP, tol_norm, tol_energy):
    dP = np.max(np.abs(got["P_mean"] - ref["P_mean"]))
    dn = np.max(np.abs(got["norm"] - ref["norm"].T))
    de = np.max(np.abs(got["energy"] - ref["energy"].T))
    assert dP <= tolP, f"max|dP| = {dP:.3e} > {tolP:.1e}"
    assert dn <= tol_norm, f"max|dnorm| = {dn:.3e}"
    assert de <= tol_energy, f"max|dE| = {de:.3e}"
    return dP, dn, de


# ------------------------------------------------------------------ inputs
@pytest.mark.parametrize("name,kw", [
    ("bosons_small", {}),
    ("ring3_small", {}),
    ("fp64_plain_small", {}),
    ("ragged_n128_1024", {"ragged_sizes": (6, 10, 64), "R": 7}),
])
def test_params_bit_exact(ctqw, name, kw):
    w = cw.get(name).with_(**kw)
    h = ctqw.build_for_workload(w)
    eps, J = h.params()
    ref = oracle_params(w)
    off = 0
    for r, (e_ref, j_ref) in enumerate(ref):
        N = len(e_ref)
        assert np.array_equal(eps[off:off + N], e_ref), r
        assert np.array_equal(J[off:off + N], j_ref), r
        off += N
    h.close()


def test_params_with_means_bit_exact(ctqw):
    w = cw.get("adjoint_n512").with_(N=16, R=3)
    rng = np.random.default_rng(0)
    em = rng.uniform(-1, 1, 16)
    jm = 1 + rng.uniform(-0.2, 0.2, 16)
    h = ctqw.build_for_workload(w, eps_mean=em, J_mean=jm)
    eps, J = h.params()
    for r, (e_ref, j_ref) in enumerate(oracle_params(w, eps_mean=em, J_mean=jm[:15])):
        assert np.array_equal(eps[16 * r:16 * r + 16], e_ref)
        assert np.array_equal(J[16 * r:16 * r + 16], j_ref)
    h.close()


@pytest.mark.parametrize("m,stats,sites", [(2, 0, (3, 5)), (2, 1, (3, 5)), (2, 1, (4, 4)),
                                           (2, 2, (1, 6)), (3, 0, (0, 2, 2)), (3, 1, (0, 2, 2)),
                                           (3, 1, (1, 1, 1)), (3, 2, (0, 3, 5))])
def test_initial_states(ctqw, m, stats, sites):
    N = 7
    w = cw.Workload(name="t", m=m, statistics=stats, periodic=False, N=N, R=2, J0=1, U=0,
                    eps_halfwidth=0, J_halfwidth=0, sites=sites, dt=0.1, K=4, n_steps=1,
                    obs_every=1, dtype=cw.C128)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C128)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C128)
    got = psi.cpu().numpy()
    ref = oracle.initial_state(N, m, sites, stats)
    for r in range(2):
        np.testing.assert_allclose(got[r * N ** m:(r + 1) * N ** m], ref, rtol=0, atol=1e-15)
    h.close()


def test_fermions_on_same_site_rejected(ctqw):
    w = cw.get("bosons_small").with_(statistics=cw.FERMIONS, R=1)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C128)
    with pytest.raises(ctqw.CtqwError, match="same site"):
        ctqw.ctqw_init_state(h, psi, [[3, 3]], cw.C128)
    with pytest.raises(ctqw.CtqwError, match="outside"):
        ctqw.ctqw_init_state(h, psi, [[3, 64]], cw.C128)
    h.close()


# ------------------------------------------------------------------ FP64 plain path
def test_taylor_fp64_plain_two_particles(ctqw):
    w = cw.get("fp64_plain_small")
    got = ctqw.run_workload(w)
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP64, 1e-12, 1e-11)


def test_taylor_fp64_three_bosons_ring(ctqw):
    w = cw.get("ring3_small").with_(dtype=cw.C128)
    got = ctqw.run_workload(w)
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP64, 1e-12, 1e-10)


@pytest.mark.parametrize("N,periodic,stats", [(40, True, 1), (36, False, 0)])
def test_taylor_fp32_three_particles_several_slabs(ctqw, N, periodic, stats):
    """The FP32 three-particle stages walk x1 in slabs of 32 with x3 across
    the lanes: N = 40 and 36 give a ragged last slab and a partly idle warp,
    on a ring (bosons) and on an open chain (distinguishable)."""
    w = cw.get("ring3_small").with_(N=N, periodic=periodic, statistics=stats, R=2,
                                    sites=(N // 2 - 1, N // 2, N // 2 + 1), n_steps=40, obs_every=20)
    got = ctqw.run_workload(w)
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP32, TOL_NORM_DRIFT, energy_tol(w))


def test_taylor_fp64_ragged_sizes_grouped(ctqw):
    w = cw.get("ragged_n128_1024").with_(ragged_sizes=(6, 10, 17), R=7, n_steps=60, obs_every=20,
                                         dtype=cw.C128, K=10)
    got = ctqw.run_workload(w)
    ref = oracle.ensemble_run(w)
    assert list(got["group_sizes"]) == ref["groups"]
    _compare(got, ref, TOL_FP64, 1e-12, 1e-10)


def test_rk4_fp64(ctqw):
    w = cw.get("bosons_small").with_(R=2, n_steps=100, obs_every=25, dtype=cw.C128)
    got = ctqw.run_workload(w, method=ctqw.RK4)
    ref = oracle.ensemble_run(w, method="rk4")
    _compare(got, ref, TOL_FP64, 1e-12, 1e-10)


def test_rk4_equals_order4_taylor_on_gpu(ctqw):
    w = cw.get("bosons_small").with_(R=2, n_steps=50, obs_every=50, dtype=cw.C128)
    a = ctqw.run_workload(w, method=ctqw.RK4)
    b = ctqw.run_workload(w, K=4, flags=ctqw.FLAG_PLAIN)
    assert np.max(np.abs(a["psi"] - b["psi"])) < 1e-13


@pytest.mark.parametrize("K", [1, 2, 5, 7])
def test_fp64_plain_any_order(ctqw, K):
    w = cw.get("bosons_small").with_(R=2, n_steps=30, obs_every=10, dtype=cw.C128, K=K)
    got = ctqw.run_workload(w)
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP64, 1e-12, 1e-10)


# ------------------------------------------------------------------ FP32 paths
def test_fused_c64_bosons(ctqw):
    w = cw.get("bosons_small")
    got = ctqw.run_workload(w)
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP32, TOL_NORM_DRIFT, energy_tol(w))
    assert np.max(np.abs(got["norm"] - 1.0)) <= TOL_NORM_DRIFT


@pytest.mark.parametrize("N,periodic,K", [(64, True, 16), (128, False, 16), (192, False, 13),
                                          (256, False, 16), (256, True, 5)])
def test_fused_c64_shapes(ctqw, N, periodic, K):
    w = cw.get("bosons_n256_u2").with_(N=N, R=2, periodic=periodic, K=K, n_steps=24, obs_every=8,
                                       sites=(N // 2 - 1, N // 2))
    got = ctqw.run_workload(w)
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP32, TOL_NORM_DRIFT, energy_tol(w))
    P = per_realization_P(got["psi"], got["st_off"], got["sizes"], 2)
    for r in range(2):
        assert np.max(np.abs(P[r] - ref["P"][r][-1])) <= TOL_FP32


@pytest.mark.parametrize("name,kw", [
    ("bosons_small", {"K": 1}), ("bosons_small", {"K": 2}), ("bosons_small", {"K": 30}),     # fused, N = 64
    ("bosons_small", {"N": 96, "sites": (47, 48), "K": 1}),                                   # register tiles
    ("bosons_small", {"N": 96, "sites": (47, 48), "K": 30}),
    ("ring3_small", {"K": 1}), ("ring3_small", {"K": 30}),                                    # m = 3 stages
])
def test_c64_orders_at_the_ends_of_the_range(ctqw, name, kw):
    """K = 1 (one final stage), K = 2 and K = 30 (the largest order) on each
    FP32 path against the oracle (the order-1 map is not unitary: both sides
    follow the same norm)."""
    w = cw.get(name).with_(R=2, n_steps=10, obs_every=5, **kw)
    got = ctqw.run_workload(w)
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP32, TOL_NORM_DRIFT, energy_tol(w))


@pytest.mark.parametrize("name,kw", [
    ("bosons_small", {"sites": (20, 41)}),                                        # fused, N = 64
    ("bosons_small", {"N": 96, "sites": (30, 61)}),                               # register tiles
    ("ring3_small", {"sites": (2, 5, 9)}),                                        # m = 3 stages
])
def test_c64_fermions_stay_antisymmetric(ctqw, name, kw):
    """Fermions (an antisymmetrised initial state) on each FP32 path: the
    oracle's P, norm and energy, and psi odd under every exchange of two
    particles (zero where two coordinates coincide)."""
    w = cw.get(name).with_(statistics=cw.FERMIONS, R=2, n_steps=30, obs_every=10, **kw)
    got = ctqw.run_workload(w)
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP32, TOL_NORM_DRIFT, energy_tol(w))
    N, m = w.N, w.m
    psi = got["psi"][got["st_off"][0]:got["st_off"][1]].reshape((N,) * m)
    scale = np.max(np.abs(psi))
    perms = [(1, 0)] if m == 2 else [(1, 0, 2), (0, 2, 1), (2, 1, 0)]
    for perm in perms:
        assert np.max(np.abs(psi + np.transpose(psi, perm))) <= 1e-6 * scale


def test_fused_snapshot_slots_do_not_change_the_result(ctqw):
    """The fused path runs S + 1 sampling intervals per launch with S
    snapshot slots in the workspace (S = bytes / state - 1): S = 0, 2 and 7
    on 47 steps sampled every 3 (launches that end mid-interval and a last
    short one) give the same state bit for bit, the same samples up to the
    order of the FP64 atomics that combine blocks, and match the oracle."""
    w = cw.get("bosons_small").with_(R=3, n_steps=47, obs_every=3)
    ref = oracle.ensemble_run(w)
    outs = []
    for S in (0, 2, 7):
        h = ctqw.build_for_workload(w)
        psi = h.new_state(cw.C64)
        ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C64)
        n_obs = h.n_obs(w.n_steps, w.obs_every)
        P = torch.empty((n_obs, h.p_width), dtype=torch.float64, device="cuda")
        nr = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
        en = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
        ws = torch.empty((S + 1) * psi.numel() * 8, dtype=torch.uint8, device="cuda")
        ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en, 0, ws)
        ctqw.ctqw_check_status(h)
        outs.append([t.cpu().numpy() for t in (psi, P, nr, en)])
        h.close()
    for other in outs[1:]:
        assert np.array_equal(outs[0][0], other[0])          # the state, bit for bit
        for a, b in zip(outs[0][1:], other[1:]):             # FP64 sums (atomic order)
            assert np.max(np.abs(a - b)) <= 1e-13
    assert np.max(np.abs(outs[0][1] - ref["P_mean"])) <= TOL_FP32
    assert np.max(np.abs(outs[0][2] - ref["norm"].T)) <= TOL_NORM_DRIFT
    assert np.max(np.abs(outs[0][3] - ref["energy"].T)) <= energy_tol(w)


def test_fused_c64_distinguishable_open(ctqw):
    w = cw.get("fp64_plain_small").with_(dtype=cw.C64, n_steps=300, obs_every=30)
    got = ctqw.run_workload(w)
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP32, TOL_NORM_DRIFT, energy_tol(w))


def test_plain_c64(ctqw):
    w = cw.get("bosons_small").with_(n_steps=100, obs_every=25)
    got = ctqw.run_workload(w, flags=ctqw.FLAG_PLAIN)
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP32, TOL_NORM_DRIFT, energy_tol(w))


@pytest.mark.parametrize("flags", [0, 1])   # fused (order-4 polynomial on chip), plain stages
def test_rk4_c64(ctqw, flags):
    w = cw.get("bosons_small").with_(R=2, n_steps=100, obs_every=25)
    got = ctqw.run_workload(w, method=ctqw.RK4, flags=flags)
    ref = oracle.ensemble_run(w, method="rk4")
    _compare(got, ref, TOL_FP32, TOL_NORM_DRIFT, energy_tol(w))


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("dtype,flags", [(cw.C128, 1), (cw.C64, 0)])
def test_zero_steps_samples_initial_state(ctqw, dtype, flags):
    w = cw.get("bosons_small").with_(R=2, n_steps=0, obs_every=5)
    got = ctqw.run_workload(w, dtype=dtype, flags=flags)
    ref = oracle.ensemble_run(w)
    assert got["P_mean"].shape == (1, w.N)
    _compare(got, ref, 1e-7 if dtype == cw.C64 else 1e-15, 1e-7, 1e-5)


def test_no_observables(ctqw):
    w = cw.get("bosons_small").with_(R=2, n_steps=10, obs_every=0)
    got = ctqw.run_workload(w)
    assert got["P_mean"] is None
    ref = oracle.ensemble_run(w.with_(obs_every=10))
    P = per_realization_P(got["psi"], got["st_off"], got["sizes"], 2)
    assert np.max(np.abs(P[0] - ref["P"][0][-1])) < TOL_FP32


def test_two_site_lattice_and_single_realization(ctqw):
    w = cw.Workload(name="tiny", m=2, statistics=cw.BOSONS, periodic=False, N=2, R=1, J0=0.9,
                    U=2.3, eps_halfwidth=0.0, J_halfwidth=0.0, sites=(0, 0), dt=0.01, K=16,
                    n_steps=310, obs_every=310, dtype=cw.C128)
    got = ctqw.run_workload(w)
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP64, 1e-12, 1e-11)


def test_ensemble_observables_pair_distribution(ctqw):
    w = cw.get("ragged_n128_1024").with_(ragged_sizes=(5, 8), R=5, n_steps=20, obs_every=20,
                                         dtype=cw.C128, K=10)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C128)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C128)
    ws = h.workspace(cw.C128)
    ctqw.ctqw_propagate_taylor(h, psi, cw.C128, w.dt, w.K, w.n_steps, 0, workspace=ws)
    joint = torch.empty(int(sum(int(g) ** 2 for g in h.group_sizes)), dtype=torch.float64,
                        device="cuda")
    P = torch.empty(h.p_width, dtype=torch.float64, device="cuda")
    ctqw.ctqw_ensemble_observables(h, psi, cw.C128, P_mean=P, P_joint=joint)
    ref = oracle.ensemble_run(w)
    off = 0
    joint = joint.cpu().numpy()
    for g in ref["groups"]:
        members = [k for k in range(w.R) if ref["sizes"][k] == g]
        expect = sum(oracle.pair_correlation(ref["psi"][k], g) for k in members) / len(members)
        np.testing.assert_allclose(joint[off:off + g * g].reshape(g, g), expect, atol=1e-13)
        off += g * g
    np.testing.assert_allclose(P.cpu().numpy(), ref["P_mean"][-1], atol=1e-13)
    h.close()


def test_bad_arguments_rejected(ctqw):
    w = cw.get("bosons_small").with_(R=1)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C128)
    with pytest.raises(ctqw.CtqwError, match="workspace"):
        ctqw.ctqw_propagate_taylor(h, psi, cw.C128, 0.01, 4, 1, 0)
    for K in (-1, 31):   # K = 0 asks for the autotuned order
        with pytest.raises(ctqw.CtqwError, match="K must be"):
            ctqw.ctqw_propagate_taylor(h, psi, cw.C128, 0.01, K, 1, 0, workspace=h.workspace(cw.C128))
    with pytest.raises(ctqw.CtqwError, match="dt"):
        ctqw.ctqw_propagate_taylor(h, psi, cw.C128, float("nan"), 4, 1, 0, workspace=h.workspace(cw.C128))
    h.close()


# ------------------------------------------------------------------ fused shapes and failure path
@pytest.mark.parametrize("N,shape", [(N, k) for N in (64, 128, 192, 256) for k in (1, 2, 4, 5, 6)])
def test_fused_c64_alternative_shapes(ctqw, N, shape):
    w = cw.get("bosons_n256_u2").with_(N=N, R=3, K=9, n_steps=12, obs_every=4,
                                       sites=(N // 2 - 1, N // 2))
    got = ctqw.run_workload(w, flags=ctqw.FUSED_SHAPE(shape))
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP32, TOL_NORM_DRIFT, energy_tol(w))


@pytest.mark.parametrize("k", [3, 7])   # no compiled shape at these indices
def test_fused_unknown_shape_rejected(ctqw, k):
    w = cw.get("bosons_small").with_(R=1, n_steps=2)
    with pytest.raises(ctqw.CtqwError, match="shape"):
        ctqw.run_workload(w, flags=ctqw.FUSED_SHAPE(k))


def test_fused_bounded_wait_gives_up_and_reports(ctqw):
    """The failure path of the fused kernel's bounded waits: with the test flag
    one thread waits on an mbarrier that nothing completes; it must give up
    (1 ms), flag the handle, and leave the GPU and the results usable."""
    w = cw.get("bosons_small").with_(R=2, n_steps=20, obs_every=10)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C64)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C64)
    ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, w.n_steps, 0,
                               flags=ctqw.FLAG_TEST_WAIT_TIMEOUT)
    with pytest.raises(ctqw.CtqwError) as ei:
        ctqw.ctqw_check_status(h)
    assert ei.value.status == ctqw.CTQW_ETIMEOUT
    ctqw.ctqw_check_status(h)          # the flag is cleared once reported
    got = ctqw.run_workload(w)         # and the device keeps working
    ref = oracle.ensemble_run(w)
    _compare(got, ref, TOL_FP32, TOL_NORM_DRIFT, energy_tol(w))
    h.close()


def test_fused_propagation_replays_from_a_cuda_graph(ctqw):
    """init + fused propagation captured once in a CUDA graph and replayed:
    identical results to eager calls (no host synchronisation or allocation
    inside the fused path)."""
    w = cw.get("bosons_n256_u2").with_(N=128, R=4, n_steps=30, obs_every=10, sites=(63, 64))
    h = ctqw.build_for_workload(w)
    sites = ctqw.initial_sites(w, h)
    n_obs = h.n_obs(w.n_steps, w.obs_every)

    def buffers():
        return (h.new_state(cw.C64),
                torch.empty((n_obs, h.p_width), dtype=torch.float64, device="cuda"),
                torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda"),
                torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda"))

    psi, P, nr, en = buffers()
    ctqw.ctqw_init_state(h, psi, sites, cw.C64)
    ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en)
    torch.cuda.synchronize()
    ref = [t.clone() for t in (psi, P, nr, en)]

    gpsi, gP, gnr, gen = buffers()
    ctqw.ctqw_init_state(h, gpsi, sites, cw.C64)   # first call outside capture (sites upload)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctqw.ctqw_propagate_taylor(h, gpsi, cw.C64, w.dt, w.K, w.n_steps, w.obs_every, gP, gnr, gen,
                                   stream=s)
    for _ in range(2):
        ctqw.ctqw_init_state(h, gpsi, sites, cw.C64)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(gpsi, ref[0])   # the state involves no atomics: bit-identical
        for a, b in zip((gP, gnr, gen), ref[1:]):   # FP64 atomics: summation order may differ
            assert torch.allclose(a, b, rtol=0, atol=1e-13)
    ctqw.ctqw_check_status(h)
    h.close()
