"""The fused path's second stream (ctqw_fused_split): while the 16-CTA
clusters run most realizations, the last ones run on the register tiles, on
the SMs that no cluster can hold.  Both parts against the FP64 oracle, the
ensemble mean against the per-realization states, the two-stream run against
the one-stream run, and the call replayed from a CUDA graph."""
import numpy as np
import pytest

import ctqw_workloads as cw
import oracle
from gpu_helpers import TOL_FP32, TOL_NORM_DRIFT, energy_tol, oracle_params, per_realization_P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# two bosons with U = 2 on N = 256: 64 realizations are several rounds of the
# resident clusters, so a share goes to the second stream
W = cw.get("bosons_n256_u2").with_(R=64, n_steps=30, obs_every=10)


@pytest.fixture(scope="module")
def ctqw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_00746_gb300 import build, ctqw as c

    build.build()
    c.load()
    return c


def _split(ctqw, w, K=None, flags=0):
    h = ctqw.build_for_workload(w)
    try:
        return ctqw.ctqw_fused_split(h, w.K if K is None else K, flags)
    finally:
        h.close()


def _oracle_run(w, r, method="taylor"):
    (eps, Jp), = oracle_params(w, [r])
    J = Jp if w.periodic else Jp[:w.N - 1]
    H = oracle.many_particle_hamiltonian(oracle.single_particle_hamiltonian(eps, J, w.periodic), w.m, w.U)
    psi0 = oracle.initial_state(w.N, w.m, w.initial_sites(w.N), w.statistics)
    return oracle.propagate(H, psi0, w.N, w.m, w.dt, w.n_steps, w.obs_every, method=method, K=w.K)


def test_split_is_planned_only_where_it_applies(ctqw):
    R_t = _split(ctqw, W)
    assert 0 < R_t < W.R // 2
    assert _split(ctqw, W, flags=ctqw.FLAG_ONE_STREAM) == 0
    assert _split(ctqw, W, flags=ctqw.FLAG_PLAIN) == 0
    assert _split(ctqw, W, flags=ctqw.FUSED_SHAPE(1)) == 0
    # one round of clusters or less: nothing to share
    assert _split(ctqw, W.with_(R=4)) == 0
    # N = 64 takes one CTA per cluster, which packs every SM
    assert _split(ctqw, W.with_(N=64)) == 0
    # the full bench size splits too, at RK4's order as well
    assert _split(ctqw, W.with_(R=1024)) > 0
    assert _split(ctqw, W.with_(R=1024), K=4) > 0


@pytest.fixture(scope="module")
def two_streams(ctqw):
    return _split(ctqw, W), ctqw.run_workload(W)


def test_both_parts_match_the_oracle(ctqw, two_streams):
    R_t, got = two_streams
    R_f = W.R - R_t
    P_final = per_realization_P(got["psi"], got["st_off"], got["sizes"], W.m)
    for r in (0, R_f - 1, R_f, W.R - 1):   # first and last of each part
        ref = _oracle_run(W, r)
        assert np.max(np.abs(P_final[r] - ref["P"][-1])) <= TOL_FP32, r
        assert np.max(np.abs(got["norm"][:, r] - ref["norm"])) <= TOL_NORM_DRIFT, r
        assert np.max(np.abs(got["energy"][:, r] - ref["energy"])) <= energy_tol(W), r


def test_the_mean_holds_both_parts(two_streams):
    """P_mean of the last sample is the mean of every realization's P of the
    returned states, and each sample's P_mean sums to the mean norm.  The GPU
    forms every |psi|^2 in FP32 (two roundings, each at most 2^-24 of the
    product) and sums the products exactly in units of 2^-48 (each rounded by
    at most 2^-49); the host squares in FP64.  P(x) holds N^(m-1) products
    per particle, weighted 1/m, so the two agree to 2^-23 P(x) + N^(m-1) 2^-49."""
    _, got = two_streams
    P_final = np.mean(per_realization_P(got["psi"], got["st_off"], got["sizes"], W.m), axis=0)
    tol = 2.0 ** -23 * P_final + W.N ** (W.m - 1) * 2.0 ** -49
    assert np.all(np.abs(got["P_mean"][-1] - P_final) <= tol)
    np.testing.assert_allclose(got["P_mean"].sum(axis=1), got["norm"].mean(axis=1), atol=1e-12)


def test_two_streams_match_one_stream(ctqw, two_streams):
    """The clusters' realizations come out bit for bit as in the one-stream
    run (the same kernel on the same inputs); the tiles' agree to FP32."""
    R_t, got = two_streams
    R_f = W.R - R_t
    one = ctqw.run_workload(W, flags=ctqw.FLAG_ONE_STREAM)
    cut = int(got["st_off"][R_f])
    assert np.array_equal(got["psi"][:cut], one["psi"][:cut])
    assert np.max(np.abs(got["psi"][cut:] - one["psi"][cut:])) <= 1e-5
    assert np.max(np.abs(got["norm"][:, :R_f] - one["norm"][:, :R_f])) <= 1e-14   # FP64 atomics
    assert np.max(np.abs(got["norm"] - one["norm"])) <= TOL_NORM_DRIFT
    assert np.max(np.abs(got["P_mean"] - one["P_mean"])) <= TOL_FP32


def test_rk4_splits_at_order_four(ctqw):
    """RK4 on the fused sizes is the order-4 Taylor polynomial (Sec. 2.3);
    its split runs the tiles at K = 4."""
    w = W.with_(n_steps=20)
    got = ctqw.run_workload(w, method=ctqw.RK4)
    R_t = _split(ctqw, w, K=4)
    assert R_t > 0
    P_final = per_realization_P(got["psi"], got["st_off"], got["sizes"], w.m)
    for r in (0, w.R - 1):
        ref = _oracle_run(w, r, method="rk4")
        assert np.max(np.abs(P_final[r] - ref["P"][-1])) <= TOL_FP32, r
        assert np.max(np.abs(got["norm"][:, r] - ref["norm"])) <= TOL_NORM_DRIFT, r


def test_degenerate_calls_with_a_split(ctqw):
    """No steps: the samples are those of the initial state and psi is
    unchanged; no observables: psi as with them."""
    z = ctqw.run_workload(W, n_steps=0)
    assert z["P_mean"].shape[0] == 1
    assert np.max(np.abs(z["norm"] - 1.0)) <= 1e-6
    init = ctqw.build_for_workload(W)
    psi0 = init.new_state(cw.C64)
    ctqw.ctqw_init_state(init, psi0, ctqw.initial_sites(W, init), cw.C64)
    assert np.array_equal(z["psi"], psi0.cpu().numpy())
    init.close()
    a = ctqw.run_workload(W, n_steps=12, obs_every=0)
    b = ctqw.run_workload(W, n_steps=12, obs_every=4)
    assert a["P_mean"] is None or a["P_mean"].size == 0
    assert np.array_equal(a["psi"], b["psi"])


def test_split_call_replays_from_a_cuda_graph(ctqw):
    """The fork to the side stream and the join back are captured with the
    call: the replay gives the eager result."""
    w = W.with_(n_steps=12, obs_every=4)
    h = ctqw.build_for_workload(w)
    assert ctqw.ctqw_fused_split(h, w.K) > 0
    sites = ctqw.initial_sites(w, h)
    psi = h.new_state(cw.C64)
    n_obs = h.n_obs(w.n_steps, w.obs_every)
    P = torch.empty((n_obs, h.p_width), dtype=torch.float64, device="cuda")
    nr = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    en = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    ws = h.workspace(cw.C64)
    ctqw.ctqw_init_state(h, psi, sites, cw.C64)
    psi0 = psi.clone()
    ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en, 0, ws)
    torch.cuda.synchronize()
    eager = (psi.cpu().numpy(), P.cpu().numpy(), nr.cpu().numpy(), en.cpu().numpy())
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en, 0, ws,
                                       stream=s)
    torch.cuda.current_stream().wait_stream(s)
    psi.copy_(psi0)
    g.replay()
    torch.cuda.synchronize()
    ctqw.ctqw_check_status(h)
    assert np.array_equal(psi.cpu().numpy(), eager[0])
    assert np.max(np.abs(P.cpu().numpy() - eager[1])) <= 1e-14   # FP64 atomics: order of additions
    assert np.max(np.abs(nr.cpu().numpy() - eager[2])) <= 1e-14
    assert np.max(np.abs(en.cpu().numpy() - eager[3])) <= 1e-12
    h.close()
