"""Autotuning: the Taylor order from the truncation bound (K = 0) and the
kernel shape by timing the compiled candidates, through the C ABI."""
import json

import numpy as np
import pytest

import ctqw_workloads as cw
import oracle
from gpu_helpers import TOL_FP32, TOL_NORM_DRIFT

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


def test_autotuned_order_matches_the_oracle_bound(ctqw):
    w = cw.get("ragged_n128_1024").with_(R=6)
    h = ctqw.build_for_workload(w)
    # the descriptor bounds |eps| <= 1, J <= 1.25, U = 1
    h_dt = oracle.hamiltonian_norm_bound(2, w.eps_halfwidth, w.J0 + w.J_halfwidth, w.U) * w.dt
    want = ctqw.ctqw_taylor_order(h_dt * (1 + 1e-6), w.n_steps, 2e-6, 8, 20)[0]
    assert ctqw.ctqw_autotune_order(h, cw.C64, w.dt, w.n_steps, 8, 20) == want == 8
    h.close()


def test_order_zero_runs_the_autotuned_order(ctqw):
    w = cw.get("bosons_small").with_(R=2, n_steps=30, obs_every=10)
    h = ctqw.build_for_workload(w)
    K = ctqw.ctqw_autotune_order(h, cw.C64, w.dt, w.n_steps)
    h.close()
    a = ctqw.run_workload(w, K=0)
    b = ctqw.run_workload(w, K=K)
    assert np.array_equal(a["psi"], b["psi"])
    # the fused kernel sums P(x) within a realization with FP32 shared-memory
    # atomics (the ensemble average in FP64): equal up to their order
    assert np.max(np.abs(a["P_mean"] - b["P_mean"])) <= 1e-7
    ref = oracle.ensemble_run(w.with_(K=K))
    assert np.max(np.abs(a["P_mean"] - ref["P_mean"])) <= TOL_FP32


def _handle_and_state(ctqw, w):
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C64)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C64)
    return h, psi


def test_shape_autotuner_times_candidates_and_caches(ctqw, tmp_path, monkeypatch):
    from paper_1612_00746_gb300 import autotune

    w = cw.get("bosons_n256_u2").with_(R=32, n_steps=8)
    h, psi = _handle_and_state(ctqw, w)
    before = psi.clone()
    timings = autotune.time_candidates(h, psi, cw.C64, w.dt, w.K, steps=2)
    names = {f for f, _ in timings}
    # N = 256: three full-row shapes, the banded kernel, the wavefront and the per-term path
    assert ctqw.FUSED_SHAPE(0) in names and ctqw.FLAG_WAVEFRONT in names and ctqw.FLAG_PLAIN in names
    assert all(ms > 0 for _, ms in timings)
    assert torch.equal(psi, before)   # the tuner works on a scratch copy
    cache = str(tmp_path / "tune.json")
    flags = autotune.tuned_flags(h, psi, cw.C64, w.dt, w.K, steps=2, cache_path=cache)
    assert flags in names
    # a second request comes from the cache, without timing anything
    monkeypatch.setattr(autotune, "time_candidates", lambda *a, **k: pytest.fail("re-timed"))
    assert autotune.tuned_flags(h, psi, cw.C64, w.dt, w.K, cache_path=cache) == flags
    h.close()


def test_shape_autotuner_on_a_ragged_batch(ctqw, tmp_path):
    from paper_1612_00746_gb300 import autotune

    w = cw.get("ragged_n128_1024").with_(R=10, ragged_sizes=(64, 128, 192, 256), n_steps=20,
                                         obs_every=10)
    h, psi = _handle_and_state(ctqw, w)
    timings = dict(autotune.time_candidates(h, psi, cw.C64, w.dt, w.K, steps=2))
    assert ctqw.FLAG_WAVEFRONT in timings and ctqw.FLAG_PLAIN in timings
    flags = autotune.tuned_flags(h, psi, cw.C64, w.dt, w.K, steps=2, cache_path=str(tmp_path / "t.json"))
    h.close()
    got = ctqw.run_workload(w, flags=flags)
    ref = oracle.ensemble_run(w)
    assert np.max(np.abs(got["P_mean"] - ref["P_mean"])) <= TOL_FP32
    assert np.max(np.abs(got["norm"] - ref["norm"].T)) <= TOL_NORM_DRIFT


def test_order_and_shape_for_a_ragged_batch(ctqw, tmp_path):
    """tune() on a ragged batch: K is the bound's order over 8..20 and the
    flags the fastest timed candidate; propagating with the pair matches
    the oracle."""
    import oracle
    from gpu_helpers import TOL_FP32
    from paper_1612_00746_gb300 import autotune

    w = cw.get("ragged_n128_1024").with_(R=5, ragged_sizes=(40, 72, 96), n_steps=40, obs_every=20)
    h = ctqw.build_for_workload(w)
    psi = h.new_state(cw.C64)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C64)
    K, flags = autotune.tune(h, psi, cw.C64, w.dt, w.n_steps, 8, 20, steps=2,
                             cache_path=str(tmp_path / "c.json"))
    assert K == ctqw.ctqw_autotune_order(h, cw.C64, w.dt, w.n_steps, 8, 20)
    assert 8 <= K <= 20
    timed = json.load(open(tmp_path / "c.json"))
    entry = next(iter(timed.values()))
    assert int(entry["flags"]) == flags
    assert entry["ms_per_step"] == min(entry["timings"].values())
    n_obs = h.n_obs(w.n_steps, w.obs_every)
    P = torch.empty((n_obs, h.p_width), dtype=torch.float64, device="cuda")
    ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, K, w.n_steps, w.obs_every, P, None, None, flags,
                               h.workspace(cw.C64, ctqw.TAYLOR, flags))
    ctqw.ctqw_check_status(h)
    ref = oracle.ensemble_run(w, K=K)
    assert np.max(np.abs(P.cpu().numpy() - ref["P_mean"])) <= TOL_FP32
    h.close()


def test_per_term_ragged_propagation_replays_from_a_cuda_graph(ctqw):
    """The whole per-term propagation of a ragged batch (one launch per stage
    and size group) captured once and replayed."""
    w = cw.get("ragged_n128_1024").with_(R=5, ragged_sizes=(96, 160, 200), n_steps=12, obs_every=4)
    h = ctqw.build_for_workload(w)
    sites = ctqw.initial_sites(w, h)
    psi = h.new_state(cw.C64)
    n_obs = h.n_obs(w.n_steps, w.obs_every)
    P = torch.empty((n_obs, h.p_width), dtype=torch.float64, device="cuda")
    nr = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    en = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    ws = h.workspace(cw.C64, ctqw.TAYLOR, ctqw.FLAG_PLAIN)
    ctqw.ctqw_init_state(h, psi, sites, cw.C64)
    psi0 = psi.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en,
                                       ctqw.FLAG_PLAIN, ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    psi.copy_(psi0)
    g.replay()
    torch.cuda.synchronize()
    P1 = P.cpu().numpy()
    ref = oracle.ensemble_run(w)
    assert np.max(np.abs(P1 - ref["P_mean"])) <= TOL_FP32
    psi.copy_(psi0)
    g.replay()
    torch.cuda.synchronize()
    assert np.max(np.abs(P.cpu().numpy() - P1)) <= 1e-14   # FP64 atomics: order of additions
    h.close()


def test_tiled_default_propagation_replays_from_a_cuda_graph(ctqw):
    """The default path for a ragged batch beyond the fused sizes (register
    tiles, one launch per size group and stage group) captured and replayed."""
    w = cw.get("ragged_n128_1024").with_(R=4, ragged_sizes=(300, 420), n_steps=6, obs_every=3)
    h = ctqw.build_for_workload(w)
    sites = ctqw.initial_sites(w, h)
    psi = h.new_state(cw.C64)
    n_obs = h.n_obs(w.n_steps, w.obs_every)
    P = torch.empty((n_obs, h.p_width), dtype=torch.float64, device="cuda")
    nr = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    en = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    ws = h.workspace(cw.C64)
    ctqw.ctqw_init_state(h, psi, sites, cw.C64)
    psi0 = psi.clone()
    # eager run first (also the first use of every kernel)
    ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en, 0, ws)
    torch.cuda.synchronize()
    P_eager, psi_eager = P.cpu().numpy(), psi.cpu().numpy()
    psi.copy_(psi0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en,
                                       0, ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    psi.copy_(psi0)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(psi.cpu().numpy(), psi_eager)
    assert np.max(np.abs(P.cpu().numpy() - P_eager)) <= 1e-14
    ref = oracle.ensemble_run(w)
    assert np.max(np.abs(P.cpu().numpy() - ref["P_mean"])) <= TOL_FP32
    h.close()
