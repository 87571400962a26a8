"""Failure detection on the GPU path, with every failure made on the host
(no GPU fault, trap or hang): the norm check fed a NaN disorder value or an
impossible drift tolerance, and device allocations that a test hook makes
fail.  The bounded mbarrier wait of the fused kernel is covered in
test_gpu_parity.py."""
import numpy as np
import pytest

import ctqw_workloads as cw

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


def _handle_with_nan(ctqw, w, bad_r, bad_site):
    """The workload's Hamiltonians with the on-site draw of one site of one
    realization replaced by NaN on the host."""
    u_eps, u_J, sizes, offs = cw.packed_draws(w)
    u_eps = u_eps.copy()
    u_eps[offs[bad_r] + bad_site] = np.nan
    return ctqw.Hamiltonian(w.m, w.statistics, w.periodic, sizes, w.J0, w.U, w.eps_halfwidth,
                            w.J_halfwidth, u_eps, u_J)


def _run(ctqw, h, w, dtype, flags=0, obs_every=None):
    obs_every = w.obs_every if obs_every is None else obs_every
    psi = h.new_state(dtype)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), dtype)
    n_obs = h.n_obs(w.n_steps, obs_every)
    norm = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    ctqw.ctqw_propagate_taylor(h, psi, dtype, w.dt, w.K, w.n_steps, obs_every, None, norm, None, flags,
                               h.workspace(dtype))
    return norm


@pytest.mark.parametrize("dtype,flags", [(cw.C64, 0), (cw.C64, 1), (cw.C128, 0)])
def test_norm_check_names_the_realization_with_a_nan_parameter(ctqw, dtype, flags):
    w = cw.get("bosons_small").with_(R=5, n_steps=30, obs_every=10)
    h = _handle_with_nan(ctqw, w, bad_r=3, bad_site=17)
    eps, _ = h.params()
    assert np.isnan(eps[3 * w.N + 17]) and np.isfinite(np.delete(eps, 3 * w.N + 17)).all()
    norm = _run(ctqw, h, w, dtype, flags).cpu().numpy()
    with pytest.raises(ctqw.CtqwError) as e:
        ctqw.ctqw_check_status(h)
    assert e.value.status == ctqw.CTQW_ENORM
    # the state was finite at step 0, NaN from the first propagated sample on
    assert "realization 3, sample 1" in str(e.value) and "not finite" in str(e.value)
    assert np.isfinite(norm[0]).all() and np.isnan(norm[1:, 3]).all()
    assert np.isfinite(np.delete(norm, 3, axis=1)).all()
    ctqw.ctqw_check_status(h)   # reported once, then clear
    h.close()


def test_norm_check_drift_tolerance(ctqw):
    w = cw.get("bosons_small").with_(R=3, n_steps=60, obs_every=20)
    h = ctqw.build_for_workload(w)
    # FP32 propagation moves the norm by ~1e-7: a bar of 1e-15 fails on the
    # first propagated sample of realization 0, a bar of 1e-5 passes
    ctqw.ctqw_set_norm_check(h, 1e-15)
    _run(ctqw, h, w, cw.C64)
    with pytest.raises(ctqw.CtqwError) as e:
        ctqw.ctqw_check_status(h)
    assert e.value.status == ctqw.CTQW_ENORM and "realization 0, sample 1" in str(e.value)
    assert "drifted" in str(e.value)
    ctqw.ctqw_set_norm_check(h, 1e-5)
    _run(ctqw, h, w, cw.C64)
    ctqw.ctqw_check_status(h)
    with pytest.raises(ctqw.CtqwError) as e:
        ctqw.ctqw_set_norm_check(h, -1.0)
    assert e.value.status == ctqw.CTQW_EINVAL
    h.close()


def test_injected_allocation_failures_give_enomem_and_leave_the_library_usable(ctqw):
    w = cw.get("bosons_small").with_(R=2, n_steps=20, obs_every=10)
    u_eps, u_J, sizes, _ = cw.packed_draws(w)
    args = (w.m, w.statistics, w.periodic, sizes, w.J0, w.U, w.eps_halfwidth, w.J_halfwidth, u_eps, u_J)
    try:
        # every allocation of the build in turn (17 of them, fewer never reach the end)
        failed = 0
        for after in range(40):
            ctqw.ctqw_inject_alloc_failure(after)
            try:
                h = ctqw.Hamiltonian(*args)
            except ctqw.CtqwError as e:
                assert e.status == ctqw.CTQW_ENOMEM, str(e)
                failed += 1
                continue
            h.close()
            break
        assert failed >= 10
        # the fused path allocates its workspace when given none: that allocation fails cleanly
        ctqw.ctqw_inject_alloc_failure(-1)
        h = ctqw.Hamiltonian(*args)
        psi = h.new_state(cw.C64)
        ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C64)
        ctqw.ctqw_inject_alloc_failure(0)
        with pytest.raises(ctqw.CtqwError) as e:
            ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, w.n_steps, 0)
        assert e.value.status == ctqw.CTQW_ENOMEM
        # and the same call succeeds once the injection is off
        ctqw.ctqw_inject_alloc_failure(-1)
        ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, w.n_steps, 0)
        ctqw.ctqw_check_status(h)
        assert torch.isfinite(torch.view_as_real(psi)).all()
        h.close()
    finally:
        ctqw.ctqw_inject_alloc_failure(-1)
