"""The ensemble-averaged one-body density matrix (ctqw_one_body_density)
against the FP64 oracle, through the C ABI: on the GPU's own final states
(the contraction alone, exact inputs) and along the whole pipeline against
oracle-propagated states; two and three particles, ragged groups, FP32 and
FP64; diagonal against P_mean, trace against the norm."""
import numpy as np
import pytest

import ctqw_workloads as cw
import oracle
from gpu_helpers import TOL_FP32, TOL_TC

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


def _run(ctqw, w, dtype):
    h = ctqw.build_for_workload(w)
    psi = h.new_state(dtype)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), dtype)
    n_obs = h.n_obs(w.n_steps, w.obs_every)
    P = torch.empty((n_obs, h.p_width), dtype=torch.float64, device="cuda")
    nr = torch.empty((n_obs, h.R), dtype=torch.float64, device="cuda")
    ws = h.workspace(dtype)
    ctqw.ctqw_propagate_taylor(h, psi, dtype, w.dt, w.K, w.n_steps, w.obs_every, P, nr, None, 0, ws)
    rho = [r.cpu().numpy() for r in ctqw.ctqw_one_body_density(h, psi, dtype)]
    out = {"rho": rho, "psi": psi.cpu().numpy(), "P": P.cpu().numpy(), "norm": nr.cpu().numpy(),
           "sizes": h.sizes.copy(), "st_off": h.st_off.copy(), "groups": [int(n) for n in h.group_sizes]}
    h.close()
    return out


def _oracle_rho_from(psi_flat, st_off, sizes, groups, m):
    """Oracle rho1 per size group from given states (FP64 arithmetic)."""
    out = []
    for N in groups:
        members = [r for r in range(len(sizes)) if sizes[r] == N]
        acc = np.zeros((N, N), dtype=np.complex128)
        for r in members:
            acc += oracle.one_body_density(psi_flat[st_off[r]:st_off[r + 1]].astype(np.complex128), N, m)
        out.append(acc / len(members))
    return out


@pytest.mark.parametrize("name,kw,dtype,tol", [
    ("bosons_small", {"R": 6, "n_steps": 30, "obs_every": 30}, cw.C64, 2e-6),
    ("fp64_plain_small", {"n_steps": 30, "obs_every": 30}, cw.C128, 1e-13),
    ("ring3_small", {"R": 3, "n_steps": 20, "obs_every": 20}, cw.C64, 2e-6),
    ("ragged_n128_1024", {"R": 7, "ragged_sizes": (40, 70, 100), "n_steps": 10, "obs_every": 10},
     cw.C64, 2e-6),
])
def test_contraction_against_oracle_on_the_same_states(ctqw, name, kw, dtype, tol):
    w = cw.get(name).with_(**kw)
    got = _run(ctqw, w, dtype)
    ref = _oracle_rho_from(got["psi"], got["st_off"], got["sizes"], got["groups"], w.m)
    for g, (a, b) in enumerate(zip(got["rho"], ref)):
        scale = np.max(np.abs(b))
        assert np.max(np.abs(a - b)) <= tol * scale, (g, np.max(np.abs(a - b)), scale)
        assert np.max(np.abs(a - a.conj().T)) <= tol * scale
    # diagonal = P_mean of the last sample, trace = mean norm
    off = 0
    for g, (a, N) in enumerate(zip(got["rho"], got["groups"])):
        members = got["sizes"] == N
        assert np.max(np.abs(np.diag(a).real - got["P"][-1][off:off + N])) <= 10 * tol
        assert abs(np.trace(a).real - got["norm"][-1][members].mean()) <= 10 * tol * N
        off += N


def test_pipeline_against_oracle_propagation(ctqw):
    w = cw.get("bosons_small").with_(R=4, n_steps=60, obs_every=60)
    got = _run(ctqw, w, cw.C64)
    N = w.N
    res = oracle.ensemble_run(w)
    ref = sum(oracle.one_body_density(p, N, w.m) for p in res["psi"]) / w.R
    assert np.max(np.abs(got["rho"][0] - ref)) <= TOL_FP32


def test_null_arguments_rejected(ctqw):
    w = cw.get("bosons_small").with_(R=1)
    h = ctqw.build_for_workload(w)
    lib = ctqw.load()
    assert lib.ctqw_one_body_density(h.handle, cw.C64, None, None, None) == ctqw.CTQW_EINVAL
    h.close()


@pytest.mark.parametrize("name,kw", [
    ("bosons_small", {"R": 6, "n_steps": 30, "obs_every": 30}),                            # N = 64
    ("bosons_small", {"N": 144, "R": 3, "sites": (71, 72), "n_steps": 20, "obs_every": 20}),  # two tile rows, ragged tail
    ("bosons_small", {"N": 16, "R": 5, "sites": (7, 8), "n_steps": 20, "obs_every": 20}),   # one small tile
    ("ring3_small", {"N": 16, "R": 3, "sites": (7, 8, 9), "n_steps": 15, "obs_every": 15}),  # m = 3 (k blocks of 256)
    ("ragged_n128_1024", {"R": 9, "ragged_sizes": (32, 48, 80, 272), "n_steps": 8, "obs_every": 8}),
])
def test_tensor_cores_against_oracle_and_cuda_cores(ctqw, name, kw):
    """The tcgen05 path (TF32, three piece products, FP32 partials over at
    most 256 k, two-word totals) against the oracle on the same final states
    and against the CUDA-core kernel, at the bound of its FP32 partial
    sums (TOL_TC); the CUDA-core kernel at the FP32 tolerance."""
    w = cw.get(name).with_(**kw)
    h = ctqw.build_for_workload(w)
    assert all(int(n) % 16 == 0 for n in h.group_sizes)
    psi = h.new_state(cw.C64)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), cw.C64)
    ctqw.ctqw_propagate_taylor(h, psi, cw.C64, w.dt, w.K, w.n_steps, 0, None, None, None, 0,
                               h.workspace(cw.C64))
    ctqw.ctqw_set_density_method(h, 0)
    tc = [r.cpu().numpy() for r in ctqw.ctqw_one_body_density(h, psi, cw.C64)]
    ctqw.ctqw_check_status(h)
    ctqw.ctqw_set_density_method(h, 1)
    cc = [r.cpu().numpy() for r in ctqw.ctqw_one_body_density(h, psi, cw.C64)]
    ref = _oracle_rho_from(psi.cpu().numpy(), h.st_off, h.sizes, [int(n) for n in h.group_sizes], w.m)
    for a, c, b in zip(tc, cc, ref):
        scale = np.max(np.abs(b))
        assert np.max(np.abs(c - b)) <= TOL_FP32 * scale   # the CUDA cores (FP64 sums)
        assert np.max(np.abs(a - b)) <= TOL_TC * scale, np.max(np.abs(a - b)) / scale
        assert np.max(np.abs(a - c)) <= TOL_TC * scale
        assert np.max(np.abs(a - a.conj().T)) <= TOL_TC * scale
    with pytest.raises(ctqw.CtqwError):
        ctqw.ctqw_set_density_method(h, 2)
    h.close()


def test_tensor_cores_at_the_largest_size(ctqw):
    """N = 2048, the largest size of the tcgen05 path (16 x 16 tiles, 136 of
    them computed), on a dense seeded random state, against the oracle at
    the bound of the FP32 partial sums (TOL_TC): every block of 256 k then
    carries terms of one size, the case that shows the accumulation's
    rounding most."""
    w = cw.get("bosons_small").with_(N=2048, R=1, statistics=cw.DISTINGUISHABLE, sites=(1000, 1001),
                                     n_steps=1, obs_every=1)
    h = ctqw.build_for_workload(w)
    rng = np.random.default_rng(11)
    v = (rng.standard_normal(2048 * 2048) + 1j * rng.standard_normal(2048 * 2048)).astype(np.complex64)
    v /= np.sqrt(np.sum(np.abs(v.astype(np.complex128)) ** 2))
    psi = h.new_state(cw.C64)
    psi.copy_(torch.from_numpy(v).to(psi.device))
    ctqw.ctqw_set_density_method(h, 0)
    got = ctqw.ctqw_one_body_density(h, psi, cw.C64)[0].cpu().numpy()
    ctqw.ctqw_check_status(h)
    ref = oracle.one_body_density(v.astype(np.complex128), 2048, 2)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= TOL_TC * scale, np.max(np.abs(got - ref)) / scale
    assert np.max(np.abs(got - got.conj().T)) <= TOL_TC * scale
    h.close()
