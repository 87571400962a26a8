"""ctypes binding of libctqw (argument marshalling only).

Every entry point of include/ctqw.h has a function of the same name here;
all compute runs in the CUDA library.  PyTorch provides device memory and
streams.  Loading fails loudly when libctqw.so is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libctqw.so")

CTQW_OK, CTQW_EINVAL, CTQW_ENOMEM, CTQW_ECUDA, CTQW_EUNSUPPORTED = 0, 1, 2, 3, 4
CTQW_ENORM = 5
CTQW_ETIMEOUT = 6
DISTINGUISHABLE, BOSONS, FERMIONS = 0, 1, 2
C64, C128 = 0, 1
FLAG_PLAIN = 0x1
FLAG_NO_COMPENSATION = 0x2
FLAG_RENORMALIZE = 0x4
FLAG_TEST_WAIT_TIMEOUT = 0x8
FLAG_ONE_STREAM = 0x10


def FUSED_SHAPE(k: int) -> int:
    return (int(k) & 0xF) << 8


SHAPE_WAVEFRONT = 8
FLAG_WAVEFRONT = FUSED_SHAPE(SHAPE_WAVEFRONT)   # the row-wavefront kernel


def FLAG_TILED(i: int) -> int:
    """The temporally blocked tiled kernel, shape i: iterate in shared memory
    (0: D = 4), in registers on 64 x 128 regions (1: D = 8), on 96 x 64
    regions (2: D = 8) or on 64 x 64 regions (3: D = 4, 4: D = 8, 5: D = 2,
    6: D = 7)."""
    return FUSED_SHAPE(9 + int(i))

TAYLOR, RK4 = 0, 1

EXPORTED = (
    "ctqw_build_hamiltonian", "ctqw_destroy_hamiltonian", "ctqw_get_params", "ctqw_state_size",
    "ctqw_output_layout", "ctqw_init_state", "ctqw_workspace_size", "ctqw_propagate_taylor",
    "ctqw_propagate_rk4", "ctqw_ensemble_observables", "ctqw_check_status", "ctqw_last_error",
    "ctqw_version", "ctqw_adjoint_workspace_size", "ctqw_adjoint_grad", "ctqw_taylor_order",
    "ctqw_autotune_order", "ctqw_one_body_density", "ctqw_propagate_taylor_switching",
    "ctqw_propagate_exact", "ctqw_graph_build", "ctqw_graph_destroy", "ctqw_graph_get_params",
    "ctqw_graph_state_size", "ctqw_graph_init_state", "ctqw_graph_workspace_size",
    "ctqw_graph_propagate_taylor", "ctqw_graph_propagate_rk4", "ctqw_graph_observables",
    "ctqw_graph_set_chunk", "ctqw_set_norm_check", "ctqw_inject_alloc_failure",
    "ctqw_set_density_method", "ctqw_fused_split",
)


class CtqwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libctqw status {status}: {msg}")
        self.status = status


class LatticeDesc(ctypes.Structure):
    _fields_ = [
        ("n_particles", ctypes.c_int32), ("statistics", ctypes.c_int32),
        ("periodic", ctypes.c_int32), ("n_realizations", ctypes.c_int32),
        ("n_sites", ctypes.POINTER(ctypes.c_int32)), ("n_sites_uniform", ctypes.c_int32),
        ("round_to_f32", ctypes.c_int32), ("J0", ctypes.c_double), ("U", ctypes.c_double),
        ("eps_halfwidth", ctypes.c_double), ("J_halfwidth", ctypes.c_double),
        ("eps_mean", ctypes.POINTER(ctypes.c_double)), ("J_mean", ctypes.POINTER(ctypes.c_double)),
        ("u_eps_host", ctypes.POINTER(ctypes.c_double)), ("u_J_host", ctypes.POINTER(ctypes.c_double)),
    ]


class GraphDesc(ctypes.Structure):
    _fields_ = [
        ("n_particles", ctypes.c_int32), ("statistics", ctypes.c_int32),
        ("n_nodes", ctypes.c_int32), ("n_edges", ctypes.c_int32),
        ("edge_u", ctypes.POINTER(ctypes.c_int32)), ("edge_v", ctypes.POINTER(ctypes.c_int32)),
        ("n_realizations", ctypes.c_int32), ("round_to_f32", ctypes.c_int32),
        ("J0", ctypes.c_double), ("U", ctypes.c_double),
        ("eps_halfwidth", ctypes.c_double), ("J_halfwidth", ctypes.c_double),
        ("u_eps_host", ctypes.POINTER(ctypes.c_double)), ("u_J_host", ctypes.POINTER(ctypes.c_double)),
    ]


_lib = None


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libctqw.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(p)
    vp, i32, i64, dbl, u32, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                  ctypes.c_uint32, ctypes.c_size_t)
    pd = ctypes.POINTER(ctypes.c_double)
    sig = {
        "ctqw_build_hamiltonian": [ctypes.POINTER(LatticeDesc), vp, ctypes.POINTER(vp)],
        "ctqw_destroy_hamiltonian": [vp],
        "ctqw_get_params": [vp, pd, pd],
        "ctqw_state_size": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)],
        "ctqw_output_layout": [vp, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32),
                               ctypes.POINTER(i32)],
        "ctqw_init_state": [vp, ctypes.POINTER(i32), i32, vp, vp],
        "ctqw_workspace_size": [vp, i32, i32, u32, ctypes.POINTER(sz)],
        "ctqw_propagate_taylor": [vp, i32, vp, dbl, i32, i64, i32, vp, vp, vp, u32, vp, sz, vp],
        "ctqw_propagate_rk4": [vp, i32, vp, dbl, i64, i32, vp, vp, vp, u32, vp, sz, vp],
        "ctqw_ensemble_observables": [vp, i32, vp, vp, vp, vp, vp, vp],
        "ctqw_check_status": [vp, vp],
        "ctqw_set_norm_check": [vp, dbl],
        "ctqw_inject_alloc_failure": [i32],
        "ctqw_set_density_method": [vp, i32],
        "ctqw_fused_split": [vp, i32, u32, ctypes.POINTER(i32)],
        "ctqw_adjoint_workspace_size": [vp, i32, i32, i64, i32, ctypes.POINTER(sz)],
        "ctqw_adjoint_grad": [vp, i32, vp, dbl, i32, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp],
        "ctqw_taylor_order": [dbl, i64, dbl, i32, i32, ctypes.POINTER(i32), pd],
        "ctqw_one_body_density": [vp, i32, vp, vp, vp],
        "ctqw_propagate_exact": [vp, i32, vp, dbl, i64, i32, vp, vp, vp, ctypes.POINTER(i32), vp],
        "ctqw_propagate_taylor_switching": [vp, i32, vp, dbl, i32, i64, i32, vp, vp, vp, u32, vp, sz,
                                            ctypes.c_uint64, dbl, vp],
        "ctqw_autotune_order": [vp, i32, dbl, i64, i32, i32, ctypes.POINTER(i32)],
        "ctqw_graph_build": [ctypes.POINTER(GraphDesc), vp, ctypes.POINTER(vp)],
        "ctqw_graph_destroy": [vp],
        "ctqw_graph_get_params": [vp, pd, pd],
        "ctqw_graph_state_size": [vp, ctypes.POINTER(i64)],
        "ctqw_graph_init_state": [vp, ctypes.POINTER(i32), i32, vp, vp],
        "ctqw_graph_workspace_size": [vp, i32, ctypes.POINTER(sz)],
        "ctqw_graph_propagate_taylor": [vp, i32, vp, dbl, i32, i64, i32, vp, vp, vp, vp, sz, vp],
        "ctqw_graph_propagate_rk4": [vp, i32, vp, dbl, i64, i32, vp, vp, vp, vp, sz, vp],
        "ctqw_graph_observables": [vp, i32, vp, vp, vp, vp, vp],
        "ctqw_graph_set_chunk": [vp, i32],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.ctqw_last_error.restype = ctypes.c_char_p
    lib.ctqw_last_error.argtypes = []
    lib.ctqw_version.restype = ctypes.c_char_p
    lib.ctqw_version.argtypes = []
    _lib = lib
    return lib


def _check(status: int) -> None:
    if status != CTQW_OK:
        raise CtqwError(status, load().ctqw_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def torch_dtype(dtype: int):
    return torch.complex64 if dtype == C64 else torch.complex128


class Hamiltonian:
    """Handle of the stochastic Hamiltonians of all realizations (ctqw_build_hamiltonian)."""

    def __init__(self, m: int, statistics: int, periodic: bool, sizes: Sequence[int], J0: float,
                 U: float, eps_halfwidth: float, J_halfwidth: float, u_eps: np.ndarray,
                 u_J: np.ndarray, eps_mean: Optional[np.ndarray] = None,
                 J_mean: Optional[np.ndarray] = None, round_to_f32: bool = True, stream=None):
        lib = load()
        self.m = int(m)
        self.statistics = int(statistics)
        self.periodic = bool(periodic)
        self.sizes = np.ascontiguousarray(np.asarray(sizes, dtype=np.int32))
        self.R = len(self.sizes)
        self._u_eps = np.ascontiguousarray(u_eps, dtype=np.float64)
        self._u_J = np.ascontiguousarray(u_J, dtype=np.float64)
        self._em = None if eps_mean is None else np.ascontiguousarray(eps_mean, dtype=np.float64)
        self._jm = None if J_mean is None else np.ascontiguousarray(J_mean, dtype=np.float64)
        d = LatticeDesc()
        d.n_particles = self.m
        d.statistics = self.statistics
        d.periodic = 1 if periodic else 0
        d.n_realizations = self.R
        d.n_sites = self.sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.n_sites_uniform = 0
        d.round_to_f32 = 1 if round_to_f32 else 0
        d.J0, d.U = float(J0), float(U)
        d.eps_halfwidth, d.J_halfwidth = float(eps_halfwidth), float(J_halfwidth)
        d.eps_mean = _dptr(self._em)
        d.J_mean = _dptr(self._jm)
        d.u_eps_host = _dptr(self._u_eps)
        d.u_J_host = _dptr(self._u_J)
        h = ctypes.c_void_p()
        _check(lib.ctqw_build_hamiltonian(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
        self._h = h
        total = ctypes.c_int64()
        st_off = np.zeros(self.R + 1, dtype=np.int64)
        _check(lib.ctqw_state_size(h, ctypes.byref(total),
                                   st_off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        self.total_amplitudes = int(total.value)
        self.st_off = st_off
        pw, ng = ctypes.c_int64(), ctypes.c_int32()
        _check(lib.ctqw_output_layout(h, ctypes.byref(pw), ctypes.byref(ng), None, None))
        gs = np.zeros(ng.value, dtype=np.int32)
        gc = np.zeros(ng.value, dtype=np.int32)
        _check(lib.ctqw_output_layout(h, None, None, gs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      gc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        self.p_width = int(pw.value)
        self.group_sizes = gs
        self.group_count = gc

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ctqw_destroy_hamiltonian(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        """(eps, J) host float64 arrays [sum_r N_r] (ctqw_get_params)."""
        n = int(self.sizes.sum())
        eps = np.zeros(n)
        J = np.zeros(n)
        _check(load().ctqw_get_params(self._h, _dptr(eps), _dptr(J)))
        return eps, J

    def new_state(self, dtype: int, device="cuda") -> torch.Tensor:
        return torch.zeros(self.total_amplitudes, dtype=torch_dtype(dtype), device=device)

    def workspace(self, dtype: int, method: int = TAYLOR, flags: int = 0, device="cuda"):
        b = ctypes.c_size_t()
        _check(load().ctqw_workspace_size(self._h, dtype, method, flags, ctypes.byref(b)))
        if b.value == 0:
            return None
        return torch.empty(b.value, dtype=torch.uint8, device=device)

    def n_obs(self, n_steps: int, obs_every: int) -> int:
        return n_steps // obs_every + 1 if obs_every > 0 else 0


class Graph:
    """Handle of m particles on a q-dimensional lattice or general graph with
    per-realization disorder (ctqw_graph_build)."""

    def __init__(self, m: int, statistics: int, n_nodes: int, edge_u, edge_v, R: int, J0: float,
                 U: float, eps_halfwidth: float, J_halfwidth: float, u_eps: np.ndarray,
                 u_J: np.ndarray, round_to_f32: bool = True, stream=None):
        lib = load()
        self.m, self.statistics, self.N, self.R = int(m), int(statistics), int(n_nodes), int(R)
        self._eu = np.ascontiguousarray(np.asarray(edge_u, dtype=np.int32))
        self._ev = np.ascontiguousarray(np.asarray(edge_v, dtype=np.int32))
        self.E = len(self._eu)
        self._u_eps = np.ascontiguousarray(u_eps, dtype=np.float64)
        self._u_J = np.ascontiguousarray(u_J, dtype=np.float64)
        d = GraphDesc()
        d.n_particles, d.statistics, d.n_nodes, d.n_edges = self.m, self.statistics, self.N, self.E
        d.edge_u = self._eu.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.edge_v = self._ev.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.n_realizations = self.R
        d.round_to_f32 = 1 if round_to_f32 else 0
        d.J0, d.U = float(J0), float(U)
        d.eps_halfwidth, d.J_halfwidth = float(eps_halfwidth), float(J_halfwidth)
        d.u_eps_host = _dptr(self._u_eps)
        d.u_J_host = _dptr(self._u_J)
        g = ctypes.c_void_p()
        _check(lib.ctqw_graph_build(ctypes.byref(d), _stream(stream), ctypes.byref(g)))
        self._g = g
        total = ctypes.c_int64()
        _check(lib.ctqw_graph_state_size(g, ctypes.byref(total)))
        self.total_amplitudes = int(total.value)
        self.Rp = (self.R + 3) // 4 * 4
        self.D = self.total_amplitudes // self.Rp

    @classmethod
    def from_workload(cls, w, realizations=None, stream=None) -> "Graph":
        """The handle of a graph workload (its link list and seeded draws)."""
        import ctqw_workloads as cw
        realizations = list(range(w.R)) if realizations is None else list(realizations)
        u, v = w.edges()
        ue, uj = cw.graph_draws(w, realizations)
        return cls(w.m, w.statistics, w.n_nodes(), u, v, len(realizations), w.J0, w.U, w.eps_halfwidth,
                   w.J_halfwidth, ue, uj, stream=stream)

    @property
    def handle(self):
        return self._g

    def close(self) -> None:
        if getattr(self, "_g", None) is not None and self._g.value:
            load().ctqw_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        """(eps [R][N], J [R][E]) host float64 arrays (ctqw_graph_get_params)."""
        eps = np.zeros((self.R, self.N))
        J = np.zeros((self.R, max(self.E, 1)))
        _check(load().ctqw_graph_get_params(self._g, _dptr(eps), _dptr(J)))
        return eps, J[:, :self.E]

    def new_state(self, dtype: int, device="cuda") -> torch.Tensor:
        return torch.zeros(self.total_amplitudes, dtype=torch_dtype(dtype), device=device)

    def workspace(self, dtype: int, device="cuda") -> torch.Tensor:
        b = ctypes.c_size_t()
        _check(load().ctqw_graph_workspace_size(self._g, dtype, ctypes.byref(b)))
        return torch.empty(b.value, dtype=torch.uint8, device=device)

    def n_obs(self, n_steps: int, obs_every: int) -> int:
        return n_steps // obs_every + 1 if obs_every > 0 else 0

    def states(self, psi: torch.Tensor) -> torch.Tensor:
        """[R][N^m] view of a graph state (stored amplitude-major, s Rp + r)."""
        return psi.reshape(self.D, self.Rp)[:, :self.R].t()


def ctqw_graph_set_chunk(g: Graph, realizations: int) -> None:
    _check(load().ctqw_graph_set_chunk(g.handle, int(realizations)))


def ctqw_graph_init_state(g: Graph, psi: torch.Tensor, sites, dtype: int, stream=None) -> None:
    s = np.ascontiguousarray(np.broadcast_to(np.asarray(sites, dtype=np.int32), (g.R, g.m)))
    _check(load().ctqw_graph_init_state(g.handle, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), dtype,
                                        _ptr(psi), _stream(stream)))


def ctqw_graph_propagate_taylor(g: Graph, psi: torch.Tensor, dtype: int, dt: float, K: int, n_steps: int,
                                obs_every: int = 0, P_mean=None, norm=None, energy=None,
                                workspace: Optional[torch.Tensor] = None, stream=None):
    if workspace is None:
        workspace = g.workspace(dtype, psi.device)
    _check(load().ctqw_graph_propagate_taylor(g.handle, dtype, _ptr(psi), float(dt), int(K), int(n_steps),
                                              int(obs_every), _ptr(P_mean), _ptr(norm), _ptr(energy),
                                              _ptr(workspace), workspace.numel(), _stream(stream)))


def ctqw_graph_propagate_rk4(g: Graph, psi: torch.Tensor, dtype: int, dt: float, n_steps: int,
                             obs_every: int = 0, P_mean=None, norm=None, energy=None,
                             workspace: Optional[torch.Tensor] = None, stream=None):
    if workspace is None:
        workspace = g.workspace(dtype, psi.device)
    _check(load().ctqw_graph_propagate_rk4(g.handle, dtype, _ptr(psi), float(dt), int(n_steps), int(obs_every),
                                           _ptr(P_mean), _ptr(norm), _ptr(energy), _ptr(workspace),
                                           workspace.numel(), _stream(stream)))


def ctqw_graph_observables(g: Graph, psi: torch.Tensor, dtype: int, P_mean=None, norm=None, energy=None,
                           stream=None):
    _check(load().ctqw_graph_observables(g.handle, dtype, _ptr(psi), _ptr(P_mean), _ptr(norm), _ptr(energy),
                                         _stream(stream)))


def ctqw_init_state(h: Hamiltonian, psi: torch.Tensor, sites, dtype: int, stream=None) -> None:
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.int32).reshape(h.R, h.m))
    _check(load().ctqw_init_state(h.handle, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), dtype,
                                  _ptr(psi), _stream(stream)))


def _outputs(h: Hamiltonian, n_obs: int, want_P: bool, want_norm: bool, want_energy: bool, device):
    P = torch.empty((n_obs, h.p_width), dtype=torch.float64, device=device) if want_P and n_obs else None
    nr = torch.empty((n_obs, h.R), dtype=torch.float64, device=device) if want_norm and n_obs else None
    en = torch.empty((n_obs, h.R), dtype=torch.float64, device=device) if want_energy and n_obs else None
    return P, nr, en


def ctqw_propagate_taylor(h: Hamiltonian, psi: torch.Tensor, dtype: int, dt: float, K: int,
                          n_steps: int, obs_every: int = 0, P_mean=None, norm=None, energy=None,
                          flags: int = 0, workspace: Optional[torch.Tensor] = None, stream=None):
    ws_bytes = 0 if workspace is None else workspace.numel()
    _check(load().ctqw_propagate_taylor(h.handle, dtype, _ptr(psi), float(dt), int(K), int(n_steps),
                                        int(obs_every), _ptr(P_mean), _ptr(norm), _ptr(energy),
                                        int(flags), _ptr(workspace), ws_bytes, _stream(stream)))


def ctqw_propagate_taylor_switching(h: Hamiltonian, psi: torch.Tensor, dtype: int, dt: float, K: int,
                                    n_steps: int, obs_every: int, P_mean, norm, energy, seed: int,
                                    p_switch: float, flags: int = 0,
                                    workspace: Optional[torch.Tensor] = None, stream=None):
    if workspace is None:
        workspace = h.workspace(dtype, TAYLOR, FLAG_PLAIN, psi.device)
    _check(load().ctqw_propagate_taylor_switching(
        h.handle, dtype, _ptr(psi), float(dt), int(K), int(n_steps), int(obs_every), _ptr(P_mean),
        _ptr(norm), _ptr(energy), int(flags), _ptr(workspace), workspace.numel(), int(seed),
        float(p_switch), _stream(stream)))


def ctqw_propagate_exact(h: Hamiltonian, psi: torch.Tensor, dt: float, n_steps: int, obs_every: int = 0,
                         P_mean=None, norm=None, energy=None, stream=None) -> np.ndarray:
    """Exact propagation by diagonalisation (FP64, N^m <= 64); returns the
    Jacobi sweeps of every realization (host, after a synchronisation)."""
    sweeps = np.zeros(h.R, dtype=np.int32)
    _check(load().ctqw_propagate_exact(h.handle, C128, _ptr(psi), float(dt), int(n_steps), int(obs_every),
                                       _ptr(P_mean), _ptr(norm), _ptr(energy),
                                       sweeps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       _stream(stream)))
    torch.cuda.synchronize()
    return sweeps


def ctqw_propagate_rk4(h: Hamiltonian, psi: torch.Tensor, dtype: int, dt: float, n_steps: int,
                       obs_every: int = 0, P_mean=None, norm=None, energy=None, flags: int = 0,
                       workspace: Optional[torch.Tensor] = None, stream=None):
    ws_bytes = 0 if workspace is None else workspace.numel()
    _check(load().ctqw_propagate_rk4(h.handle, dtype, _ptr(psi), float(dt), int(n_steps),
                                     int(obs_every), _ptr(P_mean), _ptr(norm), _ptr(energy),
                                     int(flags), _ptr(workspace), ws_bytes, _stream(stream)))


def ctqw_ensemble_observables(h: Hamiltonian, psi: torch.Tensor, dtype: int, P_mean=None,
                              P_joint=None, norm=None, energy=None, stream=None):
    _check(load().ctqw_ensemble_observables(h.handle, dtype, _ptr(psi), _ptr(P_mean), _ptr(P_joint),
                                            _ptr(norm), _ptr(energy), _stream(stream)))


def ctqw_taylor_order(h_dt: float, n_steps: int, tol: float, K_min: int = 1, K_max: int = 30):
    """(K, bound): smallest order whose summed truncation bound is within tol/10."""
    K = ctypes.c_int32()
    b = ctypes.c_double()
    _check(load().ctqw_taylor_order(float(h_dt), int(n_steps), float(tol), int(K_min), int(K_max),
                                    ctypes.byref(K), ctypes.byref(b)))
    return K.value, b.value


def ctqw_autotune_order(h: Hamiltonian, dtype: int, dt: float, n_steps: int, K_min: int = 1,
                        K_max: int = 30) -> int:
    """Order the library picks for this handle (as K = 0 in ctqw_propagate_taylor)."""
    K = ctypes.c_int32()
    _check(load().ctqw_autotune_order(h.handle, dtype, float(dt), int(n_steps), int(K_min),
                                      int(K_max), ctypes.byref(K)))
    return K.value


def ctqw_one_body_density(h: Hamiltonian, psi: torch.Tensor, dtype: int, stream=None):
    """Per size group, the ensemble-averaged one-body density matrix: a list of
    complex128 device tensors [N_g, N_g] (ctqw_one_body_density)."""
    sizes = [int(n) for n in h.group_sizes]
    total = sum(n * n for n in sizes)
    rho = torch.empty(2 * total, dtype=torch.float64, device=psi.device)
    _check(load().ctqw_one_body_density(h.handle, dtype, _ptr(psi), _ptr(rho), _stream(stream)))
    out, off = [], 0
    c = torch.view_as_complex(rho.view(total, 2))
    for n in sizes:
        out.append(c[off:off + n * n].view(n, n))
        off += n * n
    return out


def ctqw_set_norm_check(h: Hamiltonian, drift_tol: float) -> None:
    _check(load().ctqw_set_norm_check(h.handle, float(drift_tol)))


def ctqw_set_density_method(h: Hamiltonian, method: int) -> None:
    """0: tensor cores where supported (the default), 1: CUDA cores."""
    _check(load().ctqw_set_density_method(h.handle, int(method)))


def ctqw_inject_alloc_failure(after: int) -> None:
    _check(load().ctqw_inject_alloc_failure(int(after)))


def ctqw_fused_split(h: Hamiltonian, K: int, flags: int = 0) -> int:
    """Realizations (the last ones) the fused path runs on the register tiles
    on its second stream."""
    r = ctypes.c_int32()
    _check(load().ctqw_fused_split(h.handle, int(K), int(flags), ctypes.byref(r)))
    return r.value


def ctqw_check_status(h: Hamiltonian, stream=None) -> None:
    _check(load().ctqw_check_status(h.handle, _stream(stream)))


def adjoint_workspace(h: Hamiltonian, dtype: int, K: int, n_steps: int, checkpoint_every: int,
                      device="cuda") -> torch.Tensor:
    b = ctypes.c_size_t()
    _check(load().ctqw_adjoint_workspace_size(h.handle, dtype, int(K), int(n_steps),
                                              int(checkpoint_every), ctypes.byref(b)))
    return torch.empty(b.value, dtype=torch.uint8, device=device)


def ctqw_adjoint_grad(h: Hamiltonian, psi0: torch.Tensor, dtype: int, dt: float, K: int,
                      n_steps: int, checkpoint_every: int, P_target: torch.Tensor, stream=None,
                      workspace: Optional[torch.Tensor] = None, per_realization: bool = True,
                      means: bool = True):
    """Loss on Pbar(x, T) and its gradients (ctqw_adjoint_grad).

    Returns (loss [1], grad_eps [sum N], grad_J [sum N], P_final [p_width],
    grad_eps_mean [p_width], grad_J_mean [p_width]) as FP64 device tensors:
    the gradients w.r.t. every realization's eps and J (None unless
    per_realization) and their sums over each size group's realizations,
    the gradients w.r.t. the means the group shares (None unless means).
    workspace: from adjoint_workspace (allocated here when None).
    """
    dev = psi0.device
    ws = workspace if workspace is not None else adjoint_workspace(h, dtype, K, n_steps,
                                                                   checkpoint_every, dev)
    n = int(h.sizes.sum())
    f64 = dict(dtype=torch.float64, device=dev)
    loss = torch.empty(1, **f64)
    ge = torch.empty(n, **f64) if per_realization else None
    gJ = torch.empty(n, **f64) if per_realization else None
    gem = torch.empty(h.p_width, **f64) if means else None
    gJm = torch.empty(h.p_width, **f64) if means else None
    Pf = torch.empty(h.p_width, **f64)
    tgt = P_target.to(device=dev, dtype=torch.float64).contiguous()
    _check(load().ctqw_adjoint_grad(h.handle, dtype, _ptr(psi0), float(dt), int(K), int(n_steps),
                                    int(checkpoint_every), _ptr(tgt), _ptr(loss), _ptr(ge), _ptr(gJ),
                                    _ptr(gem), _ptr(gJm), _ptr(Pf), _ptr(ws), ws.numel(),
                                    _stream(stream)))
    return loss, ge, gJ, Pf, gem, gJm


class EnsembleOccupationLoss(torch.autograd.Function):
    """loss = sum_x (Pbar(x, T) - P_target(x))^2 as a function of the mean on-site
    energies and hoppings shared by all realizations (each realization adds its
    own disorder drawn from the uniform draws of the workload).

    forward(eps_mean [N], J_mean [N], w, P_target [N], dtype, checkpoint_every)
    runs the CUDA adjoint once and keeps the gradients for backward.
    """

    @staticmethod
    def forward(ctx, eps_mean, J_mean, w, P_target, dtype=C64, checkpoint_every=50):
        em = eps_mean.detach().to("cpu", torch.float64).numpy()
        jm = J_mean.detach().to("cpu", torch.float64).numpy()
        h = build_for_workload(w, eps_mean=em, J_mean=jm)
        psi = h.new_state(dtype, P_target.device if P_target.is_cuda else "cuda")
        ctqw_init_state(h, psi, initial_sites(w, h), dtype)
        loss, _, _, _, gem, gJm = ctqw_adjoint_grad(h, psi, dtype, w.dt, w.K, w.n_steps,
                                                    checkpoint_every, P_target, per_realization=False)
        ctx.save_for_backward(gem.to(eps_mean.device, eps_mean.dtype),
                              gJm.to(J_mean.device, J_mean.dtype))
        h.close()
        return loss[0].to(eps_mean.device, eps_mean.dtype)

    @staticmethod
    def backward(ctx, g):
        ge, gJ = ctx.saved_tensors
        return g * ge, g * gJ, None, None, None, None


def ctqw_version() -> str:
    return load().ctqw_version().decode()


# ------------------------------------------------------------------ workloads
def build_for_workload(w, realizations=None, eps_mean=None, J_mean=None, round_to_f32=True,
                       stream=None) -> Hamiltonian:
    """Hamiltonian handle of (a subset of) a ctqw_workloads.Workload."""
    import ctqw_workloads as cw

    u_eps, u_J, sizes, _ = cw.packed_draws(w, realizations)
    return Hamiltonian(w.m, w.statistics, w.periodic, sizes, w.J0, w.U, w.eps_halfwidth,
                       w.J_halfwidth, u_eps, u_J, eps_mean, J_mean, round_to_f32, stream)


def initial_sites(w, h: Hamiltonian) -> np.ndarray:
    return np.array([w.initial_sites(int(n)) for n in h.sizes], dtype=np.int32)


def run_workload(w, realizations=None, method: int = TAYLOR, dtype: Optional[int] = None,
                 n_steps: Optional[int] = None, obs_every: Optional[int] = None,
                 K: Optional[int] = None, flags: int = 0, device="cuda"):
    """Build, initialise and propagate a workload; returns host results."""
    dtype = w.dtype if dtype is None else dtype
    n_steps = w.n_steps if n_steps is None else n_steps
    obs_every = w.obs_every if obs_every is None else obs_every
    K = w.K if K is None else K
    h = build_for_workload(w, realizations)
    psi = h.new_state(dtype, device)
    ctqw_init_state(h, psi, initial_sites(w, h), dtype)
    n_obs = h.n_obs(n_steps, obs_every)
    P, nr, en = _outputs(h, n_obs, True, True, True, device)
    ws = h.workspace(dtype, method, flags, device)
    if method == TAYLOR:
        ctqw_propagate_taylor(h, psi, dtype, w.dt, K, n_steps, obs_every, P, nr, en, flags, ws)
    else:
        ctqw_propagate_rk4(h, psi, dtype, w.dt, n_steps, obs_every, P, nr, en, flags, ws)
    ctqw_check_status(h)
    out = {"psi": psi.cpu().numpy(), "st_off": h.st_off, "sizes": h.sizes,
           "group_sizes": h.group_sizes, "p_width": h.p_width}
    out["P_mean"] = P.cpu().numpy() if P is not None else None
    out["norm"] = nr.cpu().numpy() if nr is not None else None
    out["energy"] = en.cpu().numpy() if en is not None else None
    h.close()
    return out
