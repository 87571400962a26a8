"""Host-side checks of the C ABI (no GPU needed).

The library must load, export every function include/ctqw.h declares, and
reject bad arguments before touching the device.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ctqw.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1612_00746_gb300 import build, ctqw

    build.build()
    return ctqw.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ctqw_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ctqw_build_hamiltonian", "ctqw_propagate_taylor", "ctqw_propagate_rk4",
                     "ctqw_ensemble_observables"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1612_00746_gb300 import ctqw

    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in ctqw.EXPORTED or name.startswith("ctqw_"), name
    assert set(ctqw.EXPORTED) <= set(declared_functions())


def test_version_and_error_string(lib):
    assert b"sm_103a" in lib.ctqw_version()
    assert isinstance(lib.ctqw_last_error(), bytes)


def _desc(ctqw, **kw):
    d = ctqw.LatticeDesc()
    d.n_particles = kw.get("m", 2)
    d.statistics = kw.get("stats", 0)
    d.periodic = 0
    d.n_realizations = kw.get("R", 1)
    d.n_sites = None
    d.n_sites_uniform = kw.get("N", 8)
    d.round_to_f32 = 1
    d.J0, d.U, d.eps_halfwidth, d.J_halfwidth = 1.0, 0.0, 0.5, 0.0
    u = kw.get("u", np.full(64, 0.5))
    d.u_eps_host = u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if u is not None else None
    d.u_J_host = d.u_eps_host
    return d, u


@pytest.mark.parametrize("bad,msg", [({"m": 4}, b"n_particles"), ({"m": 1}, b"n_particles"),
                                     ({"stats": 5}, b"statistics"), ({"R": 0}, b"n_realizations"),
                                     ({"N": 1}, b"outside"), ({"N": 70000}, b"outside"),
                                     ({"u": None}, b"uniform")])
def test_build_rejects_bad_descriptions_before_any_launch(lib, bad, msg):
    from paper_1612_00746_gb300 import ctqw

    d, _keep = _desc(ctqw, **bad)
    h = ctypes.c_void_p()
    st = lib.ctqw_build_hamiltonian(ctypes.byref(d), None, ctypes.byref(h))
    assert st == ctqw.CTQW_EINVAL
    assert msg in lib.ctqw_last_error()
    assert not h.value


def test_entry_points_reject_null_handles(lib):
    from paper_1612_00746_gb300 import ctqw

    E = ctqw.CTQW_EINVAL
    assert lib.ctqw_propagate_taylor(None, 0, None, 0.01, 4, 1, 0, None, None, None, 0, None, 0, None) == E
    assert lib.ctqw_propagate_rk4(None, 0, None, 0.01, 1, 0, None, None, None, 0, None, 0, None) == E
    assert lib.ctqw_ensemble_observables(None, 0, None, None, None, None, None, None) == E
    assert lib.ctqw_state_size(None, None, None) == E
    assert lib.ctqw_get_params(None, None, None) == E
    assert lib.ctqw_init_state(None, None, 0, None, None) == E
    r = ctypes.c_int32(-1)
    assert lib.ctqw_fused_split(None, 16, 0, ctypes.byref(r)) == E
    assert lib.ctqw_destroy_hamiltonian(None) == ctqw.CTQW_OK


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1612_00746_gb300 import ctqw

    saved = ctqw._lib
    try:
        ctqw._lib = None
        with pytest.raises(RuntimeError, match="missing"):
            ctqw.load(str(tmp_path / "nope.so"))
    finally:
        ctqw._lib = saved


def _graph_desc(ctqw, **kw):
    d = ctqw.GraphDesc()
    eu = np.array(kw.pop("eu", [0, 1, 2]), dtype=np.int32)
    ev = np.array(kw.pop("ev", [1, 2, 0]), dtype=np.int32)
    ue = np.full(64, 0.5)
    d.n_particles, d.statistics, d.n_nodes, d.n_edges = 2, 0, 3, len(eu)
    d.edge_u = eu.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    d.edge_v = ev.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    d.n_realizations, d.round_to_f32 = 1, 1
    d.J0, d.U, d.eps_halfwidth, d.J_halfwidth = 1.0, 0.0, 0.5, 0.1
    d.u_eps_host = ue.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.u_J_host = ue.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for k, v in kw.items():
        setattr(d, k, v)
    return d, (eu, ev, ue)


@pytest.mark.parametrize("kw,msg", [
    ({"eu": [0, 1, 1], "ev": [1, 2, 1]}, "itself"),
    ({"eu": [0, 1, 2], "ev": [1, 2, 3]}, "out of range"),
    ({"n_particles": 4}, "n_particles"),
    ({"n_nodes": 1}, "n_nodes"),
    ({"n_nodes": 50000}, "2^31"),
    ({"n_realizations": 0}, "n_realizations"),
    ({"u_eps_host": None}, "draws"),
])
def test_graph_build_rejects_bad_descriptions_before_any_launch(lib, kw, msg):
    from paper_1612_00746_gb300 import ctqw

    d, keep = _graph_desc(ctqw, **kw)
    g = ctypes.c_void_p()
    st = lib.ctqw_graph_build(ctypes.byref(d), None, ctypes.byref(g))
    assert st == ctqw.CTQW_EINVAL
    assert msg in lib.ctqw_last_error().decode()
    assert not g.value


def test_graph_entry_points_reject_null_handles(lib):
    from paper_1612_00746_gb300 import ctqw

    assert lib.ctqw_graph_propagate_taylor(None, 0, None, 0.1, 4, 1, 0, None, None, None, None, 0,
                                           None) == ctqw.CTQW_EINVAL
    assert lib.ctqw_graph_propagate_rk4(None, 0, None, 0.1, 1, 0, None, None, None, None, 0,
                                        None) == ctqw.CTQW_EINVAL
    assert lib.ctqw_graph_observables(None, 0, None, None, None, None, None) == ctqw.CTQW_EINVAL
    assert lib.ctqw_graph_init_state(None, None, 0, None, None) == ctqw.CTQW_EINVAL
    assert lib.ctqw_graph_destroy(None) == ctqw.CTQW_OK
