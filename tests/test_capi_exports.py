"""The C-ABI library loads and exports every function declared in include/omm.h (no GPU
needed; nothing is computed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "omm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(omm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("omm_create", "omm_set_poles", "omm_iterate", "omm_solve", "omm_energy", "omm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1603_09724_gb300 as omm
    lib = ctypes.CDLL(omm._LIBPATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(omm.EXPORTED)


def test_host_only_entry_points_work_without_gpu():
    """Pole rules, defaults and status strings are host code (no device needed)."""
    import numpy as np
    import paper_1603_09724_gb300 as omm
    assert omm.lib.omm_strerror(omm.OMM_ESHIFT).decode().startswith("H - sigma")
    p = omm.default_params()
    assert p.gmres_m == 15 and p.gmres_cycles == 5 and abs(p.gmres_rtol - 1e-5) < 1e-20
    assert p.launch_overlap == 1 and p.trsv_persistent == 0 and p.fixed_iters == 0
    z, w = omm.poles_fermi(-10.0, -2.0, -1.6, 8)
    assert z.shape == (8,)
    with pytest.raises(omm.OmmError):
        omm.poles_fermi(-1.0, 2.0, 1.0, 8)   # b > c: invalid interval
    with pytest.raises(omm.OmmError):
        omm.poles_fermi(-1.0, 1.0, 2.0, 7)   # odd P
    assert np.all(np.isfinite(w))


def test_create_rejects_bad_arguments_before_touching_the_device():
    """omm_create validates its arguments on the host before any allocation: a shift that
    leaves H - sigma indefinite (Sec. 1: E_omm is then unbounded below), an unsupported grid
    size, malformed parameters."""
    import ctypes as C
    import numpy as np
    import paper_1603_09724_gb300 as omm
    m, L = 16, 10.0
    V = np.zeros(m * m)
    Vp = V.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()

    def create(grid, shift, prm=None, Np=4):
        return omm.lib.omm_create(C.byref(grid), Vp, Np, shift, C.byref(prm) if prm is not None else None, None,
                                  C.byref(h))

    g = omm.make_grid(2, m, L)
    tmax = 2 * np.pi ** 2 / L ** 2 * 2 * (m // 2) ** 2
    assert create(g, 0.5 * tmax) == omm.OMM_ESHIFT
    assert create(omm.make_grid(2, 14, L), 2 * tmax) == omm.OMM_EUNSUPPORTED    # 14 = 2 * 7
    assert create(omm.make_grid(4, m, L), 2 * tmax) == omm.OMM_EINVAL
    bad = omm.default_params(gmres_m=0)
    assert create(g, 2 * tmax, bad) == omm.OMM_EINVAL
    bad = omm.default_params(stencil_radius=2)
    assert create(g, 2 * tmax, bad) == omm.OMM_EINVAL
    bad = omm.default_params(launch_overlap=2)
    assert create(g, 2 * tmax, bad) == omm.OMM_EINVAL
    assert create(g, 2 * tmax, None, Np=0) == omm.OMM_EINVAL
    assert not h.value


def test_create_rejects_non_finite_inputs_before_touching_the_device():
    """Injected faults, caught on the host: a NaN or an infinity in V, a non-finite shift,
    NaN or negative tolerances and pivot floor all return OMM_EINVAL and leave no handle."""
    import ctypes as C
    import numpy as np
    import paper_1603_09724_gb300 as omm
    m, L = 16, 10.0
    g = omm.make_grid(2, m, L)
    shift = 2 * (2 * np.pi ** 2 / L ** 2 * 2 * (m // 2) ** 2)
    h = C.c_void_p()

    def create(V, shift, prm=None):
        V = np.ascontiguousarray(V, dtype=np.float64)
        return omm.lib.omm_create(C.byref(g), V.ctypes.data_as(C.POINTER(C.c_double)), 4, shift,
                                  C.byref(prm) if prm is not None else None, None, C.byref(h))

    for bad in (np.nan, np.inf, -np.inf):
        V = np.zeros(m * m)
        V[37] = bad
        assert create(V, shift) == omm.OMM_EINVAL
    V = np.zeros(m * m)
    for s in (np.nan, np.inf):
        assert create(V, s) == omm.OMM_EINVAL
    for kw in (dict(gmres_rtol=np.nan), dict(gmres_rtol=-1e-5), dict(tol=np.nan), dict(tol=-1.0),
               dict(pivot_floor=np.nan), dict(pivot_floor=-1e-12), dict(tol=np.inf)):
        assert create(V, shift, omm.default_params(**kw)) == omm.OMM_EINVAL, kw
    assert not h.value


def test_failing_allocator_hook_leaks_nothing():
    """Fault injection through omm_set_allocator: the k-th of omm_create's device
    allocations fails (k = 1..18, all of which come before its first CUDA runtime call):
    the call returns OMM_ENOMEM, leaves no handle, makes no further allocation and has
    released every block it got."""
    import ctypes as C
    import numpy as np
    import paper_1603_09724_gb300 as omm
    ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
    FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
    live, state = {}, {"calls": 0, "fail_at": 0, "bad_free": 0}

    def alloc(size, ctx):
        state["calls"] += 1
        if state["calls"] == state["fail_at"]:
            return None
        buf = C.create_string_buffer(int(size))
        live[C.addressof(buf)] = buf
        return C.addressof(buf)

    def release(p, ctx):
        if live.pop(p, None) is None:
            state["bad_free"] += 1

    a_cb, f_cb = ALLOC(alloc), FREE(release)
    m, L = 16, 10.0
    V = np.zeros(m * m)
    g = omm.make_grid(2, m, L)
    shift = 2 * (2 * np.pi ** 2 / L ** 2 * 2 * (m // 2) ** 2)
    h = C.c_void_p()
    assert omm.lib.omm_set_allocator(a_cb, f_cb, None) == omm.OMM_OK
    try:
        for k in range(1, 19):
            state.update(calls=0, fail_at=k)
            rc = omm.lib.omm_create(C.byref(g), V.ctypes.data_as(C.POINTER(C.c_double)), 4, shift, None, None,
                                    C.byref(h))
            assert rc == omm.OMM_ENOMEM and not h.value, k
            assert state["calls"] == k and not live and state["bad_free"] == 0, k
    finally:
        omm.lib.omm_set_allocator(None, None, None)
    assert omm.lib.omm_set_allocator(a_cb, None, None) == omm.OMM_EINVAL   # both hooks or neither
