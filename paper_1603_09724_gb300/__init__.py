"""Python binding of the GB300 OMM library (libomm.so, C ABI in include/omm.h).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
PyTorch provides device memory (torch tensors on cuda) and the stream.  Importing this
package without the built library raises ImportError: there is no CPU fallback.

The functions keep the C names (omm_create, omm_set_poles, omm_iterate, omm_solve,
omm_energy, ...).  `Solver` is a small convenience wrapper around one handle.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libomm.so")
if not os.path.exists(_LIBPATH):
    raise ImportError(
        f"{_LIBPATH} not found: build the CUDA library first "
        "(python paper_1603_09724_gb300/build.py); there is no CPU fallback")
lib = C.CDLL(_LIBPATH)

OMM_OK, OMM_EINVAL, OMM_ENOMEM, OMM_EUNSUPPORTED, OMM_ENOTCONV = 0, -1, -2, -3, -4
OMM_ETIMEOUT, OMM_ECUDA, OMM_ESHIFT, OMM_ESTATE = -5, -6, -7, -8
OMM_FP64, OMM_MIXED = 0, 1
OMM_INNER_SPARSIFY, OMM_INNER_KINETIC, OMM_INNER_NONE = 0, 1, 2


class omm_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("m", C.c_int * 3), ("box_len", C.c_double)]


class omm_params(C.Structure):
    _fields_ = [("precision", C.c_int), ("inner", C.c_int), ("gmres_m", C.c_int), ("gmres_cycles", C.c_int),
                ("gmres_rtol", C.c_double), ("gmres_fixed", C.c_int), ("stencil_radius", C.c_int),
                ("pivot_floor", C.c_double), ("tol", C.c_double), ("maxit", C.c_int), ("refilter", C.c_int),
                ("gram_tensor", C.c_int), ("real_orbitals", C.c_int), ("trsv_streams", C.c_int),
                ("trsv_persistent", C.c_int), ("fixed_iters", C.c_int), ("refilter_rtol", C.c_double),
                ("gap", C.c_double), ("launch_overlap", C.c_int), ("device_factor", C.c_int)]


class omm_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("filters", C.c_int), ("converged", C.c_int), ("energy", C.c_double),
                ("energy_fp64", C.c_double), ("resid_fp64", C.c_double), ("gmres_relres_max", C.c_double),
                ("gmres_iters_max", C.c_int), ("gmres_iters_total", C.c_int), ("grad_norm", C.c_double),
                ("resid_orth", C.c_double), ("angle_bound", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_vp, _dp, _ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
_SIGS = {
    "omm_strerror": (C.c_char_p, [C.c_int]),
    "omm_last_error_message": (C.c_char_p, []),
    "omm_default_params": (C.c_int, [C.POINTER(omm_params)]),
    "omm_default_shift": (C.c_int, [C.POINTER(omm_grid), _dp, _dp]),
    "omm_create": (C.c_int, [C.POINTER(omm_grid), _dp, C.c_int, C.c_double, C.POINTER(omm_params), _vp,
                             C.POINTER(_vp)]),
    "omm_destroy": (None, [_vp]),
    "omm_poles_fermi": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int, _dp, _dp]),
    "omm_poles_circle": (C.c_int, [C.c_double, C.c_double, C.c_int, _dp, _dp]),
    "omm_set_poles": (C.c_int, [_vp, C.c_int, _dp, _dp]),
    "omm_set_orbitals": (C.c_int, [_vp, _vp]),
    "omm_build_projector": (C.c_int, [_vp, _vp, C.c_int, C.POINTER(omm_stats)]),
    "omm_drop_projector": (C.c_int, [_vp]),
    "omm_set_gtpa": (C.c_int, [_vp, C.c_int, _dp, C.c_double]),
    "omm_drop_gtpa": (C.c_int, [_vp]),
    "omm_get_orbitals": (C.c_int, [_vp, _vp]),
    "omm_filter": (C.c_int, [_vp]),
    "omm_iterate": (C.c_int, [_vp, C.c_int, C.POINTER(omm_stats)]),
    "omm_solve": (C.c_int, [_vp, C.POINTER(omm_stats)]),
    "omm_energy": (C.c_int, [_vp, _dp]),
    "omm_solve_enqueue": (C.c_int, [_vp]),
    "omm_read_result": (C.c_int, [_vp, C.POINTER(omm_stats)]),
    "omm_apply_h": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_double, C.c_double]),
    "omm_gram": (C.c_int, [_vp, _vp, C.c_int, _vp, C.c_int, _vp]),
    "omm_gradient": (C.c_int, [_vp, _vp, _vp, _vp]),
    "omm_quartic": (C.c_int, [_vp, _vp, _vp, _dp, _dp]),
    "omm_precond_apply": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int]),
    "omm_pole_solve": (C.c_int, [_vp, _vp, _vp, C.POINTER(omm_stats)]),
    "omm_factor_info": (C.c_int, [_vp, C.c_int, _ip, C.POINTER(C.c_longlong), _dp, _ip]),
    "omm_set_allocator": (C.c_int, [_vp, _vp, _vp]),
    "omm_device_bytes": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "omm_profile_enable": (C.c_int, [_vp, C.c_int]),
    "omm_profile_read": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), _dp, _dp]),
    "omm_profile_class_name": (C.c_char_p, [C.c_int]),
    "omm_profile_read_impl": (C.c_int, [_vp, C.c_int, _dp]),
    "omm_profile_read_flops": (C.c_int, [_vp, C.c_int, _dp]),
    "omm_gram_noalloc": (C.c_int, [C.c_int, _vp, C.c_int, _vp, C.c_int, C.c_size_t, _vp, _vp]),
}
PROFILE_CLASSES = ("happly", "greenq", "trsv_levels", "orth", "gram", "block_update", "vector", "small", "trsv_leaf")
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = tuple(_SIGS)


class OmmError(RuntimeError):
    def __init__(self, status, where):
        msg = lib.omm_strerror(status).decode()
        extra = lib.omm_last_error_message().decode()
        super().__init__(f"{where}: {msg} ({status}){' - ' + extra if extra and status == OMM_ECUDA else ''}")
        self.status = status


def check(status, where="omm"):
    if status != OMM_OK:
        raise OmmError(status, where)
    return status


def _darr(x):
    import numpy as np
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a, a.ctypes.data_as(_dp)


def make_grid(dim: int, m: int, L: float) -> omm_grid:
    g = omm_grid()
    g.dim = dim
    g.m[0] = m
    g.m[1] = m
    g.m[2] = m if dim == 3 else 1
    g.box_len = L
    return g


def default_params(**kw) -> omm_params:
    p = omm_params()
    check(lib.omm_default_params(C.byref(p)), "omm_default_params")
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def default_shift(dim, m, L, V) -> float:
    g = make_grid(dim, m, L)
    a, ptr = _darr(V)
    s = C.c_double()
    check(lib.omm_default_shift(C.byref(g), ptr, C.byref(s)), "omm_default_shift")
    return s.value


def poles_fermi(a: float, b: float, c: float, P: int):
    import numpy as np
    z = np.zeros(2 * P)
    w = np.zeros(2 * P)
    check(lib.omm_poles_fermi(a, b, c, P, z.ctypes.data_as(_dp), w.ctypes.data_as(_dp)), "omm_poles_fermi")
    return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]


def poles_circle(center: float, radius: float, P: int):
    import numpy as np
    z = np.zeros(2 * P)
    w = np.zeros(2 * P)
    check(lib.omm_poles_circle(center, radius, P, z.ctypes.data_as(_dp), w.ctypes.data_as(_dp)), "omm_poles_circle")
    return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]


class Solver:
    """One OMM handle on the current CUDA device and stream.

    V: host array of n reals; N states; shift sigma (default: omm_default_shift);
    params: omm_params or keyword overrides.  Blocks are torch tensors of shape (N, n)
    (row j = column j of X), dtype complex128 (FP64) or complex64 (mixed)."""

    def __init__(self, dim, m, L, V, N, shift=None, params=None, stream=None, **kw):
        import torch
        self.torch = torch
        self.dim, self.m, self.L, self.N = dim, m, float(L), int(N)
        self.n = m ** dim
        self.grid = make_grid(dim, m, L)
        self.params = params if params is not None else default_params(**kw)
        self._V, vptr = _darr(V)
        self.shift = default_shift(dim, m, L, V) if shift is None else float(shift)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = C.c_void_p()
        check(lib.omm_create(C.byref(self.grid), vptr, self.N, self.shift, C.byref(self.params), C.c_void_p(stream),
                             C.byref(h)), "omm_create")
        self.h = h
        self.dtype = torch.complex128 if self.params.precision == OMM_FP64 else torch.complex64

    def close(self):
        if getattr(self, "h", None):
            lib.omm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _t(self, x, cols=None):
        t = self.torch
        assert isinstance(x, t.Tensor) and x.is_cuda and x.dtype == self.dtype and x.is_contiguous(), \
            "expected a contiguous CUDA tensor of the handle's complex dtype"
        if cols is not None:
            assert x.numel() == cols * self.n
        return C.c_void_p(x.data_ptr())

    def empty(self, cols=None):
        return self.torch.empty((cols or self.N, self.n), dtype=self.dtype, device="cuda")

    def set_poles(self, z, w):
        import numpy as np
        z = np.asarray(z, dtype=np.complex128)
        w = np.asarray(w, dtype=np.complex128)
        zz, zp = _darr(np.stack([z.real, z.imag], 1).ravel())
        ww, wp = _darr(np.stack([w.real, w.imag], 1).ravel())
        check(lib.omm_set_poles(self.h, len(z), zp, wp), "omm_set_poles")
        self.P = len(z)

    def set_orbitals(self, X):
        check(lib.omm_set_orbitals(self.h, self._t(X, self.N)), "omm_set_orbitals")

    def get_orbitals(self, X=None):
        X = self.empty() if X is None else X
        check(lib.omm_get_orbitals(self.h, self._t(X, self.N)), "omm_get_orbitals")
        self.torch.cuda.current_stream().synchronize()
        return X

    def filter(self):
        check(lib.omm_filter(self.h), "omm_filter")

    def iterate(self, k):
        st = omm_stats()
        check(lib.omm_iterate(self.h, k, C.byref(st)), "omm_iterate")
        return st.as_dict()

    def solve(self, allow_notconv=True):
        st = omm_stats()
        s = lib.omm_solve(self.h, C.byref(st))
        if not (s == OMM_OK or (allow_notconv and s == OMM_ENOTCONV)):
            check(s, "omm_solve")
        return st.as_dict()

    def solve_enqueue(self):
        """Enqueue a fixed-schedule solve without host synchronisation (capturable in a CUDA
        graph); read it with read_result()."""
        check(lib.omm_solve_enqueue(self.h), "omm_solve_enqueue")

    def read_result(self, allow_notconv=True):
        st = omm_stats()
        s = lib.omm_read_result(self.h, C.byref(st))
        if not (s == OMM_OK or (allow_notconv and s == OMM_ENOTCONV)):
            check(s, "omm_read_result")
        return st.as_dict()

    def energy(self):
        e = C.c_double()
        check(lib.omm_energy(self.h, C.byref(e)), "omm_energy")
        return e.value

    def apply_h(self, X, s=0.0):
        cols = X.numel() // self.n
        Y = self.torch.empty_like(X)
        s = complex(s)
        check(lib.omm_apply_h(self.h, self._t(X), self._t(Y), cols, s.real, s.imag), "omm_apply_h")
        return Y

    def gram(self, A, B):
        na, nb = A.numel() // self.n, B.numel() // self.n
        Cm = self.torch.empty((na, nb), dtype=self.torch.complex128, device="cuda")
        check(lib.omm_gram(self.h, self._t(A), na, self._t(B), nb, C.c_void_p(Cm.data_ptr())), "omm_gram")
        return Cm

    def gradient(self, X):
        HX = self.empty()
        G = self.empty()
        check(lib.omm_gradient(self.h, self._t(X, self.N), self._t(HX), self._t(G)), "omm_gradient")
        return HX, G

    def quartic(self, X, D):
        import numpy as np
        c = np.zeros(5)
        t = C.c_double()
        check(lib.omm_quartic(self.h, self._t(X, self.N), self._t(D, self.N), c.ctypes.data_as(_dp), C.byref(t)),
              "omm_quartic")
        return c, t.value

    def precond_apply(self, pole, B):
        cols = B.numel() // self.n
        U = self.torch.empty_like(B)
        check(lib.omm_precond_apply(self.h, pole, self._t(B), self._t(U), cols), "omm_precond_apply")
        return U

    def pole_solve(self, R):
        Y = self.torch.empty_like(R)
        st = omm_stats()
        check(lib.omm_pole_solve(self.h, self._t(R, self.N), self._t(Y), C.byref(st)), "omm_pole_solve")
        self.torch.cuda.current_stream().synchronize()
        return Y, st.as_dict()

    def build_projector(self, B):
        """Algorithm 2: U = orthonormal basis of N dominant columns of the pole expansion
        applied to B (N or 2N columns, row-stored (cols, n)); the handle then preconditions
        with U U^*."""
        st = omm_stats()
        cols = B.shape[0]
        check(lib.omm_build_projector(self.h, self._t(B, cols), cols, C.byref(st)), "omm_build_projector")
        self.torch.cuda.current_stream().synchronize()
        return st.as_dict()

    def drop_projector(self):
        check(lib.omm_drop_projector(self.h), "omm_drop_projector")

    def set_gtpa(self, t, tau, coeffs=None):
        """Fourier-diagonal TPA-type preconditioner (Sec. 2.2, eqs. Lap, TPA, gTPA) of degree t
        with s = |k|^2 / tau; coeffs: c_0..c_{t+1} (None: the library's default family, eq. TPA
        at t = 3).  While set it replaces the pole expansion and solve() does not filter."""
        c = None
        if coeffs is not None:
            if len(coeffs) != t + 2:
                raise ValueError("coeffs needs t + 2 values")
            c = (C.c_double * (t + 2))(*[float(v) for v in coeffs])
        check(lib.omm_set_gtpa(self.h, int(t), c, float(tau)), "omm_set_gtpa")

    def drop_gtpa(self):
        check(lib.omm_drop_gtpa(self.h), "omm_drop_gtpa")

    def factor_info(self, pole):
        ns, nnz, pr, npt = C.c_int(), C.c_longlong(), C.c_double(), C.c_int()
        check(lib.omm_factor_info(self.h, pole, C.byref(ns), C.byref(nnz), C.byref(pr), C.byref(npt)),
              "omm_factor_info")
        return dict(nsuper=ns.value, nnz=nnz.value, pivot_ratio=pr.value, nperturbed=npt.value)

    def profile(self, on=True):
        """True: reset the counters, CUDA-event timing on; 'count': reset, counting only
        (no events); False: events off."""
        mode = 2 if on == "count" else (1 if on else 0)
        check(lib.omm_profile_enable(self.h, mode), "omm_profile_enable")

    def profile_read(self):
        out = {}
        for c, name in enumerate(PROFILE_CLASSES):
            calls, kern, ms, by = C.c_longlong(), C.c_longlong(), C.c_double(), C.c_double()
            check(lib.omm_profile_read(self.h, c, C.byref(calls), C.byref(kern), C.byref(ms), C.byref(by)),
                  "omm_profile_read")
            ib, fl = C.c_double(), C.c_double()
            check(lib.omm_profile_read_impl(self.h, c, C.byref(ib)), "omm_profile_read_impl")
            check(lib.omm_profile_read_flops(self.h, c, C.byref(fl)), "omm_profile_read_flops")
            out[name] = dict(calls=calls.value, kernels=kern.value, ms=ms.value, bytes=by.value, impl_bytes=ib.value,
                             flops=fl.value)
        return out

    def device_bytes(self):
        b = C.c_size_t()
        check(lib.omm_device_bytes(self.h, C.byref(b)), "omm_device_bytes")
        return b.value
