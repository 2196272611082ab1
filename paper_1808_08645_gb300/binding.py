"""ctypes binding of libbbwadg (include/bbwadg.h), argument marshalling only.

Every function here forwards to the C ABI of the same name; no step of the
solver runs in Python. Host arrays are numpy arrays (copied to contiguous
float64/int64 as the ABI requires); device arrays are anything with a
``data_ptr()`` (torch tensors) or a raw integer address. Importing this module
never loads the library; the first call does, and raises ``RuntimeError`` if
``_lib/libbbwadg.so`` has not been built (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["BBWError", "lib", "lib_path", "Solver", "Batch", "ElasticSolver", "mesh_analyze", "projection_coeffs",
           "lsrk_coeffs", "validate_tables", "wadg_update", "wadg_update_noalloc", "EXPORTS", "F32", "F64"]

F32, F64 = 32, 64
_HERE = os.path.dirname(os.path.abspath(__file__))

STATUS = {0: "BBW_OK", -1: "BBW_ERR_ARG", -2: "BBW_ERR_MESH", -3: "BBW_ERR_NONPOS_C2",
          -4: "BBW_ERR_CUDA", -5: "BBW_ERR_NONFINITE", -6: "BBW_ERR_TIMEOUT",
          -7: "BBW_ERR_UNSUPPORTED"}

_p = C.c_void_p
_i64 = C.c_int64
_d = C.c_double
_int = C.c_int
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)
_i8p = C.POINTER(C.c_int8)
_ip = C.POINTER(C.c_int)

# name -> (restype, argtypes), in the order of include/bbwadg.h
EXPORTS = {
    "bbw_version": (_int, []),
    "bbw_last_error": (C.c_char_p, []),
    "bbw_create": (_int, [_i64, _dp, _i64, _i64p, _int, _int, _int, _p, C.POINTER(_p)]),
    "bbw_destroy": (None, [_p]),
    "bbw_info": (_int, [_p, _i64p, _ip, _ip, _ip, _ip, _ip]),
    "bbw_get_connectivity": (_int, [_p, _i32p, _i8p, _i8p]),
    "bbw_get_face_node_map": (_int, [_p, _i64p]),
    "bbw_mesh_analyze": (_int, [_i64, _dp, _i64, _i64p, _int, _i32p, _i8p, _i8p, _i64p, _dp, _dp]),
    "bbw_get_geometry": (_int, [_p, _dp, _dp]),
    "bbw_set_c2": (_int, [_p, _dp]),
    "bbw_set_params": (_int, [_p, _d, _d]),
    "bbw_set_state": (_int, [_p, _dp, _dp, _d]),
    "bbw_set_state_device": (_int, [_p, _p, _p, _int, _d]),
    "bbw_get_state": (_int, [_p, _dp, _dp, _dp]),
    "bbw_get_state_device": (_int, [_p, _p, _p, _int]),
    "bbw_set_point_source": (_int, [_p, _dp, _dp, _i64, _i64p]),
    "bbw_set_source": (_int, [_p, _i64, _dp, _dp, _i64]),
    "bbw_set_forcing": (_int, [_p, _i64, _i64p, _dp, _dp, _i64]),
    "bbw_clear_source": (_int, [_p]),
    "bbw_stage": (_int, [_p, _int, _d]),
    "bbw_step": (_int, [_p, _d, _i64]),
    "bbw_cfl_dt": (_int, [_p, _d, _dp]),
    "bbw_advance": (_int, [_p, _d, _d, _dp, _i64p]),
    "bbw_sync": (_int, [_p]),
    "bbw_get_time": (_int, [_p, _dp, _i64p]),
    "bbw_projection_coeffs": (_int, [_int, _int, _dp]),
    "bbw_lsrk_coeffs": (_int, [_dp, _dp, _dp]),
    "bbw_validate_tables": (_int, [_int, _int, _int]),
    "bbw_wadg_update": (_int, [_int, _int, _int, _i64, _p, _p, _p, _p]),
    "bbw_wadg_update_noalloc": (_int, [_int, _int, _int, _i64, _p, _p, _p, _p]),
    "bbw_set_receivers": (_int, [_p, _i64, _dp, _i64p]),
    "bbw_record": (_int, [_p, _d, _i64, _i64, _dp]),
    "bbw_adjoint": (_int, [_p, _dp, _dp, _dp]),
    "bbw_batch_create": (_int, [_int, _i64p, C.POINTER(_dp), _i64p, C.POINTER(_i64p), _ip, _int, _int, _p,
                                C.POINTER(_p)]),
    "bbw_batch_destroy": (None, [_p]),
    "bbw_batch_info": (_int, [_p, _ip, _ip, _i64p]),
    "bbw_batch_member": (_int, [_p, _int, _ip, _i64p, _ip, _ip, _i64p]),
    "bbw_batch_set_c2": (_int, [_p, _int, _dp]),
    "bbw_batch_set_state": (_int, [_p, _int, _dp, _dp]),
    "bbw_batch_get_state": (_int, [_p, _int, _dp, _dp]),
    "bbw_batch_set_params": (_int, [_p, _d, _d]),
    "bbw_batch_set_point_source": (_int, [_p, _int, _dp, _dp, _i64, _i64p]),
    "bbw_batch_clear_sources": (_int, [_p]),
    "bbw_batch_cfl_dt": (_int, [_p, _d, _dp]),
    "bbw_batch_member_cfl_dt": (_int, [_p, _int, _d, _dp]),
    "bbw_batch_set_instance_steps": (_int, [_p, _dp, _i64p]),
    "bbw_batch_instance_time": (_int, [_p, _int, _dp, _i64p]),
    "bbw_batch_set_time": (_int, [_p, _d]),
    "bbw_batch_step": (_int, [_p, _d, _i64, _int]),
    "bbw_batch_autotune": (_int, [_p, _int, _ip, _dp]),
    "bbw_batch_sync": (_int, [_p]),
    "bbw_batch_get_time": (_int, [_p, _dp, _i64p]),
    "bbw_elastic_create": (_int, [_i64, _dp, _i64, _i64p, _int, _int, _int, _p, C.POINTER(_p)]),
    "bbw_elastic_destroy": (None, [_p]),
    "bbw_elastic_info": (_int, [_p, _i64p, _ip, _ip, _ip, _ip, _ip]),
    "bbw_elastic_set_media": (_int, [_p, _dp, _dp, _dp]),
    "bbw_elastic_set_params": (_int, [_p, _d, _d]),
    "bbw_elastic_set_state": (_int, [_p, _dp, _dp, _d]),
    "bbw_elastic_get_state": (_int, [_p, _dp, _dp, _dp]),
    "bbw_elastic_set_state_device": (_int, [_p, _p, _p, _int, _d]),
    "bbw_elastic_get_state_device": (_int, [_p, _p, _p, _int]),
    "bbw_elastic_stage": (_int, [_p, _int, _d]),
    "bbw_elastic_step": (_int, [_p, _d, _i64]),
    "bbw_elastic_cfl_dt": (_int, [_p, _d, _dp]),
    "bbw_elastic_advance": (_int, [_p, _d, _d, _dp, _i64p]),
    "bbw_elastic_sync": (_int, [_p]),
    "bbw_elastic_get_time": (_int, [_p, _dp, _i64p]),
    # include/bbw_nn.h: the surrogate's kernels
    "bbw_nn_gemm": (_int, [_int, _int, _int, _p, _int, C.c_longlong, _int, _p, _int, C.c_longlong, _int, _p, _int,
                           C.c_longlong, _int, C.c_float, C.c_float, _p, _p, _int, _int, _p]),
    "bbw_nn_gelu_backward": (_int, [_p, _p, C.c_longlong, _p]),
    "bbw_nn_axis_transform": (_int, [_p, _int, _int, _p, _p, C.c_longlong, _int, _int, C.c_float, _p, _int, _p]),
    "bbw_nn_bias_grad": (_int, [_p, _p, C.c_longlong, _int, _p]),
    "bbw_nn_gather_receivers": (_int, [_p, _p, _p, _p, _p, _int, _int, _int, _int, _int, _int, _int, _p]),
    "bbw_nn_shift_traces": (_int, [_p, _p, _p, _p, C.c_longlong, _int, _p]),
    "bbw_nn_mse": (_int, [_p, _p, _p, _p, C.c_longlong, _p]),
    "bbw_nn_adam": (_int, [_p, _p, _p, _p, C.c_longlong, _int, C.c_float, C.c_float, C.c_float, C.c_float, _p]),
}


class BBWError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")


_LIB = None


def lib_path() -> str:
    return os.path.join(_HERE, "_lib", "libbbwadg.so")


def lib():
    """The loaded library (loads it on first use; raises if not built)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libbbwadg.so is not built ({path}); run "
                               "`python -m paper_1808_08645_gb300.build`")
        L = C.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(status: int, where: str):
    if status != 0:
        raise BBWError(status, where, lib().bbw_last_error().decode())


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _dev(x) -> int | None:
    if x is None:
        return None
    return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)


def projection_coeffs(N: int, M: int) -> np.ndarray:
    out = np.zeros(N + 1)
    _check(lib().bbw_projection_coeffs(N, M, _ptr(out, C.c_double)), "bbw_projection_coeffs")
    return out


def validate_tables(N: int, M: int, precision: int = F32):
    """bbw_validate_tables: raises BBWError naming the first table mismatch."""
    _check(lib().bbw_validate_tables(N, M, precision), "bbw_validate_tables")


def lsrk_coeffs():
    a, b, c = np.zeros(5), np.zeros(5), np.zeros(5)
    _check(lib().bbw_lsrk_coeffs(_ptr(a, C.c_double), _ptr(b, C.c_double), _ptr(c, C.c_double)),
           "bbw_lsrk_coeffs")
    return a, b, c


def ricker_samples(dt: float, nsteps: int, f0: float = 10.0, t0: float | None = None,
                   t_start: float = 0.0) -> np.ndarray:
    """Amplitude samples of a Ricker wavelet of peak frequency f0 and delay t0
    (default 1/f0) for nsteps RK steps of size dt starting at t_start, one per
    stage at the library's stage times (bbw_lsrk_coeffs): the ``amp`` argument
    of the source calls."""
    from . import inputs
    return inputs.ricker_samples(f0, 1.0 / f0 if t0 is None else t0, dt, nsteps, lsrk_coeffs()[2], t_start)


def mesh_analyze(vxyz, etov, N: int):
    """Host-only connectivity, face-node map and geometry (bbw_mesh_analyze)."""
    vxyz = _f64(vxyz)
    etov = np.ascontiguousarray(etov, dtype=np.int64)
    K = len(etov)
    nfp = (N + 1) * (N + 2) // 2
    etoe = np.empty((K, 4), np.int32)
    etof = np.empty((K, 4), np.int8)
    fperm = np.empty((K, 4), np.int8)
    nmap = np.empty((K, 4, nfp), np.int64)
    grad = np.empty((K, 4, 3))
    vol = np.empty(K)
    _check(lib().bbw_mesh_analyze(len(vxyz), _ptr(vxyz, C.c_double), K, _ptr(etov, C.c_int64), N,
                                  _ptr(etoe, C.c_int32), _ptr(etof, C.c_int8), _ptr(fperm, C.c_int8),
                                  _ptr(nmap, C.c_int64), _ptr(grad, C.c_double), _ptr(vol, C.c_double)),
           "bbw_mesh_analyze")
    return dict(etoe=etoe, etof=etof, fperm=fperm, nmap=nmap, grad=grad, vol=vol)


def wadg_update(N: int, M: int, precision: int, K: int, rhs, c2, out, stream=None):
    """bbw_wadg_update on device arrays (torch tensors or raw addresses)."""
    _check(lib().bbw_wadg_update(N, M, precision, K, _dev(rhs), _dev(c2), _dev(out), _dev(stream)),
           "bbw_wadg_update")


def wadg_update_noalloc(N: int, M: int, precision: int, K: int, rhs, c2, out, stream=None):
    """bbw_wadg_update_noalloc: as wadg_update, allocating no device memory."""
    _check(lib().bbw_wadg_update_noalloc(N, M, precision, K, _dev(rhs), _dev(c2), _dev(out), _dev(stream)),
           "bbw_wadg_update_noalloc")


class Solver:
    """Owner of one ``bbw_solver`` handle; methods map one-to-one to the ABI."""

    def __init__(self, vxyz, etov, N: int, M: int, precision: int = F32, stream=None):
        vxyz = _f64(vxyz)
        etov = np.ascontiguousarray(etov, dtype=np.int64)
        h = C.c_void_p()
        _check(lib().bbw_create(len(vxyz), _ptr(vxyz, C.c_double), len(etov), _ptr(etov, C.c_int64),
                                N, M, precision, _dev(stream), C.byref(h)), "bbw_create")
        self._h = h
        self.K, self.N, self.M, self.precision = len(etov), N, M, precision
        self.Np = (N + 1) * (N + 2) * (N + 3) // 6
        self.Nfp = (N + 1) * (N + 2) // 2
        self.Mp = (M + 1) * (M + 2) * (M + 3) // 6

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().bbw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- mesh --------------------------------------------------------------
    def connectivity(self):
        etoe = np.empty((self.K, 4), np.int32)
        etof = np.empty((self.K, 4), np.int8)
        fperm = np.empty((self.K, 4), np.int8)
        _check(lib().bbw_get_connectivity(self._h, _ptr(etoe, C.c_int32), _ptr(etof, C.c_int8),
                                          _ptr(fperm, C.c_int8)), "bbw_get_connectivity")
        return etoe, etof, fperm

    def face_node_map(self):
        out = np.empty((self.K, 4, self.Nfp), np.int64)
        _check(lib().bbw_get_face_node_map(self._h, _ptr(out, C.c_int64)), "bbw_get_face_node_map")
        return out

    def geometry(self):
        grad = np.empty((self.K, 4, 3))
        vol = np.empty(self.K)
        _check(lib().bbw_get_geometry(self._h, _ptr(grad, C.c_double), _ptr(vol, C.c_double)),
               "bbw_get_geometry")
        return grad, vol

    # -- inputs -------------------------------------------------------------
    def set_c2(self, c2):
        c2 = _f64(c2).reshape(self.K, self.Mp)
        _check(lib().bbw_set_c2(self._h, _ptr(c2, C.c_double)), "bbw_set_c2")

    def set_params(self, tau_p: float, tau_u: float):
        _check(lib().bbw_set_params(self._h, tau_p, tau_u), "bbw_set_params")

    def set_state(self, q, res=None, t: float = 0.0):
        q = _f64(q).reshape(4, self.K, self.Np)
        r = None if res is None else _f64(res).reshape(4, self.K, self.Np)
        _check(lib().bbw_set_state(self._h, _ptr(q, C.c_double),
                                   None if r is None else _ptr(r, C.c_double), t), "bbw_set_state")

    def set_state_device(self, q, res=None, dtype: int = F32, t: float = 0.0):
        _check(lib().bbw_set_state_device(self._h, _dev(q), _dev(res), dtype, t), "bbw_set_state_device")

    def get_state(self, with_res: bool = False, out=None):
        """(q, t) or (q, res, t); ``out`` (a C-contiguous float64 array of
        shape (4, K, Np), e.g. a view of pinned memory) receives q if given."""
        if out is not None:
            if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != 4 * self.K * self.Np:
                raise ValueError("out must be a C-contiguous float64 array of 4*K*Np values")
            q = out.reshape(4, self.K, self.Np)
        else:
            q = np.empty((4, self.K, self.Np))
        r = np.empty((4, self.K, self.Np)) if with_res else None
        t = C.c_double()
        _check(lib().bbw_get_state(self._h, _ptr(q, C.c_double),
                                   None if r is None else _ptr(r, C.c_double), C.byref(t)),
               "bbw_get_state")
        return (q, r, t.value) if with_res else (q, t.value)

    def get_state_device(self, q, res=None, dtype: int = F32):
        _check(lib().bbw_get_state_device(self._h, _dev(q), _dev(res), dtype), "bbw_get_state_device")

    def set_point_source(self, xs, amp) -> int:
        """Point source at xs with amplitude samples amp (one per RK stage,
        sample 5 n + s at stage s of step n since set_state); its element."""
        xs = _f64(xs)
        a = _f64(amp).ravel()
        e = C.c_int64()
        _check(lib().bbw_set_point_source(self._h, _ptr(xs, C.c_double), _ptr(a, C.c_double), a.size,
                                          C.byref(e)), "bbw_set_point_source")
        return e.value

    def set_source(self, elem: int, coeffs, amp):
        c = _f64(coeffs)
        a = _f64(amp).ravel()
        _check(lib().bbw_set_source(self._h, elem, _ptr(c, C.c_double), _ptr(a, C.c_double), a.size),
               "bbw_set_source")

    def set_forcing(self, elems, coeffs, amp):
        """Forcing a(t) g(x): g by coefficients coeffs [n, Np] on elements
        elems [n], a(t) by the samples amp."""
        el = np.ascontiguousarray(elems, dtype=np.int64).ravel()
        c = _f64(coeffs).reshape(el.size, self.Np)
        a = _f64(amp).ravel()
        _check(lib().bbw_set_forcing(self._h, el.size, _ptr(el, C.c_int64), _ptr(c, C.c_double),
                                     _ptr(a, C.c_double), a.size), "bbw_set_forcing")

    def clear_source(self):
        _check(lib().bbw_clear_source(self._h), "bbw_clear_source")

    # -- time stepping -------------------------------------------------------
    def stage(self, s: int, dt: float):
        _check(lib().bbw_stage(self._h, s, dt), "bbw_stage")

    def step(self, dt: float, nsteps: int = 1):
        _check(lib().bbw_step(self._h, dt, nsteps), "bbw_step")

    def cfl_dt(self, cfl: float) -> float:
        dt = C.c_double()
        _check(lib().bbw_cfl_dt(self._h, cfl, C.byref(dt)), "bbw_cfl_dt")
        return dt.value

    def advance(self, T: float, cfl: float):
        dt = C.c_double()
        n = C.c_int64()
        _check(lib().bbw_advance(self._h, T, cfl, C.byref(dt), C.byref(n)), "bbw_advance")
        return dt.value, n.value

    def sync(self):
        _check(lib().bbw_sync(self._h), "bbw_sync")

    # -- receivers and the adjoint ---------------------------------------------
    def set_receivers(self, xyz):
        xyz = _f64(xyz).reshape(-1, 3)
        el = np.empty(len(xyz), np.int64)
        _check(lib().bbw_set_receivers(self._h, len(xyz), _ptr(xyz, C.c_double), _ptr(el, C.c_int64)),
               "bbw_set_receivers")
        self.nrec = len(xyz)
        return el

    def record(self, dt: float, nsteps: int, checkpoint_every: int = 1):
        """Run nsteps steps keeping checkpoints (checkpoint_every = 0: every
        stage's pressure bracket instead); returns the traces [nsteps][nrec].
        ``runs`` counts the recorded runs of this solver (bbw_adjoint
        differentiates the latest one)."""
        tr = np.empty((nsteps, getattr(self, "nrec", 0)))
        _check(lib().bbw_record(self._h, dt, nsteps, checkpoint_every,
                                _ptr(tr, C.c_double) if tr.size else None), "bbw_record")
        self.runs = getattr(self, "runs", 0) + 1
        return tr

    def adjoint(self, trace_grad, want_q0: bool = False):
        """Gradients (grad_c2 [K][Mp], grad_q0 [4][K][Np] or None) of
        sum(trace_grad * traces) over the recorded run."""
        g = _f64(trace_grad)
        gc = np.empty((self.K, self.Mp))
        gq = np.empty((4, self.K, self.Np)) if want_q0 else None
        _check(lib().bbw_adjoint(self._h, _ptr(g, C.c_double) if g.size else None, _ptr(gc, C.c_double),
                                 None if gq is None else _ptr(gq, C.c_double)), "bbw_adjoint")
        return gc, gq

    def time(self):
        t = C.c_double()
        n = C.c_int64()
        _check(lib().bbw_get_time(self._h, C.byref(t), C.byref(n)), "bbw_get_time")
        return t.value, n.value


class Batch:
    """Owner of one ``bbw_batch`` handle: n independent instances (meshes of
    uneven size, degrees N_i) advanced together; methods map one-to-one to
    the ABI, instance arrays as for ``Solver``."""

    def __init__(self, meshes, Ns, M: int, precision: int = F32, stream=None):
        meshes = [(_f64(v), np.ascontiguousarray(e, dtype=np.int64)) for v, e in meshes]
        n = len(meshes)
        if n != len(Ns):
            raise ValueError("one degree per mesh")
        self._keep = meshes
        nverts = np.array([len(v) for v, _ in meshes], np.int64)
        K = np.array([len(e) for _, e in meshes], np.int64)
        vptr = (_dp * n)(*[_ptr(v, C.c_double) for v, _ in meshes])
        eptr = (_i64p * n)(*[_ptr(e, C.c_int64) for _, e in meshes])
        Nn = np.array(Ns, np.int32)
        h = C.c_void_p()
        _check(lib().bbw_batch_create(n, _ptr(nverts, C.c_int64), vptr, _ptr(K, C.c_int64), eptr,
                                      _ptr(Nn, C.c_int), M, precision, _dev(stream), C.byref(h)),
               "bbw_batch_create")
        self._h = h
        self._keep = None
        self.n, self.M, self.precision = n, M, precision
        self.Ns = [int(x) for x in Ns]
        self.Ks = [int(x) for x in K]
        self.Mp = (M + 1) * (M + 2) * (M + 3) // 6

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().bbw_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def np_(self, i: int) -> int:
        N = self.Ns[i]
        return (N + 1) * (N + 2) * (N + 3) // 6

    def info(self):
        n, nb, el = C.c_int(), C.c_int(), C.c_int64()
        _check(lib().bbw_batch_info(self._h, C.byref(n), C.byref(nb), C.byref(el)), "bbw_batch_info")
        return n.value, nb.value, el.value

    def member(self, i: int):
        N, K, Np, b, e0 = C.c_int(), C.c_int64(), C.c_int(), C.c_int(), C.c_int64()
        _check(lib().bbw_batch_member(self._h, i, C.byref(N), C.byref(K), C.byref(Np), C.byref(b), C.byref(e0)),
               "bbw_batch_member")
        return dict(N=N.value, K=K.value, Np=Np.value, bucket=b.value, first=e0.value)

    def set_c2(self, i: int, c2):
        c2 = _f64(c2).reshape(self.Ks[i], self.Mp)
        _check(lib().bbw_batch_set_c2(self._h, i, _ptr(c2, C.c_double)), "bbw_batch_set_c2")

    def set_state(self, i: int, q, res=None):
        shape = (4, self.Ks[i], self.np_(i))
        q = _f64(q).reshape(shape)
        r = None if res is None else _f64(res).reshape(shape)
        _check(lib().bbw_batch_set_state(self._h, i, _ptr(q, C.c_double),
                                         None if r is None else _ptr(r, C.c_double)), "bbw_batch_set_state")

    def get_state(self, i: int, with_res: bool = False):
        shape = (4, self.Ks[i], self.np_(i))
        q = np.empty(shape)
        r = np.empty(shape) if with_res else None
        _check(lib().bbw_batch_get_state(self._h, i, _ptr(q, C.c_double),
                                         None if r is None else _ptr(r, C.c_double)), "bbw_batch_get_state")
        return (q, r) if with_res else q

    def set_params(self, tau_p: float, tau_u: float):
        _check(lib().bbw_batch_set_params(self._h, tau_p, tau_u), "bbw_batch_set_params")

    def set_point_source(self, i: int, xs, amp) -> int:
        """Point source of instance i at xs with amplitude samples amp (one per
        RK stage, sample 5 n + s at stage s of step n since set_time)."""
        xs = _f64(xs)
        a = _f64(amp).ravel()
        e = C.c_int64()
        _check(lib().bbw_batch_set_point_source(self._h, i, _ptr(xs, C.c_double), _ptr(a, C.c_double),
                                                a.size, C.byref(e)), "bbw_batch_set_point_source")
        return e.value

    def clear_sources(self):
        _check(lib().bbw_batch_clear_sources(self._h), "bbw_batch_clear_sources")

    def cfl_dt(self, cfl: float) -> float:
        dt = C.c_double()
        _check(lib().bbw_batch_cfl_dt(self._h, cfl, C.byref(dt)), "bbw_batch_cfl_dt")
        return dt.value

    def member_cfl_dt(self, i: int, cfl: float) -> float:
        dt = C.c_double()
        _check(lib().bbw_batch_member_cfl_dt(self._h, i, cfl, C.byref(dt)), "bbw_batch_member_cfl_dt")
        return dt.value

    def set_instance_steps(self, dt=None, nsteps=None):
        """Per-instance time steps dt [n] and step budgets nsteps [n] (None:
        the common dt of ``step`` / no budget)."""
        d = None if dt is None else _f64(dt)
        k = None if nsteps is None else np.ascontiguousarray(nsteps, dtype=np.int64)
        _check(lib().bbw_batch_set_instance_steps(self._h, None if d is None else _ptr(d, C.c_double),
                                                  None if k is None else _ptr(k, C.c_int64)),
               "bbw_batch_set_instance_steps")

    def instance_time(self, i: int):
        t = C.c_double()
        n = C.c_int64()
        _check(lib().bbw_batch_instance_time(self._h, i, C.byref(t), C.byref(n)), "bbw_batch_instance_time")
        return t.value, n.value

    def set_time(self, t: float):
        _check(lib().bbw_batch_set_time(self._h, t), "bbw_batch_set_time")

    def step(self, dt: float, nsteps: int = 1, graph: bool = True):
        _check(lib().bbw_batch_step(self._h, dt, nsteps, 1 if graph else 0), "bbw_batch_step")

    def autotune(self, steps: int = 3):
        """Time the candidate launch schedules and keep the fastest; returns
        (schedule index, ms per step)."""
        c = C.c_int()
        ms = C.c_double()
        _check(lib().bbw_batch_autotune(self._h, steps, C.byref(c), C.byref(ms)), "bbw_batch_autotune")
        return c.value, ms.value

    def sync(self):
        _check(lib().bbw_batch_sync(self._h), "bbw_batch_sync")

    def time(self):
        t = C.c_double()
        n = C.c_int64()
        _check(lib().bbw_batch_get_time(self._h, C.byref(t), C.byref(n)), "bbw_batch_get_time")
        return t.value, n.value


class ElasticSolver:
    """Owner of one ``bbw_elastic`` handle (the velocity-stress solver of
    Sec. 2.2); methods map one-to-one to the ``bbw_elastic_*`` ABI. State
    arrays are [9, K, Np]: (v_x, v_y, v_z, s_xx, s_yy, s_zz, s_yz, s_xz, s_xy)."""

    NF = 9

    def __init__(self, vxyz, etov, N: int, M: int, precision: int = F32, stream=None):
        vxyz = _f64(vxyz)
        etov = np.ascontiguousarray(etov, dtype=np.int64)
        h = C.c_void_p()
        _check(lib().bbw_elastic_create(len(vxyz), _ptr(vxyz, C.c_double), len(etov), _ptr(etov, C.c_int64),
                                        N, M, precision, _dev(stream), C.byref(h)), "bbw_elastic_create")
        self._h = h
        self.K, self.N, self.M, self.precision = len(etov), N, M, precision
        self.Np = (N + 1) * (N + 2) * (N + 3) // 6
        self.Mp = (M + 1) * (M + 2) * (M + 3) // 6

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().bbw_elastic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_media(self, rho_inv, lam, mu):
        a, b, c = (_f64(x).reshape(self.K, self.Mp) for x in (rho_inv, lam, mu))
        _check(lib().bbw_elastic_set_media(self._h, _ptr(a, C.c_double), _ptr(b, C.c_double),
                                           _ptr(c, C.c_double)), "bbw_elastic_set_media")

    def set_params(self, tau_v: float, tau_s: float):
        _check(lib().bbw_elastic_set_params(self._h, tau_v, tau_s), "bbw_elastic_set_params")

    def set_state(self, q, res=None, t: float = 0.0):
        q = _f64(q).reshape(9, self.K, self.Np)
        r = None if res is None else _f64(res).reshape(9, self.K, self.Np)
        _check(lib().bbw_elastic_set_state(self._h, _ptr(q, C.c_double),
                                           None if r is None else _ptr(r, C.c_double), t),
               "bbw_elastic_set_state")

    def get_state(self, with_res: bool = False, out=None):
        """(q, t) or (q, res, t); ``out`` (C-contiguous float64, 9*K*Np values)
        receives q if given."""
        if out is not None:
            if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != 9 * self.K * self.Np:
                raise ValueError("out must be a C-contiguous float64 array of 9*K*Np values")
            q = out.reshape(9, self.K, self.Np)
        else:
            q = np.empty((9, self.K, self.Np))
        r = np.empty((9, self.K, self.Np)) if with_res else None
        t = C.c_double()
        _check(lib().bbw_elastic_get_state(self._h, _ptr(q, C.c_double),
                                           None if r is None else _ptr(r, C.c_double), C.byref(t)),
               "bbw_elastic_get_state")
        return (q, r, t.value) if with_res else (q, t.value)

    def set_state_device(self, q, res=None, dtype: int = F32, t: float = 0.0):
        _check(lib().bbw_elastic_set_state_device(self._h, _dev(q), _dev(res), dtype, t),
               "bbw_elastic_set_state_device")

    def get_state_device(self, q, res=None, dtype: int = F32):
        _check(lib().bbw_elastic_get_state_device(self._h, _dev(q), _dev(res), dtype),
               "bbw_elastic_get_state_device")

    def stage(self, s: int, dt: float):
        _check(lib().bbw_elastic_stage(self._h, s, dt), "bbw_elastic_stage")

    def step(self, dt: float, nsteps: int = 1):
        _check(lib().bbw_elastic_step(self._h, dt, nsteps), "bbw_elastic_step")

    def cfl_dt(self, cfl: float) -> float:
        dt = C.c_double()
        _check(lib().bbw_elastic_cfl_dt(self._h, cfl, C.byref(dt)), "bbw_elastic_cfl_dt")
        return dt.value

    def advance(self, T: float, cfl: float):
        dt = C.c_double()
        n = C.c_int64()
        _check(lib().bbw_elastic_advance(self._h, T, cfl, C.byref(dt), C.byref(n)), "bbw_elastic_advance")
        return dt.value, n.value

    def sync(self):
        _check(lib().bbw_elastic_sync(self._h), "bbw_elastic_sync")

    def time(self):
        t = C.c_double()
        n = C.c_int64()
        _check(lib().bbw_elastic_get_time(self._h, C.byref(t), C.byref(n)), "bbw_elastic_get_time")
        return t.value, n.value

