"""Thin ctypes binding of libvlb.so (C-ABI in include/vlb.h).

Argument marshalling only: every step of the method runs in the CUDA
library. There is no CPU fallback; if libvlb.so is missing or cannot be
loaded the binding raises. Function and field names follow the header.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvlb.so")

VLB_OK, VLB_EINVAL, VLB_EGEOM, VLB_ENOCONV, VLB_ENOMEM, VLB_ECUDA, VLB_ENONFINITE = range(7)
VLB_D2Q9, VLB_D3Q19, VLB_D3Q39 = 9, 19, 39
VLB_PERIODIC, VLB_WALL = 0, 1
VLB_F64, VLB_F32, VLB_F16, VLB_BF16 = 0, 1, 2, 3
VLB_REF_UNIFORM, VLB_REF_REST = 0, 1
VLB_COEF_AUTO, VLB_COEF_FULL, VLB_COEF_PLANE = 0, 1, 2
VLB_WALL_LINKS_ZERO, VLB_WALL_LINKS_GHOST = 0, 1
_CODES = {1: "EINVAL", 2: "EGEOM", 3: "ENOCONV", 4: "ENOMEM", 5: "ECUDA", 6: "ENONFINITE"}


class VlbError(RuntimeError):
    def __init__(self, rc, what, msg):
        super().__init__("%s failed: %s (%s)" % (what, _CODES.get(rc, rc), msg))
        self.rc = rc
        self.code = _CODES.get(rc, str(rc))


class vlb_mesh_desc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("lattice", C.c_int32), ("n", C.c_int64 * 3),
                ("x", C.POINTER(C.c_double)), ("bc", C.c_int32 * 3),
                ("period_shift", (C.c_double * 3) * 3), ("period_rot", (C.c_double * 9) * 3),
                ("dx", C.c_double), ("wall_links", C.c_int32)]


class vlb_params(C.Structure):
    _fields_ = [("tau", C.c_double), ("precision", C.c_int32), ("coef_mode", C.c_int32),
                ("body_force", C.c_double * 3), ("wall_u", ((C.c_double * 3) * 2) * 3),
                ("wall_omega", ((C.c_double * 3) * 2) * 3), ("max_iter", C.c_int32),
                ("tol", C.c_double), ("stream", C.c_void_p), ("reference", C.c_int32)]


class vlb_mesh_stats(C.Structure):
    _fields_ = [("J_min", C.c_double), ("J_max", C.c_double), ("feq_rest_min", C.c_double),
                ("ginv_diag_min", C.c_double), ("ginv_diag_max", C.c_double),
                ("invariant_fast_axis", C.c_int32), ("ncell", C.c_int64)]


_lib = None
_DP = C.POINTER(C.c_double)


def load():
    """Load libvlb.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libvlb.so not found at %s: build it with "
                           "paper_2401_17183_gb300.build.build()" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    sig = {
        "vlb_lattice": ([C.c_int32, C.POINTER(C.c_int32), _DP], C.c_int),
        "vlb_mesh_create": ([C.POINTER(vlb_mesh_desc), C.POINTER(vp)], C.c_int),
        "vlb_mesh_info": ([vp, C.POINTER(vlb_mesh_stats)], C.c_int),
        "vlb_mesh_geometry": ([vp, _DP, _DP, _DP, _DP], C.c_int),
        "vlb_mesh_destroy": ([vp], None),
        "vlb_init": ([vp, C.POINTER(vlb_params), _DP, _DP, C.POINTER(vp)], C.c_int),
        "vlb_reset": ([vp, _DP, _DP], C.c_int),
        "vlb_step": ([vp, C.c_int64], C.c_int),
        "vlb_sync": ([vp], C.c_int),
        "vlb_moments": ([vp, _DP, _DP, _DP, _DP], C.c_int),
        "vlb_get_state": ([vp, _DP], C.c_int),
        "vlb_set_state": ([vp, _DP], C.c_int),
        "vlb_time": ([vp], C.c_int64),
        "vlb_sim_layout": ([vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                            C.POINTER(C.c_int64)], C.c_int),
        "vlb_destroy": ([vp], None),
        "vlb_last_error": ([], C.c_char_p),
        "vlb_totals_noalloc": ([vp, vp], C.c_int),
        "vlb_batch_create": ([C.POINTER(vp), C.c_int32, C.POINTER(vp)], C.c_int),
        "vlb_batch_step": ([vp, C.c_int64], C.c_int),
        "vlb_batch_tune": ([vp, C.c_int32, C.POINTER(C.c_int64)], C.c_int),
        "vlb_batch_tune_steps": ([vp, C.c_int32, C.POINTER(C.c_int64)], C.c_int),
        "vlb_batch_shape": ([vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)], C.c_int),
        "vlb_batch_set_shape": ([vp, C.c_int32], C.c_int),
        "vlb_batch_layout": ([vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                              C.POINTER(C.c_int64)], C.c_int),
        "vlb_batch_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc, what):
    if rc != VLB_OK:
        raise VlbError(rc, what, load().vlb_last_error().decode())


def _ptr(a):
    return a.ctypes.data_as(_DP) if a is not None else None


def lattice(q):
    """Library velocity order: c (q, 3) int32 and weights w (q,)."""
    lib = load()
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    _check(lib.vlb_lattice(q, c.ctypes.data_as(C.POINTER(C.c_int32)), _ptr(w)), "vlb_lattice")
    return c, w


def make_params(params, precision=VLB_F64, coef_mode=VLB_COEF_AUTO, stream=None,
                reference=VLB_REF_UNIFORM):
    p = vlb_params()
    p.tau = float(params["tau"])
    p.precision = int(precision)
    p.coef_mode = int(coef_mode)
    bf = params.get("body_force", (0.0, 0.0, 0.0))
    for d in range(3):
        p.body_force[d] = float(bf[d])
    wu = params.get("wall_u")
    wo = params.get("wall_omega")
    wu = np.zeros((3, 2, 3)) if wu is None else np.asarray(wu, dtype=np.float64)
    wo = np.zeros((3, 2, 3)) if wo is None else np.asarray(wo, dtype=np.float64)
    for a in range(3):
        for s in range(2):
            for d in range(3):
                p.wall_u[a][s][d] = float(wu[a, s, d])
                p.wall_omega[a][s][d] = float(wo[a, s, d])
    p.max_iter = int(params.get("max_iter", 0))
    p.tol = float(params.get("tol", 0.0))
    p.stream = stream
    p.reference = int(reference)
    return p


class Mesh:
    """vlb_mesh_create / vlb_mesh_info / vlb_mesh_geometry / vlb_mesh_destroy."""

    def __init__(self, mesh):
        lib = load()
        self.dim = int(mesh["dim"])
        self.q = int(mesh["q"])
        self.n = tuple(int(v) for v in mesh["n"])
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        x = np.ascontiguousarray(mesh["x"], dtype=np.float64)
        d = vlb_mesh_desc()
        d.dim = self.dim
        d.lattice = self.q
        for a in range(3):
            d.n[a] = self.n[a]
            d.bc[a] = int(mesh["bc"][a])
            for k in range(3):
                d.period_shift[a][k] = float(mesh["shift"][a][k])
            for k in range(9):
                d.period_rot[a][k] = float(mesh["rot"][a][k])
        d.dx = float(mesh.get("dx", 1.0))
        d.wall_links = int(mesh.get("wall_links", 0))
        d.x = _ptr(x)
        h = C.c_void_p()
        _check(lib.vlb_mesh_create(C.byref(d), C.byref(h)), "vlb_mesh_create")
        self.h = h

    def info(self):
        s = vlb_mesh_stats()
        _check(load().vlb_mesh_info(self.h, C.byref(s)), "vlb_mesh_info")
        return {k: getattr(s, k) for k, _ in vlb_mesh_stats._fields_}

    def geometry(self):
        n, D, q = self.ncell, self.dim, self.q
        J = np.zeros(n)
        gl = np.zeros((n, D, D))
        gi = np.zeros((n, D, D))
        K = np.zeros((n, q, D))
        _check(load().vlb_mesh_geometry(self.h, _ptr(J), _ptr(gl), _ptr(gi), _ptr(K)),
               "vlb_mesh_geometry")
        return {"J": J, "g_low": gl, "ginv": gi, "K": K}

    def close(self):
        if getattr(self, "h", None):
            load().vlb_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sim:
    """vlb_init / vlb_step / vlb_moments / vlb_get_state / vlb_set_state / vlb_destroy."""

    def __init__(self, mesh, params, rho, u, precision=VLB_F64, coef_mode=VLB_COEF_AUTO,
                 stream=None, reference=VLB_REF_UNIFORM):
        lib = load()
        self.mesh = mesh          # keeps the mesh alive
        self.p = make_params(params, precision, coef_mode, stream, reference)
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        if rho.size != mesh.ncell or u.size != mesh.ncell * mesh.dim:
            raise ValueError("rho/u sizes do not match the mesh")
        h = C.c_void_p()
        _check(lib.vlb_init(mesh.h, C.byref(self.p), _ptr(rho), _ptr(u), C.byref(h)), "vlb_init")
        self.h = h

    def reset(self, rho, u):
        _check(load().vlb_reset(self.h, _ptr(rho), _ptr(u)), "vlb_reset")

    def reset_ptr(self, rho_ptr, u_ptr):
        """vlb_reset with raw host pointers (e.g. pinned torch tensors)."""
        _check(load().vlb_reset(self.h, C.cast(rho_ptr, _DP), C.cast(u_ptr, _DP)), "vlb_reset")

    def step(self, n=1):
        _check(load().vlb_step(self.h, int(n)), "vlb_step")

    def sync(self):
        _check(load().vlb_sync(self.h), "vlb_sync")

    def moments(self, fields=True):
        n, D = self.mesh.ncell, self.mesh.dim
        tot = np.zeros(7)
        if fields:
            rho = np.zeros(n)
            u = np.zeros((n, D))
            ut = np.zeros((n, D))
            _check(load().vlb_moments(self.h, _ptr(rho), _ptr(u), _ptr(ut), _ptr(tot)),
                   "vlb_moments")
        else:
            rho = u = ut = None
            _check(load().vlb_moments(self.h, None, None, None, _ptr(tot)), "vlb_moments")
        return {"rho": rho, "u": u, "u_tilde": ut, "mass": tot[0], "P": tot[1:1 + D],
                "M": tot[4:4 + D]}

    def moments_ptr(self, rho_ptr, u_ptr, ut_ptr, tot_ptr):
        """vlb_moments into raw host pointers (any may be 0)."""
        cast = lambda p: C.cast(p, _DP) if p else None  # noqa: E731
        _check(load().vlb_moments(self.h, cast(rho_ptr), cast(u_ptr), cast(ut_ptr),
                                  cast(tot_ptr)), "vlb_moments")

    def totals_noalloc(self, d_totals_ptr):
        """vlb_totals_noalloc into 7 doubles of caller-owned device memory."""
        _check(load().vlb_totals_noalloc(self.h, C.c_void_p(d_totals_ptr)), "vlb_totals_noalloc")

    def get_state(self):
        N = np.zeros((self.mesh.q, self.mesh.ncell))
        _check(load().vlb_get_state(self.h, _ptr(N)), "vlb_get_state")
        return N

    def set_state(self, N):
        N = np.ascontiguousarray(N, dtype=np.float64)
        _check(load().vlb_set_state(self.h, _ptr(N)), "vlb_set_state")

    def time(self):
        return int(load().vlb_time(self.h))

    def layout(self):
        a, b, c = C.c_int32(), C.c_int32(), C.c_int64()
        _check(load().vlb_sim_layout(self.h, C.byref(a), C.byref(b), C.byref(c)), "vlb_sim_layout")
        return {"coef_per_cell": a.value, "plane": bool(b.value), "records": c.value}

    def close(self):
        if getattr(self, "h", None):
            load().vlb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """vlb_batch_create / vlb_batch_step / vlb_batch_tune / vlb_batch_destroy:
    many simulations advanced by one kernel launch per time step."""

    def __init__(self, sims):
        lib = load()
        self.sims = list(sims)    # keeps the members alive
        arr = (C.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        h = C.c_void_p()
        _check(lib.vlb_batch_create(arr, len(self.sims), C.byref(h)), "vlb_batch_create")
        self.h = h

    def step(self, n=1):
        _check(load().vlb_batch_step(self.h, int(n)), "vlb_batch_step")

    def tune(self, steps=10):
        r = C.c_int64()
        _check(load().vlb_batch_tune(self.h, int(steps), C.byref(r)), "vlb_batch_tune")
        return r.value

    def set_shape(self, shape):
        _check(load().vlb_batch_set_shape(self.h, int(shape)), "vlb_batch_set_shape")

    def tune_steps(self, steps=10):
        """How many steps tune(steps) advances every member by."""
        r = C.c_int64()
        _check(load().vlb_batch_tune_steps(self.h, int(steps), C.byref(r)), "vlb_batch_tune_steps")
        return r.value

    def layout(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(load().vlb_batch_layout(self.h, C.byref(a), C.byref(b), C.byref(c)), "vlb_batch_layout")
        th, mb = C.c_int32(), C.c_int32()
        _check(load().vlb_batch_shape(self.h, C.byref(th), C.byref(mb)), "vlb_batch_shape")
        return {"blocks": a.value, "run_length": b.value, "cells": c.value, "threads": th.value,
                "min_blocks": mb.value}

    def close(self):
        if getattr(self, "h", None):
            load().vlb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
