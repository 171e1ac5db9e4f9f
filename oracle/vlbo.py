"""ctypes wrapper of the FP64 CPU oracle (oracle/vlb_oracle.c).

TEST INFRASTRUCTURE: only tests/, the smoke check and bench.py's CPU-baseline
leg use it. A mesh is the plain dict produced by the seeded input module
(keys dim, q, n, x, bc, shift, rot, dx); params is a dict with tau,
body_force, wall_u, wall_omega, max_iter, tol.
"""
import ctypes as C

import numpy as np

from .build import build_oracle

VLBO_QMAX = 39
_lib = None


class _Mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("q", C.c_int32), ("n", C.c_int64 * 3),
                ("x", C.POINTER(C.c_double)), ("bc", C.c_int32 * 3),
                ("shift", (C.c_double * 3) * 3), ("rot", (C.c_double * 9) * 3),
                ("dx", C.c_double), ("wall_links", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("tau", C.c_double), ("body_force", C.c_double * 3),
                ("wall_u", ((C.c_double * 3) * 2) * 3),
                ("wall_omega", ((C.c_double * 3) * 2) * 3),
                ("max_iter", C.c_int32), ("tol", C.c_double)]


class _Cell(C.Structure):
    _fields_ = [("J", C.c_double), ("g_low", (C.c_double * 3) * 3),
                ("g_up", (C.c_double * 3) * 3), ("gij", (C.c_double * 3) * 3),
                ("ginv", (C.c_double * 3) * 3),
                ("theta", ((C.c_double * 3) * 3) * VLBO_QMAX),
                ("wall_link", C.c_int32 * VLBO_QMAX),
                ("uw", (C.c_double * 3) * VLBO_QMAX), ("G", C.c_double * 3)]


_ERR = {1: "EINVAL", 2: "EGEOM", 3: "ENOCONV", 4: "ENOMEM"}


class OracleError(RuntimeError):
    def __init__(self, rc, what):
        super().__init__("oracle %s failed: %s" % (what, _ERR.get(rc, rc)))
        self.rc = rc
        self.code = _ERR.get(rc, str(rc))


def _check(rc, what):
    if rc != 0:
        raise OracleError(rc, what)


def _configure(lib):
    dp = C.POINTER(C.c_double)
    lib.vlbo_lattice.argtypes = [C.c_int32, C.POINTER(C.c_int32), dp, dp]
    lib.vlbo_position.argtypes = [C.POINTER(_Mesh), C.POINTER(C.c_int64), dp]
    lib.vlbo_cell_geometry.argtypes = [C.POINTER(_Mesh), C.POINTER(_Params),
                                       C.POINTER(C.c_int64), C.POINTER(_Cell)]
    lib.vlbo_equilibrium.argtypes = [C.c_int32, C.c_double, dp, dp, dp, dp]
    lib.vlbo_collide.argtypes = [C.c_int32, C.POINTER(_Cell), C.POINTER(_Params), dp,
                                 dp, dp, dp, dp, dp, dp, C.POINTER(C.c_int32)]
    lib.vlbo_create.argtypes = [C.POINTER(_Mesh), C.POINTER(_Params), C.POINTER(C.c_void_p)]
    lib.vlbo_destroy.argtypes = [C.c_void_p]
    lib.vlbo_destroy.restype = None
    lib.vlbo_init.argtypes = [C.c_void_p, dp, dp]
    lib.vlbo_step.argtypes = [C.c_void_p, C.c_int64]
    lib.vlbo_moments.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
    lib.vlbo_get_state.argtypes = [C.c_void_p, dp]
    lib.vlbo_set_state.argtypes = [C.c_void_p, dp]
    lib.vlbo_get_cell.argtypes = [C.c_void_p, C.c_int64, C.POINTER(_Cell)]
    lib.vlbo_last_iters.argtypes = [C.c_void_p]
    lib.vlbo_last_iters.restype = C.c_int32
    lib.vlbo_set_threads.argtypes = [C.c_int32]
    lib.vlbo_set_threads.restype = C.c_int
    return lib


def load():
    global _lib
    if _lib is None:
        _lib = _configure(C.CDLL(build_oracle()))
    return _lib


def set_threads(n):
    """Threads the oracle's time step may use in this process (OpenMP over
    the cells; the same results bit for bit on any count). n <= 0 keeps the
    setting. Returns the count in effect."""
    return int(load().vlbo_set_threads(int(n)))


def load_library(path):
    """A separately built copy of the oracle (the tests build mutated copies
    to show that a pin fails when the oracle is wrong)."""
    return _configure(C.CDLL(path))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _mesh_struct(mesh):
    """Build the C mesh struct; returns (struct, keep-alive array)."""
    x = np.ascontiguousarray(mesh["x"], dtype=np.float64)
    m = _Mesh()
    m.dim = int(mesh["dim"])
    m.q = int(mesh["q"])
    for a in range(3):
        m.n[a] = int(mesh["n"][a])
        m.bc[a] = int(mesh["bc"][a])
        for d in range(3):
            m.shift[a][d] = float(mesh["shift"][a][d])
        for k in range(9):
            m.rot[a][k] = float(mesh["rot"][a][k])
    m.dx = float(mesh.get("dx", 1.0))
    m.wall_links = int(mesh.get("wall_links", 0))
    m.x = _dp(x)
    return m, x


def _params_struct(params):
    p = _Params()
    p.tau = float(params["tau"])
    bf = params.get("body_force", (0.0, 0.0, 0.0))
    for d in range(3):
        p.body_force[d] = float(bf[d])
    wu = np.zeros((3, 2, 3)) if params.get("wall_u") is None else np.asarray(params["wall_u"])
    wo = (np.zeros((3, 2, 3)) if params.get("wall_omega") is None
          else np.asarray(params["wall_omega"]))
    for a in range(3):
        for s in range(2):
            for d in range(3):
                p.wall_u[a][s][d] = float(wu[a, s, d])
                p.wall_omega[a][s][d] = float(wo[a, s, d])
    p.max_iter = int(params.get("max_iter", 0))
    p.tol = float(params.get("tol", 0.0))
    return p


def lattice(q):
    """Velocity set of the oracle: c (q, 3) int, w (q,), T0."""
    lib = load()
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    t0 = C.c_double()
    _check(lib.vlbo_lattice(q, c.ctypes.data_as(C.POINTER(C.c_int32)), _dp(w), C.byref(t0)),
           "lattice")
    return c, w, t0.value


def position(mesh, p):
    lib = load()
    m, keep = _mesh_struct(mesh)
    pp = (C.c_int64 * 3)(*[int(v) for v in p])
    out = np.zeros(3)
    _check(lib.vlbo_position(C.byref(m), pp, _dp(out)), "position")
    return out


def _cell_dict(cell, q):
    d = {"J": cell.J}
    for name in ("g_low", "g_up", "gij", "ginv", "uw"):
        d[name] = np.array([[v for v in row] for row in getattr(cell, name)])
    d["theta"] = np.array([[[v for v in r] for r in m] for m in cell.theta])[:q]
    d["wall_link"] = np.array(list(cell.wall_link))[:q]
    d["uw"] = d["uw"][:q]
    d["G"] = np.array(list(cell.G))
    d["_struct"] = cell
    return d


def cell_geometry(mesh, qi, params=None):
    """Geometry of one in-domain cell qi (section 2.1)."""
    lib = load()
    m, keep = _mesh_struct(mesh)
    pp = (C.c_int64 * 3)(*[int(v) for v in qi])
    cell = _Cell()
    pr = _params_struct(params) if params is not None else None
    _check(lib.vlbo_cell_geometry(C.byref(m), C.byref(pr) if pr is not None else None, pp,
                                  C.byref(cell)), "cell_geometry")
    return _cell_dict(cell, int(mesh["q"]))


def equilibrium(q, rho, U, Ut, ginv):
    lib = load()
    U3 = np.zeros(3)
    Ut3 = np.zeros(3)
    U3[:len(U)] = U
    Ut3[:len(Ut)] = Ut
    g = np.zeros((3, 3))
    gi = np.asarray(ginv, dtype=np.float64)
    g[:gi.shape[0], :gi.shape[1]] = gi
    g = np.ascontiguousarray(g)
    feq = np.zeros(q)
    _check(lib.vlbo_equilibrium(q, float(rho), _dp(U3), _dp(Ut3), _dp(g), _dp(feq)),
           "equilibrium")
    return feq


def collide(q, cell, params, N):
    """One collision of arrived populations N at a cell; returns a dict."""
    lib = load()
    p = _params_struct(params)
    N = np.ascontiguousarray(N, dtype=np.float64)
    out = {k: np.zeros(q) for k in ("Np", "feq", "dN", "Om")}
    F = np.zeros(3)
    dPi = np.zeros(9)
    it = C.c_int32()
    _check(lib.vlbo_collide(q, C.byref(cell["_struct"]), C.byref(p), _dp(N), _dp(out["Np"]),
                            _dp(F), _dp(out["feq"]), _dp(dPi), _dp(out["dN"]), _dp(out["Om"]),
                            C.byref(it)), "collide")
    out["F"] = F
    out["dPi"] = dPi.reshape(3, 3)
    out["iters"] = it.value
    return out


class OracleSim:
    """Whole-mesh FP64 simulation: geometry, init, step, moments."""

    def __init__(self, mesh, params, lib=None):
        self.lib = load() if lib is None else lib
        self.mesh = mesh
        self.q = int(mesh["q"])
        self.dim = int(mesh["dim"])
        self.n = tuple(int(v) for v in mesh["n"])
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        m, keep = _mesh_struct(mesh)
        p = _params_struct(params)
        h = C.c_void_p()
        _check(self.lib.vlbo_create(C.byref(m), C.byref(p), C.byref(h)), "create")
        self.h = h

    def close(self):
        if self.h:
            self.lib.vlbo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho, u):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        assert rho.size == self.ncell and u.size == self.ncell * self.dim
        _check(self.lib.vlbo_init(self.h, _dp(rho), _dp(u)), "init")

    def step(self, n=1):
        _check(self.lib.vlbo_step(self.h, int(n)), "step")

    def moments(self):
        rho = np.zeros(self.ncell)
        u = np.zeros((self.ncell, self.dim))
        ut = np.zeros((self.ncell, self.dim))
        F = np.zeros((self.ncell, self.dim))
        tot = np.zeros(7)
        _check(self.lib.vlbo_moments(self.h, _dp(rho), _dp(u), _dp(ut), _dp(F), _dp(tot)),
               "moments")
        return {"rho": rho, "u": u, "u_tilde": ut, "F": F, "mass": tot[0],
                "P": tot[1:1 + self.dim], "M": tot[4:4 + self.dim]}

    def get_state(self):
        N = np.zeros((self.q, self.ncell))
        _check(self.lib.vlbo_get_state(self.h, _dp(N)), "get_state")
        return N

    def set_state(self, N):
        N = np.ascontiguousarray(N, dtype=np.float64)
        assert N.size == self.q * self.ncell
        _check(self.lib.vlbo_set_state(self.h, _dp(N)), "set_state")

    def cell(self, idx):
        cell = _Cell()
        _check(self.lib.vlbo_get_cell(self.h, int(idx), C.byref(cell)), "get_cell")
        return _cell_dict(cell, self.q)

    def geometry(self):
        """Per-cell arrays J, g_low, ginv, theta, wall_link (for parity tests)."""
        J = np.zeros(self.ncell)
        gl = np.zeros((self.ncell, 3, 3))
        gi = np.zeros((self.ncell, 3, 3))
        th = np.zeros((self.ncell, self.q, 3, 3))
        wl = np.zeros((self.ncell, self.q), dtype=np.int32)
        for k in range(self.ncell):
            c = self.cell(k)
            J[k] = c["J"]
            gl[k] = c["g_low"]
            gi[k] = c["ginv"]
            th[k] = c["theta"]
            wl[k] = c["wall_link"]
        return {"J": J, "g_low": gl, "ginv": gi, "theta": th, "wall_link": wl}

    def last_iters(self):
        return int(self.lib.vlbo_last_iters(self.h))
