"""ctypes front end of the FP64 CPU oracle (oracle/txgel_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the benchmark's CPU
baseline leg, never by the library.  It builds the oracle with the host C++ compiler (no CUDA).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "txgel_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "libtxgel_oracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_MESH_INVERTED", 4: "ERR_INFEASIBLE",
          5: "ERR_NEWTON_MAXIT", 6: "ERR_PCG_MAXIT", 7: "ERR_LINESEARCH", 8: "ERR_CCD_MAXIT"}


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build (plain g++, -O2, portable flags; OpenMP when the
    compiler has it -- the parallel loops give bitwise the same results as one thread)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        base = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.check_call(base + ["-Wno-unknown-pragmas"])
        os.replace(tmp, _OUT)
    return _OUT


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's parallel loops (0: all host cores); returns the count in use.
    The results are bitwise independent of it."""
    L = lib()
    L.or_set_threads(int(n))
    return int(L.or_get_threads())


def threads() -> int:
    return int(lib().or_get_threads())


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(L):
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    L.or_create.restype = ctypes.c_void_p
    L.or_create.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip, u8p, ctypes.c_double,
                            ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, ctypes.c_int, ip,
                            dp, dp, ip, ip]
    L.or_destroy.argtypes = [ctypes.c_void_p]
    L.or_step.restype = ctypes.c_int
    L.or_step.argtypes = [ctypes.c_void_p, dp, ctypes.c_double, ip, dp]
    L.or_get_state.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
    L.or_set_state.argtypes = [ctypes.c_void_p, dp, dp, dp]
    L.or_reset.argtypes = [ctypes.c_void_p]
    L.or_info.argtypes = [ctypes.c_void_p, dp, ip]
    L.or_mass.argtypes = [ctypes.c_void_p, dp]
    L.or_energy.restype = ctypes.c_double
    L.or_energy.argtypes = [ctypes.c_void_p, dp, dp, ctypes.c_double, dp, dp]
    L.or_gradient.restype = ctypes.c_int
    L.or_gradient.argtypes = [ctypes.c_void_p, dp, dp, ctypes.c_double, dp, dp, dp, ctypes.c_int,
                              ctypes.c_int, ip, ip, dp]
    L.or_tet.restype = ctypes.c_int
    L.or_tet.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp, dp]
    L.or_psi.restype = ctypes.c_int
    L.or_psi.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
    L.or_distance2.restype = ctypes.c_double
    L.or_distance2.argtypes = [ctypes.c_int, dp, ip]
    L.or_pair_barrier.restype = ctypes.c_int
    L.or_pair_barrier.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  dp, dp, dp]
    L.or_accd.restype = ctypes.c_int
    L.or_accd.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
    L.or_psd_project.argtypes = [ctypes.c_int, dp]
    L.or_eigh.argtypes = [ctypes.c_int, dp, dp, dp]
    L.or_pcg_csr.restype = ctypes.c_int
    L.or_pcg_csr.argtypes = [ctypes.c_int, ip, ip, dp, dp, dp, ctypes.c_double, ctypes.c_int]
    L.or_pair_counts.argtypes = [ctypes.c_void_p, dp, dp, ip]
    L.or_components.restype = ctypes.c_int
    L.or_components.argtypes = [ctypes.c_void_p, ip]
    L.or_set_friction.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
    L.or_step_attached.restype = ctypes.c_int
    L.or_step_attached.argtypes = [ctypes.c_void_p, dp, dp, ctypes.c_double, ip, dp]
    L.or_set_case_pose.argtypes = [ctypes.c_void_p, dp]
    L.or_markers.argtypes = [ctypes.c_void_p, dp, ctypes.c_int, dp, dp, ip]
    L.or_height_map.argtypes = [ctypes.c_void_p, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, dp]
    L.or_stationary_rule.restype = ctypes.c_int
    L.or_stationary_rule.argtypes = [ctypes.c_double, ctypes.c_double]
    L.or_last_stationary.restype = ctypes.c_int
    L.or_last_stationary.argtypes = [ctypes.c_void_p]
    L.or_last_kappa_doublings.restype = ctypes.c_int
    L.or_last_kappa_doublings.argtypes = [ctypes.c_void_p]
    L.or_kappa.restype = ctypes.c_double
    L.or_kappa.argtypes = [ctypes.c_void_p]
    L.or_set_kappa_adapt.restype = None
    L.or_set_kappa_adapt.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
    L.or_set_threads.argtypes = [ctypes.c_int]
    L.or_get_threads.restype = ctypes.c_int
    L.or_friction_pair.restype = ctypes.c_int
    L.or_friction_pair.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
    return L


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__(STATUS.get(status, str(status)))
        self.status = status


class OracleGel:
    """One gel + indenter scene held by the oracle."""

    def __init__(self, verts, tets, dirichlet, material, ind_verts, ind_tris, pose0, dhat=1e-4,
                 kappa=0.0, newton_tol=1e-5, pcg_tol=1e-10, gravity=(0.0, 0.0, 0.0),
                 newton_max=200, pcg_max=200000, ls_max=80, accd_max=1000000, split_depth=4,
                 friction=0.0, eps_v=1e-3, kappa_adapt_max=0.0, kappa_adapt_dmin=0.0):
        L = lib()
        self.N = int(len(verts))
        self.M = int(len(ind_verts))
        self._keep = []
        X, Xp = _d(verts)
        T, Tp = _i(tets)
        D = np.ascontiguousarray(dirichlet, dtype=np.uint8)
        IV, IVp = _d(ind_verts if len(ind_verts) else np.zeros((0, 3)))
        IT, ITp = _i(ind_tris if len(ind_tris) else np.zeros((0, 3)))
        P0, P0p = _d(pose0)
        fp, fpp = _d([dhat, kappa, newton_tol, pcg_tol, *gravity])
        ipar, ipp = _i([newton_max, pcg_max, ls_max, accd_max, split_depth])
        st = ctypes.c_int(0)
        self._h = L.or_create(self.N, Xp, len(T), Tp, D.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                              material[0], material[1], material[2], self.M, IVp, len(IT), ITp, P0p,
                              fpp, ipp, ctypes.byref(st))
        if not self._h:
            raise OracleError(st.value)
        if friction > 0.0:  # IPC lagged friction (coefficient, velocity threshold [m/s])
            L.or_set_friction(self._h, float(friction), float(eps_v))
        if kappa_adapt_max > 0.0:  # adaptive kappa: cap (multiple of kappa0), threshold distance [m]
            L.or_set_kappa_adapt(self._h, float(kappa_adapt_max), float(kappa_adapt_dmin))

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(wl.gel.verts, wl.gel.tets, wl.gel.dirichlet, wl.material, wl.indenter.verts,
                   wl.indenter.tris, wl.pose0, dhat=wl.dhat, newton_tol=kw.pop("newton_tol", wl.newton_tol),
                   **kw)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def step(self, pose, dt):
        P, Pp = _d(pose)
        stats = np.zeros(5, dtype=np.int32)
        fst = np.zeros(2)
        s = lib().or_step(self._h, Pp, float(dt), stats.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          fst.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        info = dict(status=s, newton_iters=int(stats[0]), pcg_iters=int(stats[1]),
                    ls_halvings=int(stats[2]), substeps=int(stats[3]), active_pairs=int(stats[4]),
                    energy=float(fst[0]), min_distance=float(fst[1]),
                    stationary=int(lib().or_last_stationary(self._h)),
                    kappa_doublings=int(lib().or_last_kappa_doublings(self._h)),
                    kappa=float(lib().or_kappa(self._h)))
        return info

    def step_attached(self, pose, case_pose, dt):
        """One step with the indenter driven to `pose` and the attached (Dirichlet) vertices driven
        with their frame to `case_pose` (their rest positions carried by it)."""
        P, Pp = _d(pose)
        C, Cp = _d(case_pose)
        stats = np.zeros(5, dtype=np.int32)
        fst = np.zeros(2)
        s = lib().or_step_attached(self._h, Pp, Cp, float(dt), stats.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   fst.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return dict(status=s, newton_iters=int(stats[0]), pcg_iters=int(stats[1]),
                    ls_halvings=int(stats[2]), substeps=int(stats[3]), active_pairs=int(stats[4]),
                    energy=float(fst[0]), min_distance=float(fst[1]))

    def markers(self, x, rest_xy):
        """Positions of markers placed at rest points (x, y) of the top surface, carried by the gel
        at positions x; and whether each lies on the top."""
        x, xp = _d(x)
        r, rp = _d(rest_xy)
        n = len(r)
        out = np.zeros((n, 3))
        found = np.zeros(n, dtype=np.int32)
        lib().or_markers(self._h, xp, n, rp, _d(out)[1], found.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return out, found.astype(bool)

    def height_map(self, x, nx, ny, x0, y0, dx, dy):
        """Top-surface height at pixel centres (x0 + (i + 1/2) dx, y0 + (j + 1/2) dy), ny x nx,
        NaN off the gel."""
        x, xp = _d(x)
        out = np.zeros((ny, nx))
        lib().or_height_map(self._h, xp, int(nx), int(ny), float(x0), float(y0), float(dx), float(dy), _d(out)[1])
        return out

    def state(self):
        x = np.zeros((self.N, 3))
        v = np.zeros((self.N, 3))
        fc = np.zeros(3)
        pose = np.zeros(7)
        lib().or_get_state(self._h, _d(x)[1], _d(v)[1], _d(fc)[1], _d(pose)[1])
        return x, v, fc, pose

    def set_state(self, x, v, pose):
        x, xp = _d(x)
        v, vp = _d(v)
        pose, pp = _d(pose)
        lib().or_set_state(self._h, xp, vp, pp)

    def reset(self):
        lib().or_reset(self._h)

    def info(self):
        f = np.zeros(5)
        c = np.zeros(4, dtype=np.int32)
        lib().or_info(self._h, _d(f)[1], c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return dict(mu=f[0], lam=f[1], kappa=f[2], bbox_diag=f[3], total_mass=f[4],
                    surf_verts=int(c[0]), surf_tris=int(c[1]), surf_edges=int(c[2]),
                    ind_edges=int(c[3]))

    def mass(self):
        m = np.zeros(self.N)
        lib().or_mass(self._h, _d(m)[1])
        return m

    def energy(self, x, xt, h, pose):
        parts = np.zeros(5)
        x, xp = _d(x)
        xt, xtp = _d(xt)
        P, Pp = _d(pose)
        e = lib().or_energy(self._h, xp, xtp, float(h), Pp, _d(parts)[1])
        return e, dict(inertia=parts[0], elastic=parts[1], barrier=parts[2], min_d=parts[3],
                       active=int(parts[4]))

    def gradient(self, x, xt, h, pose, hessian=False, project=True):
        x, xp = _d(x)
        xt, xtp = _d(xt)
        P, Pp = _d(pose)
        g = np.zeros(3 * self.N)
        fc = np.zeros(3)
        if not hessian:
            lib().or_gradient(self._h, xp, xtp, float(h), Pp, _d(g)[1], _d(fc)[1], int(project), 0,
                              None, None, None)
            return g.reshape(-1, 3), fc
        cap = 200 * 9 * self.N
        r = np.zeros(cap, dtype=np.int32)
        c = np.zeros(cap, dtype=np.int32)
        v = np.zeros(cap)
        n = lib().or_gradient(self._h, xp, xtp, float(h), Pp, _d(g)[1], _d(fc)[1], int(project),
                              cap, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                              c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(v)[1])
        assert n >= 0
        return g.reshape(-1, 3), fc, (r[:n].copy(), c[:n].copy(), v[:n].copy())

    def pair_counts(self, x, pose):
        """Candidate pairs of each type (PT, TP, EE, SPT, SEE), then the active ones (d < d_hat)."""
        c = np.zeros(10, dtype=np.int32)
        x, xp = _d(x)
        pose, pp = _d(pose)
        lib().or_pair_counts(self._h, xp, pp, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return c

    def components(self):
        """(number of connected components of the tet mesh, component of each vertex)."""
        n = lib().or_components(self._h, None)
        comp = np.zeros(self.N, dtype=np.int32)
        lib().or_components(self._h, comp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return n, comp


# ---- unit-level helpers ----
def tet(X, x, mu, lam, project=True, derivs=True):
    e = ctypes.c_double(0.0)
    g = np.zeros(12)
    H = np.zeros(144)
    X, Xp = _d(X)
    x, xp = _d(x)
    s = lib().or_tet(Xp, xp, mu, lam, int(project), ctypes.byref(e),
                     _d(g)[1] if derivs else None, _d(H)[1] if derivs else None)
    return s, e.value, g, H.reshape(12, 12)


def psi(F, mu, lam):
    p = ctypes.c_double(0.0)
    P = np.zeros(9)
    C = np.zeros(81)
    F, Fp = _d(F)
    s = lib().or_psi(Fp, mu, lam, ctypes.byref(p), _d(P)[1], _d(C)[1])
    return s, p.value, P.reshape(3, 3), C.reshape(9, 9)


def distance2(kind, P):
    t = np.zeros(5, dtype=np.int32)
    P, Pp = _d(P)
    d2 = lib().or_distance2(int(kind), Pp, t.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return d2, tuple(int(v) for v in t)


def pair_barrier(kind, P, dhat, eps_x=0.0, free_mask=0):
    b = ctypes.c_double(0.0)
    g = np.zeros(12)
    H = np.zeros(144)
    P, Pp = _d(P)
    s = lib().or_pair_barrier(int(kind), Pp, dhat, eps_x, int(free_mask), ctypes.byref(b),
                              _d(g)[1], _d(H)[1])
    return s, b.value, g, H.reshape(12, 12)


def accd(kind, P, dP, s=0.1, tc=1.0, maxit=1000000):
    t = ctypes.c_double(1.0)
    P, Pp = _d(P)
    dP, dPp = _d(dP)
    r = lib().or_accd(int(kind), Pp, dPp, s, tc, maxit, ctypes.byref(t))
    return r, t.value


def friction_pair(kind, Plag, Pnow, dhat, kappa, eps_x, mu, eh):
    """Lagged friction of one pair (IPC, Li et al. 2020 Sec. 5): set up from the points at the
    step start, evaluated at the current points.  Returns (active, D, dD/dP (12), d2D/dP2 (12x12),
    lagged normal force)."""
    e = ctypes.c_double(0.0)
    lam = ctypes.c_double(0.0)
    g = np.zeros(12)
    H = np.zeros(144)
    Plag, Pl = _d(Plag)
    Pnow, Pn = _d(Pnow)
    a = lib().or_friction_pair(int(kind), Pl, Pn, dhat, kappa, eps_x, mu, eh, ctypes.byref(e), _d(g)[1],
                               _d(H)[1], ctypes.byref(lam))
    return a, e.value, g, H.reshape(12, 12), lam.value


def stationary_rule(gp, E):
    """True if a failed line search with model decrease -gp at energy E ends the solve as
    converged (stationary to FP64 energy resolution), False if the step fails."""
    return bool(lib().or_stationary_rule(float(gp), float(E)))


def psd_project(A):
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    lib().or_psd_project(n, _d(A)[1])
    return A


def eigh(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n))
    lib().or_eigh(n, _d(A)[1], _d(w)[1], _d(V)[1])
    return w, V


def pcg_csr(indptr, indices, data, b, tol=1e-12, maxit=100000):
    n = len(indptr) - 1
    x = np.zeros(n)
    indptr, ipp = _i(indptr)
    indices, iip = _i(indices)
    data, dp = _d(data)
    b, bp = _d(b)
    it = lib().or_pcg_csr(n, ipp, iip, dp, bp, _d(x)[1], tol, maxit)
    return it, x
