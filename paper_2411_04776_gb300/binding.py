"""Thin ctypes binding of the C ABI in include/tx_gel.h (libtxgel.so).

Argument marshalling only: every step of the solve runs in the CUDA library.  Functions keep the
C names (tx_gel_create, tx_gel_step, tx_gel_state, ...).  Arrays are numpy (host) or torch CUDA
tensors (device pointers); PyTorch supplies device memory and the CUDA stream.  The library is
loaded lazily; if it is missing the first call raises (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libtxgel.so")

TX_OK = 0
STATUS_NAMES = {0: "TX_OK", 1: "TX_ERR_ARG", 2: "TX_ERR_OOM", 3: "TX_ERR_MESH_INVERTED",
                4: "TX_ERR_INFEASIBLE", 5: "TX_ERR_NEWTON_MAXIT", 6: "TX_ERR_PCG_MAXIT",
                7: "TX_ERR_LINESEARCH", 8: "TX_ERR_CCD_MAXIT", 9: "TX_ERR_CUDA",
                10: "TX_ERR_DEVICE_TIMEOUT"}
TX_PREC_FP64 = 0
TX_PREC_MIXED = 1

c_dp = ctypes.POINTER(ctypes.c_double)
c_ip = ctypes.POINTER(ctypes.c_int32)


class tx_params(ctypes.Structure):
    _fields_ = [("dhat", ctypes.c_double), ("kappa", ctypes.c_double), ("newton_tol", ctypes.c_double),
                ("pcg_rel_tol", ctypes.c_double), ("pcg_rel_tol_far", ctypes.c_double),
                ("gravity", ctypes.c_double * 3),
                ("newton_max_iter", ctypes.c_int32), ("pcg_max_iter", ctypes.c_int32),
                ("ls_max_halvings", ctypes.c_int32), ("accd_max_iter", ctypes.c_int32),
                ("max_split_depth", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("refine_max", ctypes.c_int32), ("pcg_cta_slices", ctypes.c_int32),
                ("pcg_plan", ctypes.c_int32), ("pcg_coarse_off", ctypes.c_int32),
                ("friction", ctypes.c_double), ("friction_eps_v", ctypes.c_double),
                ("kappa_adapt_max", ctypes.c_double), ("kappa_adapt_dmin", ctypes.c_double)]


class tx_gel_desc(ctypes.Structure):
    _fields_ = [("n_verts", ctypes.c_int32), ("verts", c_dp), ("n_tets", ctypes.c_int32),
                ("tets", c_ip), ("dirichlet", ctypes.POINTER(ctypes.c_uint8)),
                ("young", ctypes.c_double), ("poisson", ctypes.c_double), ("density", ctypes.c_double),
                ("n_ind_verts", ctypes.c_int32), ("ind_verts", c_dp), ("n_ind_tris", ctypes.c_int32),
                ("ind_tris", c_ip), ("ind_pose", ctypes.c_double * 7), ("params", tx_params)]


class tx_step_stats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int32), ("pcg_iters", ctypes.c_int32),
                ("ls_halvings", ctypes.c_int32), ("substeps", ctypes.c_int32),
                ("active_pairs", ctypes.c_int32), ("candidate_pairs", ctypes.c_int32),
                ("refine_rounds", ctypes.c_int32), ("status", ctypes.c_int32),
                ("energy", ctypes.c_double), ("min_distance", ctypes.c_double),
                ("contact_force", ctypes.c_double * 3), ("mean_position", ctypes.c_double * 3),
                ("kappa", ctypes.c_double), ("soft_pairs_cut", ctypes.c_int32), ("reserved1", ctypes.c_int32)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k in ("contact_force", "mean_position") else getattr(self, k))
                for k, _ in self._fields_}


PROFILE_MAX = 12


class tx_profile(ctypes.Structure):
    _fields_ = [("n_phases", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("names", ctypes.c_char_p * PROFILE_MAX), ("ms", ctypes.c_double * PROFILE_MAX),
                ("launches", ctypes.c_int64 * PROFILE_MAX), ("flops", ctypes.c_double * PROFILE_MAX),
                ("bytes", ctypes.c_double * PROFILE_MAX), ("pcg_iters", ctypes.c_int64),
                ("newton_iters", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("pcg_resident_launches", ctypes.c_int64), ("pcg_streaming_launches", ctypes.c_int64),
                ("pcg_pool_launches", ctypes.c_int64)]

    def as_dict(self):
        phases = {}
        for k in range(self.n_phases):
            phases[self.names[k].decode()] = dict(ms=self.ms[k], launches=int(self.launches[k]),
                                                  flops=self.flops[k], bytes=self.bytes[k])
        return dict(phases=phases, pcg_iters=int(self.pcg_iters), newton_iters=int(self.newton_iters),
                    kernel_launches=int(self.kernel_launches),
                    pcg_resident_launches=int(self.pcg_resident_launches),
                    pcg_streaming_launches=int(self.pcg_streaming_launches),
                    pcg_pool_launches=int(self.pcg_pool_launches))


class TxError(RuntimeError):
    def __init__(self, status, where=""):
        msg = f"{where}: {STATUS_NAMES.get(status, status)}"
        if status == 9 and _lib_obj is not None:
            msg += " (" + _lib_obj.tx_last_error().decode() + ")"
        super().__init__(msg)
        self.status = status


_lock = threading.Lock()
_lib_obj = None

# (name, restype, argtypes)
_SIGS = [
    ("tx_params_default", None, [ctypes.POINTER(tx_params)]),
    ("tx_status_str", ctypes.c_char_p, [ctypes.c_int]),
    ("tx_last_error", ctypes.c_char_p, []),
    ("tx_debug_inject", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32]),
    ("tx_peak_fma", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, c_dp, c_dp, ctypes.c_void_p]),
    ("tx_gel_create", ctypes.c_int, [ctypes.POINTER(tx_gel_desc), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("tx_gel_step", ctypes.c_int, [ctypes.c_void_p, c_dp, ctypes.c_double]),
    ("tx_gel_step_attached", ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, ctypes.c_double]),
    ("tx_gel_case_pose", ctypes.c_int, [ctypes.c_void_p, c_dp]),
    ("tx_gel_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, c_dp,
                                    ctypes.POINTER(tx_step_stats), ctypes.c_int32]),
    ("tx_gel_get_state", ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, c_dp]),
    ("tx_gel_set_state", ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, c_dp]),
    ("tx_gel_reset", ctypes.c_int, [ctypes.c_void_p]),
    ("tx_gel_destroy", None, [ctypes.c_void_p]),
    ("tx_gel_footprint_bytes", ctypes.c_size_t, [ctypes.POINTER(tx_gel_desc)]),
    ("tx_gel_energy", ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, ctypes.c_double, c_dp, c_dp, c_dp]),
    ("tx_gel_gradient", ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, ctypes.c_double, c_dp, c_dp, c_dp]),
    ("tx_batch_create", ctypes.c_int, [ctypes.POINTER(tx_gel_desc), ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    ("tx_batch_destroy", None, [ctypes.c_void_p]),
    ("tx_batch_size", ctypes.c_int32, [ctypes.c_void_p]),
    ("tx_batch_step", ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, c_ip]),
    ("tx_batch_step_attached", ctypes.c_int, [ctypes.c_void_p, c_dp, c_dp, c_dp, c_ip]),
    ("tx_gel_markers", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_dp, c_dp, c_ip]),
    ("tx_batch_markers", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, c_dp, c_dp, c_ip]),
    ("tx_gel_height_map", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double, c_dp]),
    ("tx_batch_height_map", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, c_dp]),
    ("tx_batch_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_ip, c_dp, c_dp]),
    ("tx_batch_advance", ctypes.c_int, [ctypes.c_void_p, c_ip, c_ip, c_ip]),
    ("tx_batch_pending", ctypes.c_int32, [ctypes.c_void_p]),
    ("tx_batch_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_dp, c_dp, c_dp,
                                      ctypes.POINTER(tx_step_stats)]),
    ("tx_batch_set_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_dp, c_dp, c_dp]),
    ("tx_batch_reset", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("tx_batch_profile", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(tx_profile)]),
    ("tx_gel_profile", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(tx_profile)]),
    ("tx_bsr_pcg", ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, c_ip,
                                  c_dp, ctypes.c_void_p]),
    ("tx_bsr_pcg_noalloc", ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int32,
                                          c_ip, c_dp, ctypes.c_void_p]),
    ("tx_eval_tets", ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    ("tx_eval_pairs", ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("tx_eval_accd", ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
]
EXPORTED = [s[0] for s in _SIGS]


def load(path: str = LIB_PATH):
    """Load libtxgel.so (raises if it was not built)."""
    global _lib_obj
    with _lock:
        if _lib_obj is None:
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library missing: {path} (run __graft_entry__.build())")
            L = ctypes.CDLL(path)
            for name, res, args in _SIGS:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib_obj = L
    return _lib_obj


def _check(status, where):
    if status != TX_OK:
        raise TxError(status, where)


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(c_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(c_ip)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:  # torch is optional for the binding
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ------------------------------------------------------------------ descriptors
def tx_params_default(**overrides) -> tx_params:
    p = tx_params()
    load().tx_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "gravity":
            p.gravity = (ctypes.c_double * 3)(*v)
        else:
            setattr(p, k, v)
    return p


class GelDesc:
    """Owns the numpy arrays a tx_gel_desc points to."""

    def __init__(self, verts, tets, dirichlet, material, ind_verts, ind_tris, ind_pose, params=None, **kw):
        self.verts, vp = _d(verts)
        self.tets, tp = _i(tets)
        self.dirichlet = None if dirichlet is None else np.ascontiguousarray(dirichlet, dtype=np.uint8)
        self.ind_verts, ivp = _d(ind_verts if len(ind_verts) else np.zeros((0, 3)))
        self.ind_tris, itp = _i(ind_tris if len(ind_tris) else np.zeros((0, 3)))
        self.params = params if params is not None else tx_params_default(**kw)
        d = tx_gel_desc()
        d.n_verts = len(self.verts)
        d.verts = vp
        d.n_tets = len(self.tets)
        d.tets = tp
        d.dirichlet = (self.dirichlet.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
                       if self.dirichlet is not None else ctypes.POINTER(ctypes.c_uint8)())
        d.young, d.poisson, d.density = (float(m) for m in material)
        d.n_ind_verts = len(self.ind_verts)
        d.ind_verts = ivp
        d.n_ind_tris = len(self.ind_tris)
        d.ind_tris = itp
        d.ind_pose = (ctypes.c_double * 7)(*[float(v) for v in ind_pose])
        d.params = self.params
        self.c = d

    @classmethod
    def from_workload(cls, wl, **kw):
        kw.setdefault("dhat", wl.dhat)
        kw.setdefault("newton_tol", wl.newton_tol)
        return cls(wl.gel.verts, wl.gel.tets, wl.gel.dirichlet, wl.material, wl.indenter.verts,
                   wl.indenter.tris, wl.pose0, **kw)


# ------------------------------------------------------------------ C entry points
TX_INJECT_ALLOC_FAIL = 1
TX_INJECT_WAIT_TIMEOUT = 2


def tx_debug_inject(kind, count):
    """Fault-injection test hook (host-side allocation failure, or device waits that give up)."""
    _check(load().tx_debug_inject(int(kind), int(count)), "tx_debug_inject")


def tx_peak_fma(bits=64, iters=20000, stream=None):
    """(flops, ms) of one FMA-peak launch (FP64: bits = 64, FP32: bits = 32)."""
    f = ctypes.c_double(0.0)
    t = ctypes.c_double(0.0)
    _check(load().tx_peak_fma(int(bits), int(iters), ctypes.byref(f), ctypes.byref(t), _stream(stream)),
           "tx_peak_fma")
    return f.value, t.value


def tx_gel_create(desc: GelDesc, stream=None):
    h = ctypes.c_void_p()
    _check(load().tx_gel_create(ctypes.byref(desc.c), _stream(stream), ctypes.byref(h)), "tx_gel_create")
    return h


def tx_gel_step(g, pose, dt) -> int:
    pose, pp = _d(pose)
    return load().tx_gel_step(g, pp, float(dt))


def tx_gel_step_attached(g, pose, case_pose, dt) -> int:
    pose, pp = _d(pose)
    case_pose, cp = _d(case_pose)
    return load().tx_gel_step_attached(g, pp, cp, float(dt))


def tx_gel_case_pose(g):
    out = np.zeros(7)
    _check(load().tx_gel_case_pose(g, _d(out)[1]), "tx_gel_case_pose")
    return out


def tx_gel_markers(g, rest_xy):
    """Markers at rest points (n x 2) of the top surface carried to the current state: (n x 3, found)."""
    rest_xy, rp = _d(rest_xy)
    n = len(rest_xy)
    out = np.zeros((n, 3))
    found = np.zeros(n, dtype=np.int32)
    _check(load().tx_gel_markers(g, n, rp, _d(out)[1], found.ctypes.data_as(c_ip)), "tx_gel_markers")
    return out, found.astype(bool)


def tx_gel_height_map(g, nx, ny, x0, y0, dx, dy):
    out = np.zeros((ny, nx))
    _check(load().tx_gel_height_map(g, int(nx), int(ny), float(x0), float(y0), float(dx), float(dy), _d(out)[1]),
           "tx_gel_height_map")
    return out


def tx_gel_state(g, n_verts, device_out=None):
    """Returns (x, v, contact force, stats).  With device_out=(x_t, v_t) (torch CUDA tensors of
    shape (n, 3), float64) the copy lands there on the gel's stream."""
    fc = np.zeros(3)
    st = tx_step_stats()
    if device_out is not None:
        xt, vt = device_out
        _check(load().tx_gel_state(g, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(vt.data_ptr()),
                                   _d(fc)[1], ctypes.byref(st), 1), "tx_gel_state")
        return xt, vt, fc, st
    x = np.zeros((n_verts, 3))
    v = np.zeros((n_verts, 3))
    _check(load().tx_gel_state(g, ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(v.ctypes.data),
                               _d(fc)[1], ctypes.byref(st), 0), "tx_gel_state")
    return x, v, fc, st


def tx_gel_get_state(g, n_verts):
    x = np.zeros((n_verts, 3))
    v = np.zeros((n_verts, 3))
    pose = np.zeros(7)
    _check(load().tx_gel_get_state(g, _d(x)[1], _d(v)[1], _d(pose)[1]), "tx_gel_get_state")
    return x, v, pose


def tx_gel_set_state(g, x, v, pose):
    x, xp = _d(x)
    v, vp = _d(v)
    pose, pp = _d(pose)
    _check(load().tx_gel_set_state(g, xp, vp, pp), "tx_gel_set_state")


def tx_gel_reset(g):
    _check(load().tx_gel_reset(g), "tx_gel_reset")


def tx_gel_destroy(g):
    if g:
        load().tx_gel_destroy(g)


def tx_gel_footprint_bytes(desc: GelDesc) -> int:
    return int(load().tx_gel_footprint_bytes(ctypes.byref(desc.c)))


def tx_gel_energy(g, x, xt, h, pose):
    x, xp = _d(x)
    xt, xtp = _d(xt)
    pose, pp = _d(pose)
    e = np.zeros(1)
    parts = np.zeros(5)
    _check(load().tx_gel_energy(g, xp, xtp, float(h), pp, _d(e)[1], _d(parts)[1]), "tx_gel_energy")
    return float(e[0]), dict(inertia=parts[0], elastic=parts[1], barrier=parts[2], min_d=parts[3],
                             active=int(parts[4]))


def tx_gel_gradient(g, x, xt, h, pose):
    x, xp = _d(x)
    xt, xtp = _d(xt)
    pose, pp = _d(pose)
    grad = np.zeros((len(x), 3))
    fc = np.zeros(3)
    _check(load().tx_gel_gradient(g, xp, xtp, float(h), pp, _d(grad)[1], _d(fc)[1]), "tx_gel_gradient")
    return grad, fc


def tx_batch_create(descs, stream=None):
    arr = (tx_gel_desc * len(descs))(*[d.c for d in descs])
    h = ctypes.c_void_p()
    _check(load().tx_batch_create(arr, len(descs), _stream(stream), ctypes.byref(h)), "tx_batch_create")
    return h


def tx_batch_destroy(b):
    if b:
        load().tx_batch_destroy(b)


def tx_batch_size(b) -> int:
    return int(load().tx_batch_size(b))


def tx_batch_step(b, poses, dts):
    poses, pp = _d(poses)
    dts, dp = _d(dts)
    st = np.zeros(len(dts), dtype=np.int32)
    s = load().tx_batch_step(b, pp, dp, st.ctypes.data_as(c_ip))
    return s, st


def tx_batch_step_attached(b, poses, case_poses, dts):
    poses, pp = _d(poses)
    case_poses, cp = _d(case_poses)
    dts, dp = _d(dts)
    st = np.zeros(len(dts), dtype=np.int32)
    s = load().tx_batch_step_attached(b, pp, cp, dp, st.ctypes.data_as(c_ip))
    return s, st


def tx_batch_submit(b, ids, poses, dts):
    ids, ip = _i(ids)
    poses, pp = _d(poses)
    dts, dp = _d(dts)
    _check(load().tx_batch_submit(b, len(ids), ip, pp, dp), "tx_batch_submit")


def tx_batch_advance(b, capacity):
    n = ctypes.c_int32(0)
    ids = np.zeros(capacity, dtype=np.int32)
    st = np.zeros(capacity, dtype=np.int32)
    _check(load().tx_batch_advance(b, ctypes.byref(n), ids.ctypes.data_as(c_ip), st.ctypes.data_as(c_ip)),
           "tx_batch_advance")
    return ids[:n.value].copy(), st[:n.value].copy()


def tx_batch_pending(b) -> int:
    return int(load().tx_batch_pending(b))


def tx_batch_state(b, gel, n_verts):
    x = np.zeros((n_verts, 3))
    v = np.zeros((n_verts, 3))
    fc = np.zeros(3)
    st = tx_step_stats()
    _check(load().tx_batch_state(b, int(gel), _d(x)[1], _d(v)[1], _d(fc)[1], ctypes.byref(st)), "tx_batch_state")
    return x, v, fc, st


def tx_batch_set_state(b, gel, x, v, pose):
    x, xp = _d(x)
    v, vp = _d(v)
    pose, pp = _d(pose)
    _check(load().tx_batch_set_state(b, int(gel), xp, vp, pp), "tx_batch_set_state")


def tx_batch_reset(b, gel):
    _check(load().tx_batch_reset(b, int(gel)), "tx_batch_reset")


def tx_gel_profile(g, enable=True):
    """Returns the per-phase counters since the previous call and sets profiling on/off."""
    p = tx_profile()
    _check(load().tx_gel_profile(g, int(enable), ctypes.byref(p)), "tx_gel_profile")
    return p.as_dict()


def tx_batch_profile(b, enable=True):
    p = tx_profile()
    _check(load().tx_batch_profile(b, int(enable), ctypes.byref(p)), "tx_batch_profile")
    return p.as_dict()


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def tx_eval_tets(X, x, mu, lam, project=True, stream=None, want_hessian=True):
    """Per-tet energy / gradient / Hessian on the GPU (torch CUDA float64 tensors (n, 12))."""
    import torch
    n = X.shape[0]
    dev = X.device
    e = torch.empty(n, dtype=torch.float64, device=dev)
    g = torch.empty(n, 12, dtype=torch.float64, device=dev)
    H = torch.empty(n, 144, dtype=torch.float64, device=dev) if want_hessian else None
    _check(load().tx_eval_tets(n, _ptr(X), _ptr(x), mu, lam, int(project), _ptr(e), _ptr(g), _ptr(H),
                               _stream(stream)), "tx_eval_tets")
    return e, g, H


def tx_eval_pairs(kind, P, dhat, eps_x=None, free_mask=None, stream=None):
    import torch
    n = P.shape[0]
    dev = P.device
    b = torch.empty(n, dtype=torch.float64, device=dev)
    g = torch.empty(n, 12, dtype=torch.float64, device=dev)
    H = torch.empty(n, 144, dtype=torch.float64, device=dev)
    dt = torch.empty(n, 5, dtype=torch.int32, device=dev)
    _check(load().tx_eval_pairs(n, _ptr(kind), _ptr(P), float(dhat), _ptr(eps_x), _ptr(free_mask), _ptr(b),
                                _ptr(g), _ptr(H), _ptr(dt), _stream(stream)), "tx_eval_pairs")
    return b, g, H, dt


def tx_eval_accd(kind, P, dP, s=0.1, tc=1.0, max_iter=1000000, stream=None):
    import torch
    n = P.shape[0]
    toi = torch.empty(n, dtype=torch.float64, device=P.device)
    hit = torch.empty(n, dtype=torch.int32, device=P.device)
    _check(load().tx_eval_accd(n, _ptr(kind), _ptr(P), _ptr(dP), float(s), float(tc), int(max_iter), _ptr(toi),
                               _ptr(hit), _stream(stream)), "tx_eval_accd")
    return toi, hit


def tx_bsr_pcg(row_ptr, col_idx, vals, b, rel_tol=1e-10, max_iter=10000, stream=None):
    """Block-Jacobi PCG on a 3x3-block CSR system (torch CUDA tensors: int32 row_ptr/col_idx,
    float64 vals (nnzb, 9) and b (3n)).  Returns (x, iterations, relative residual)."""
    import torch
    n = row_ptr.numel() - 1
    x = torch.empty(3 * n, dtype=torch.float64, device=b.device)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    _check(load().tx_bsr_pcg(n, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(b), _ptr(x), float(rel_tol),
                             int(max_iter), ctypes.byref(it), ctypes.byref(rr), _stream(stream)), "tx_bsr_pcg")
    return x, it.value, rr.value


def tx_bsr_pcg_noalloc(row_ptr, col_idx, vals, b, x=None, rel_tol=1e-10, max_iter=10000, stream=None):
    """tx_bsr_pcg with the library's fixed scratch array (no device allocation by the library;
    the output x may be passed in preallocated).  n <= 65536 block rows."""
    import torch
    n = row_ptr.numel() - 1
    if x is None:
        x = torch.empty(3 * n, dtype=torch.float64, device=b.device)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    _check(load().tx_bsr_pcg_noalloc(n, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(b), _ptr(x),
                                     float(rel_tol), int(max_iter), ctypes.byref(it), ctypes.byref(rr),
                                     _stream(stream)), "tx_bsr_pcg_noalloc")
    return x, it.value, rr.value


# ------------------------------------------------------------------ convenience wrapper
class Gel:
    """One gel + indenter scene on the GPU (wraps a tx_gel handle)."""

    def __init__(self, desc: GelDesc, stream=None):
        self.desc = desc
        self.n = desc.c.n_verts
        self.h = tx_gel_create(desc, stream)

    @classmethod
    def from_workload(cls, wl, stream=None, **kw):
        return cls(GelDesc.from_workload(wl, **kw), stream)

    def step(self, pose, dt):
        s = tx_gel_step(self.h, pose, dt)
        return s

    def step_attached(self, pose, case_pose, dt):
        return tx_gel_step_attached(self.h, pose, case_pose, dt)

    def case_pose(self):
        return tx_gel_case_pose(self.h)

    def markers(self, rest_xy):
        return tx_gel_markers(self.h, rest_xy)

    def height_map(self, nx, ny, x0, y0, dx, dy):
        return tx_gel_height_map(self.h, nx, ny, x0, y0, dx, dy)

    def state(self):
        return tx_gel_state(self.h, self.n)

    def stats(self):
        return self.state()[3].as_dict()

    def set_state(self, x, v, pose):
        tx_gel_set_state(self.h, x, v, pose)

    def get_state(self):
        return tx_gel_get_state(self.h, self.n)

    def reset(self):
        tx_gel_reset(self.h)

    def profile(self, enable=True):
        return tx_gel_profile(self.h, enable)

    def energy(self, x, xt, h, pose):
        return tx_gel_energy(self.h, x, xt, h, pose)

    def gradient(self, x, xt, h, pose):
        return tx_gel_gradient(self.h, x, xt, h, pose)

    def close(self):
        if getattr(self, "h", None):
            tx_gel_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
