"""Thin ctypes binding of ``libngravs.so`` (declared in ``include/ngravs.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library. Functions keep the C names. Particle arrays are torch CUDA tensors
laid out as the header states (positions float64 [3, n], accelerations and
velocities float32 [3, n], species uint8 [n], masses float32 [n]); their
device pointers are handed to the library as is. The stream is torch's
current stream unless one is given.

There is no fallback: if the library was not built (``__graft_entry__.build()``
or ``python -m paper_1502_07442_gb300.build``), loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

NG_MAX_SPECIES = 6
NG_OK, NG_EINVAL, NG_ENOMEM, NG_ECUDA, NG_ETIMEOUT, NG_EBUSY, NG_ESTATE = 0, -1, -2, -3, -4, -5, -6
NG_NEWTON, NG_YUKAWA, NG_YUKAWA_PURE, NG_MAHALO = 0, 1, 2, 3

_M6d = (ctypes.c_double * NG_MAX_SPECIES) * NG_MAX_SPECIES
_M6i = (ctypes.c_int32 * NG_MAX_SPECIES) * NG_MAX_SPECIES


class NgParams(ctypes.Structure):
    """Mirror of ``ng_params``."""

    _fields_ = [
        ("D", ctypes.c_int32), ("pm_mesh", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
        ("group_size", ctypes.c_int32), ("table_size", ctypes.c_int32),
        ("group_cell", ctypes.c_int32),
        ("G", _M6d), ("law", _M6i), ("yuk_a", _M6d), ("yuk_l", _M6d),
        ("eps", ctypes.c_double), ("box", ctypes.c_double), ("asmth", ctypes.c_double),
        ("rcut_over_rs", ctypes.c_double), ("theta", ctypes.c_double),
        ("opening", ctypes.c_int32), ("reserved1", ctypes.c_int32), ("alpha", ctypes.c_double),
        ("pure_tree", ctypes.c_int32), ("ignore_nperp", ctypes.c_int32), ("beta", ctypes.c_double),
        ("accumulate_fp64", ctypes.c_int32), ("reserved2", ctypes.c_int32),
    ]


NG_REQ_FORCE, NG_REQ_STEPS = 0, 1
NG_OPEN_GEOMETRIC, NG_OPEN_RELATIVE = 0, 1


class NgRequest(ctypes.Structure):
    """Mirror of ``ng_request`` (host arrays given as addresses)."""

    _fields_ = [("kind", ctypes.c_int32), ("nsteps", ctypes.c_int32), ("dt", ctypes.c_double),
                ("params", NgParams), ("n", ctypes.c_int64),
                ("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("type", ctypes.c_void_p),
                ("mass", ctypes.c_void_p), ("pos_out", ctypes.c_void_p),
                ("vel_out", ctypes.c_void_p), ("acc_out", ctypes.c_void_p)]


class NgResult(ctypes.Structure):
    """Mirror of ``ng_result``."""

    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class NgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ngravs error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libngravs.so is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.ng_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(NgParams), vp]
        L.ng_destroy.argtypes = [vp]
        L.ng_set_stream.argtypes = [vp, vp]
        L.ng_build_tree.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.ng_tree_force.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint64)]
        L.ng_count_interactions.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint64)]
        L.ng_set_acc_old.argtypes = [vp, i64, vp]
        L.ng_step_host.argtypes = [vp, i64, vp, vp, vp, vp, vp, i32, i32, d]
        L.ng_timestep.argtypes = [vp, i64, vp, d, d, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_float)]
        L.ng_pm_force.argtypes = [vp, vp]
        L.ng_force.argtypes = [vp, vp]
        L.ng_stage_times.argtypes = [vp, i64, vp, vp, vp, vp, vp, d, vp]
        L.ng_step.argtypes = [vp, i64, vp, vp, vp, vp, vp, i32, i32, d]
        L.ng_tree_export.argtypes = [vp, ctypes.POINTER(i64)] + [vp] * 9
        L.ng_type_order.argtypes = [vp, vp, vp]
        L.ng_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        L.ng_sort_passes.argtypes = [vp, ctypes.POINTER(i32)]
        L.ng_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(NgParams), vp]
        L.ng_batch_destroy.argtypes = [vp]
        L.ng_batch_step.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, i32, d]
        L.ng_batch_size.argtypes = [vp]
        L.ng_batch_walk_launches.argtypes = [vp]
        L.ng_batch_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        L.ng_batch_last_error.argtypes = [vp]
        L.ng_batch_last_error.restype = ctypes.c_char_p
        L.ng_serve_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.c_size_t]
        L.ng_serve_destroy.argtypes = [vp]
        L.ng_serve_submit.argtypes = [vp, ctypes.POINTER(NgRequest), ctypes.POINTER(NgResult),
                                      ctypes.POINTER(i64)]
        L.ng_serve_cancel.argtypes = [vp, i64]
        L.ng_serve_poll.argtypes = [vp, ctypes.POINTER(i32)]
        L.ng_serve_pending.argtypes = [vp]
        L.ng_serve_wait.argtypes = [vp, d]
        L.ng_serve.argtypes = [vp, ctypes.POINTER(NgRequest), ctypes.POINTER(NgResult), i32, vp, d]
        L.ng_sort_keys_noalloc.argtypes = [i64, vp, vp, d, vp, vp, vp]
        L.ng_sort_keys_noalloc.restype = ctypes.c_int
        L.ng_serve_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(i64),
                                     ctypes.POINTER(i64)]
        L.ng_serve_stats.restype = ctypes.c_int
        L.ng_serve_request_bytes.argtypes = [ctypes.POINTER(NgRequest)]
        L.ng_serve_request_bytes.restype = ctypes.c_size_t
        L.ng_serve_last_error.argtypes = [vp]
        L.ng_serve_last_error.restype = ctypes.c_char_p
        L.ng_last_error.argtypes = [vp]
        L.ng_last_error.restype = ctypes.c_char_p
        L.ng_version.restype = ctypes.c_char_p
        for f in ("ng_create", "ng_destroy", "ng_set_stream", "ng_build_tree", "ng_tree_force",
                  "ng_count_interactions", "ng_pm_force", "ng_force", "ng_stage_times", "ng_step",
                  "ng_tree_export",
                  "ng_type_order", "ng_launch_count", "ng_sort_passes", "ng_batch_create",
                  "ng_batch_destroy",
                  "ng_batch_step", "ng_batch_size", "ng_batch_walk_launches",
                  "ng_batch_launch_count", "ng_serve_create", "ng_serve_destroy",
                  "ng_serve_submit", "ng_serve_cancel", "ng_serve_poll", "ng_serve_pending",
                  "ng_serve_wait", "ng_serve", "ng_set_acc_old", "ng_timestep", "ng_step_host"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def exported_symbols():
    """Names the header declares (used by the ABI test)."""
    return ["ng_create", "ng_destroy", "ng_set_stream", "ng_build_tree", "ng_tree_force",
            "ng_count_interactions", "ng_pm_force", "ng_force", "ng_stage_times", "ng_step",
            "ng_tree_export", "ng_type_order",
            "ng_launch_count", "ng_sort_passes", "ng_last_error", "ng_version", "ng_batch_create",
            "ng_batch_destroy", "ng_batch_step", "ng_batch_size", "ng_batch_walk_launches",
            "ng_batch_launch_count", "ng_batch_last_error", "ng_serve_create",
            "ng_serve_destroy", "ng_serve_submit", "ng_serve_cancel", "ng_serve_poll",
            "ng_serve_pending", "ng_serve_wait", "ng_serve", "ng_serve_last_error",
            "ng_serve_request_bytes", "ng_serve_stats", "ng_sort_keys_noalloc", "ng_set_acc_old",
            "ng_timestep", "ng_step_host"]


def _check(ctx, code):
    if code != NG_OK:
        msg = lib().ng_last_error(ctx)
        raise NgError(code, msg.decode() if msg else "")


def make_params(D, G, *, eps, box=1.0, pm_mesh=0, asmth=1.25, rcut_over_rs=4.5, theta=0.5,
                leaf_size=8, group_size=32, table_size=0, law=None, yuk_a=None, yuk_l=None,
                group_cell=0, opening=0, alpha=0.0, pure_tree=0, ignore_nperp=0, beta=0.0,
                accumulate_fp64=0):
    p = NgParams()
    p.D, p.pm_mesh, p.leaf_size, p.group_size, p.table_size = (int(D), int(pm_mesh), int(leaf_size),
                                                               int(group_size), int(table_size))
    p.eps, p.box, p.asmth, p.rcut_over_rs, p.theta = (float(eps), float(box), float(asmth),
                                                      float(rcut_over_rs), float(theta))
    p.group_cell = int(group_cell)
    p.opening, p.reserved1, p.alpha = int(opening), 0, float(alpha)
    p.pure_tree, p.ignore_nperp, p.beta = int(pure_tree), int(ignore_nperp), float(beta)
    p.accumulate_fp64, p.reserved2 = int(accumulate_fp64), 0
    G = np.asarray(G, np.float64)
    law = np.zeros((D, D), np.int32) if law is None else np.asarray(law, np.int32)
    ya = np.zeros((D, D)) if yuk_a is None else np.asarray(yuk_a, np.float64)
    yl = np.ones((D, D)) if yuk_l is None else np.asarray(yuk_l, np.float64)
    for i in range(D):
        for j in range(D):
            p.G[i][j] = G[i, j]
            p.law[i][j] = int(law[i, j])
            p.yuk_a[i][j] = ya[i, j]
            p.yuk_l[i][j] = yl[i, j]
    return p


def params_from_workload(w: dict, **over) -> NgParams:
    """ng_params for a parameter dict from ``inputs.workload``."""
    q = dict(w)
    q.update(over)
    mesh = int(q["pm_mesh"])
    box = float(q["box"])
    rs = float(q["rs"])
    asmth = rs * mesh / box if mesh > 0 else rs / box
    return make_params(q["D"], q["G"], eps=q["eps"], box=box, pm_mesh=mesh, asmth=asmth,
                       rcut_over_rs=float(q["rcut"]) / rs, theta=q["theta"],
                       leaf_size=q.get("leaf_size", 8), law=q["law"], yuk_a=q["ya"], yuk_l=q["yl"],
                       table_size=q.get("table_size", 0), group_cell=q.get("group_cell", 0),
                       opening=q.get("opening", 0), alpha=q.get("alpha", 0.0),
                       pure_tree=q.get("pure_tree", 0), ignore_nperp=q.get("ignore_nperp", 0),
                       beta=q.get("beta", 0.0), accumulate_fp64=q.get("accumulate_fp64", 0))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def ng_create(params: NgParams, stream=None):
    ctx = ctypes.c_void_p()
    _check(None, lib().ng_create(ctypes.byref(ctx), ctypes.byref(params), _stream(stream)))
    return ctx


def ng_destroy(ctx):
    lib().ng_destroy(ctx)


def ng_set_stream(ctx, stream=None):
    _check(ctx, lib().ng_set_stream(ctx, _stream(stream)))


def ng_build_tree(ctx, pos, typ, mass, keys_out=None, perm_out=None):
    n = typ.numel()
    _check(ctx, lib().ng_build_tree(ctx, n, _ptr(pos), _ptr(typ), _ptr(mass), _ptr(keys_out),
                                    _ptr(perm_out)))


def ng_set_acc_old(ctx, acc_old):
    """|a_old| for the relative criterion from a device float32[3][n] tensor."""
    n = acc_old.shape[-1]
    _check(ctx, lib().ng_set_acc_old(ctx, int(n), _ptr(acc_old)))


def ng_timestep(ctx, acc, eta, dt_max):
    """Synchronous step of Eq. (our_timestep); returns (dt, |a|_max)."""
    dt, amax = ctypes.c_double(0.0), ctypes.c_float(0.0)
    _check(ctx, lib().ng_timestep(ctx, int(acc.shape[-1]), _ptr(acc), float(eta), float(dt_max),
                                  ctypes.byref(dt), ctypes.byref(amax)))
    return dt.value, amax.value


def ng_tree_force(ctx, acc_out, count=False):
    v = ctypes.c_uint64(0)
    _check(ctx, lib().ng_tree_force(ctx, _ptr(acc_out), ctypes.byref(v) if count else None))
    return int(v.value) if count else None


def ng_count_interactions(ctx, counts_out=None):
    v = ctypes.c_uint64(0)
    _check(ctx, lib().ng_count_interactions(ctx, _ptr(counts_out), ctypes.byref(v)))
    return int(v.value)


def ng_pm_force(ctx, acc_out):
    _check(ctx, lib().ng_pm_force(ctx, _ptr(acc_out)))


def ng_force(ctx, acc_out):
    """Short-range tree plus long-range PM acceleration, summed in the library."""
    _check(ctx, lib().ng_force(ctx, _ptr(acc_out)))


STAGES = ("keys", "radix", "gather", "octree", "monopoles", "groups", "type_order", "deposit",
          "fft_fwd", "kspace", "fft_inv", "interp", "walk")


def ng_stage_times(ctx, pos, vel, typ, mass, acc, dt):
    """Milliseconds of each stage of one ng_step step (dict); advances the
    state (pos, vel, acc) by three steps."""
    out = (ctypes.c_float * len(STAGES))()
    _check(ctx, lib().ng_stage_times(ctx, typ.numel(), _ptr(pos), _ptr(vel), _ptr(typ), _ptr(mass),
                                     _ptr(acc), float(dt), out))
    return {k: float(v) for k, v in zip(STAGES, out)}


def ng_step(ctx, pos, vel, typ, mass, acc, acc_valid, nsteps, dt):
    n = typ.numel()
    _check(ctx, lib().ng_step(ctx, n, _ptr(pos), _ptr(vel), _ptr(typ), _ptr(mass), _ptr(acc),
                              int(bool(acc_valid)), int(nsteps), float(dt)))


def ng_step_host(ctx, pos, vel, typ, mass, acc, acc_valid, nsteps, dt):
    """ng_step on host tensors/arrays (updated in place); pinned memory copies fastest."""
    n = typ.shape[-1]
    _check(ctx, lib().ng_step_host(ctx, int(n), _ptr(pos), _ptr(vel), _ptr(typ), _ptr(mass),
                                   _ptr(acc), int(bool(acc_valid)), int(nsteps), float(dt)))


def ng_tree_export(ctx, D):
    """Returns a dict of numpy arrays (canonical node order)."""
    nn = ctypes.c_int64(0)
    L = lib()
    _check(ctx, L.ng_tree_export(ctx, ctypes.byref(nn), *([None] * 9)))
    n = nn.value
    out = dict(level=np.zeros(n, np.int32), prefix=np.zeros(n, np.uint64),
               first=np.zeros(n, np.int64), count=np.zeros(n, np.int64),
               nchild=np.zeros(n, np.int32), child_first=np.zeros(n, np.int64),
               cnt=np.zeros((n, D), np.uint32), mass=np.zeros((n, D)), com=np.zeros((n, D, 3)))
    keys = ("level", "prefix", "first", "count", "nchild", "child_first", "cnt", "mass", "com")
    _check(ctx, L.ng_tree_export(ctx, ctypes.byref(nn),
                                 *[out[k].ctypes.data_as(ctypes.c_void_p) for k in keys]))
    return out


def ng_type_order(ctx, D, order_out=None):
    offs = np.zeros(D + 1, np.int64)
    _check(ctx, lib().ng_type_order(ctx, offs.ctypes.data_as(ctypes.c_void_p), _ptr(order_out)))
    return offs


def ng_launch_count(ctx):
    v = ctypes.c_uint64(0)
    _check(ctx, lib().ng_launch_count(ctx, ctypes.byref(v)))
    return int(v.value)


def ng_sort_passes(ctx):
    v = ctypes.c_int32(0)
    _check(ctx, lib().ng_sort_passes(ctx, ctypes.byref(v)))
    return int(v.value)


def _bcheck(b, code):
    if code != NG_OK:
        msg = lib().ng_batch_last_error(b) if b else None
        if not msg:
            msg = lib().ng_last_error(None)
        raise NgError(code, msg.decode() if msg else "")


def ng_batch_create(params_list, stream=None):
    arr = (NgParams * len(params_list))(*params_list)
    b = ctypes.c_void_p()
    _bcheck(None, lib().ng_batch_create(ctypes.byref(b), len(params_list), arr, _stream(stream)))
    return b


def ng_batch_destroy(b):
    lib().ng_batch_destroy(b)


def ng_batch_step(b, pos, vel, typ, mass, acc, acc_valid, nsteps, dt):
    """Each argument is a list of torch CUDA tensors, one per simulation."""
    S = len(pos)
    n = (ctypes.c_int64 * S)(*[t.numel() for t in typ])
    P = lambda ts: (ctypes.c_void_p * S)(*[t.data_ptr() for t in ts])
    _bcheck(b, lib().ng_batch_step(b, n, P(pos), P(vel), P(typ), P(mass), P(acc),
                                   int(bool(acc_valid)), int(nsteps), float(dt)))


def ng_batch_walk_launches(b):
    return int(lib().ng_batch_walk_launches(b))


def ng_batch_launch_count(b):
    v = ctypes.c_uint64(0)
    _bcheck(b, lib().ng_batch_launch_count(b, ctypes.byref(v)))
    return int(v.value)


def _scheck(s, code):
    if code != NG_OK:
        msg = lib().ng_serve_last_error(s)
        raise NgError(code, msg.decode() if msg else "")


def ng_serve_create(slots, hbm_budget):
    s = ctypes.c_void_p()
    _scheck(None, lib().ng_serve_create(ctypes.byref(s), int(slots), int(hbm_budget)))
    return s


def ng_serve_destroy(s):
    lib().ng_serve_destroy(s)


def ng_serve_submit(s, req: NgRequest, res: NgResult):
    i = ctypes.c_int64(-1)
    _scheck(s, lib().ng_serve_submit(s, ctypes.byref(req), ctypes.byref(res), ctypes.byref(i)))
    return int(i.value)


def ng_serve_cancel(s, rid):
    _scheck(s, lib().ng_serve_cancel(s, int(rid)))


def ng_serve_poll(s):
    k = ctypes.c_int(0)
    _scheck(s, lib().ng_serve_poll(s, ctypes.byref(k)))
    return int(k.value)


def ng_serve_pending(s):
    return int(lib().ng_serve_pending(s))


def ng_serve_wait(s, timeout_s):
    _scheck(s, lib().ng_serve_wait(s, float(timeout_s)))


def ng_serve(s, reqs, results, arrival_s=None, timeout_s=600.0):
    """reqs / results: ctypes arrays of NgRequest / NgResult; arrival_s: numpy float64."""
    arr = None if arrival_s is None else arrival_s.ctypes.data_as(ctypes.c_void_p)
    _scheck(s, lib().ng_serve(s, reqs, results, len(reqs), arr, float(timeout_s)))


def ng_serve_stats(s):
    """(bytes held now, peak bytes held, requests rerun with a larger tree,
    slot reconfigurations)."""
    held, peak = ctypes.c_size_t(0), ctypes.c_size_t(0)
    retries, reconf = ctypes.c_int64(0), ctypes.c_int64(0)
    _scheck(s, lib().ng_serve_stats(s, ctypes.byref(held), ctypes.byref(peak), ctypes.byref(retries),
                                    ctypes.byref(reconf)))
    return int(held.value), int(peak.value), int(retries.value), int(reconf.value)


def ng_serve_request_bytes(req: NgRequest):
    return int(lib().ng_serve_request_bytes(ctypes.byref(req)))


def make_request(kind, params: NgParams, pos, typ, mass, vel=None, nsteps=0, dt=0.0,
                 pos_out=None, vel_out=None, acc_out=None) -> NgRequest:
    """Request over HOST arrays (numpy or pinned torch CPU tensors); the caller
    keeps them alive until the request completes."""
    def addr(a):
        if a is None:
            return None
        return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
    r = NgRequest()
    r.kind, r.nsteps, r.dt, r.params = int(kind), int(nsteps), float(dt), params
    r.n = int(typ.shape[0])
    r.pos, r.vel, r.type, r.mass = addr(pos), addr(vel), addr(typ), addr(mass)
    r.pos_out, r.vel_out, r.acc_out = addr(pos_out), addr(vel_out), addr(acc_out)
    return r


def ng_sort_keys_noalloc(pos, typ, keys_out, perm_out, box=1.0, stream=None):
    """Sorted keys and permutation with no allocation (n <= 2^18); returns the
    status code."""
    return int(lib().ng_sort_keys_noalloc(typ.numel(), _ptr(pos), _ptr(typ), float(box),
                                          _ptr(keys_out), _ptr(perm_out), _stream(stream)))


def ng_version():
    return lib().ng_version().decode()


class Simulation:
    """Owns one ng_ctx; convenience wrapper over the functions above."""

    def __init__(self, params: NgParams, stream=None):
        self.D = params.D
        self.ctx = ng_create(params, stream)

    def close(self):
        if self.ctx is not None:
            ng_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def force(self, pos, typ, mass, acc=None, pm=True):
        """Build the tree, then the total acceleration (ng_force: short + long
        when the context has a mesh) or, with pm=False, the short-range tree
        acceleration alone (ng_tree_force); float32 [3, n]."""
        import torch
        n = typ.numel()
        if acc is None:
            acc = torch.empty((3, n), dtype=torch.float32, device=pos.device)
        ng_build_tree(self.ctx, pos, typ, mass)
        if pm:
            ng_force(self.ctx, acc)
        else:
            ng_tree_force(self.ctx, acc)
        return acc
