"""Python binding of libbhtree, the GB300 tree-code force evaluation.

Argument marshalling only: every step of the evaluation runs in the CUDA
library (include/bhtree.h).  PyTorch supplies device memory and streams.
The binding raises if the compiled library is missing; there is no fallback.

Functions keep the C names: bh_create / tree_build / tree_moments /
tree_force / direct_force / bh_status / bh_stats / bh_export, and
`Context` bundles them for one particle-set capacity.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbhtree.so")

BH_OK = 0
BH_ERR_INVALID = -1
BH_ERR_TOO_LARGE = -2
BH_ERR_NONFINITE = -3
BH_ERR_CAPACITY = -4
BH_ERR_DEVICE_TIMEOUT = -5
BH_ERR_CUDA = -6
BH_ERR_STATE = -7
BH_ERR_NOMEM = -8

EXPORT = dict(keys=1, perm=2, spos=3, node_first=4, node_count=5, node_child=6, node_nchild=7,
              node_level=8, com_m=9, seff=10, quad=11, group_first=12, group_count=13, box=14, next=15)

# the symbols declared in include/bhtree.h
SYMBOLS = ["bh_version", "bh_strerror", "bh_config_default", "bh_create", "bh_destroy", "tree_build",
           "tree_moments", "tree_force", "tree_force_particles", "tree_neighbors", "direct_force", "bh_kick_drift",
           "bh_status", "bh_stats", "bh_export", "bh_tree_force_static", "bh_mac_set", "bh_mac_label",
           "bh_mlp_train", "bh_mlp_grad", "bh_mlp_forward", "bh_batch_layout", "bh_force_batched", "bh_graph_capture_batched",
           "bh_graph_launch", "bh_graph_destroy", "bh_selftest_wait", "tree_softening", "direct_force_sym"]
BATCH_MAX_N = 65536
MLP_NPARAM = 1313
MLP_ACT = 135  # floats of training scratch per sample
STATIC_MAX_N = 32768
PWALK_UNSOFTENED_CELLS = 1
PWALK_INDIVIDUAL_SOFTENING = 2
CURVE_MORTON = 0
CURVE_HILBERT = 1
WALK_ONE_WARP = 0
WALK_PAIRED = 1
WALK_TMA = 2
SELFTEST_TILE_RING = 0
SELFTEST_LOOKBACK = 1
SELFTEST_TMA = 2


class BhConfig(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("group_size", ctypes.c_int), ("order", ctypes.c_int),
                ("fp64_node_threshold", ctypes.c_int), ("block_threads", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("max_systems", ctypes.c_int), ("curve", ctypes.c_int),
                ("max_level", ctypes.c_int), ("walk_variant", ctypes.c_int)]


class BhStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_groups", ctypes.c_int64), ("n_pp", ctypes.c_int64), ("n_pc", ctypes.c_int64),
                ("max_leaf_count", ctypes.c_int64), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("box", ctypes.c_float * 4),
                ("n_pp_total", ctypes.c_int64), ("n_pc_total", ctypes.c_int64), ("launches", ctypes.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("reserved", "box")}
        d["box"] = list(self.box)
        return d


class BhError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, _lib_or_none_strerror(code), code))


_lib = None


def _lib_or_none_strerror(code):
    try:
        return lib().bh_strerror(code).decode()
    except Exception:  # library missing while formatting an error
        return "error"


def lib():
    """Load libbhtree.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libbhtree.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.bh_version.restype = i32
        L.bh_strerror.argtypes = [i32]
        L.bh_strerror.restype = ctypes.c_char_p
        L.bh_config_default.argtypes = [ctypes.POINTER(BhConfig)]
        L.bh_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(BhConfig), i64, i32]
        L.bh_create.restype = i32
        L.bh_destroy.argtypes = [vp]
        L.tree_build.argtypes = [vp, vp, i64, vp]
        L.tree_build.restype = i32
        L.tree_moments.argtypes = [vp, ctypes.c_float, vp]
        L.tree_moments.restype = i32
        L.tree_force.argtypes = [vp, ctypes.c_float, vp, vp]
        L.tree_force.restype = i32
        L.tree_force_particles.argtypes = [vp, ctypes.c_float, i32, vp, vp]
        L.tree_force_particles.restype = i32
        L.tree_softening.argtypes = [vp, vp, vp]
        L.tree_softening.restype = i32
        L.tree_neighbors.argtypes = [vp, vp, ctypes.c_float, vp, vp, vp]
        L.tree_neighbors.restype = i32
        L.direct_force.argtypes = [vp, i64, vp, vp, i64, ctypes.c_double, vp, i32, vp]
        L.direct_force.restype = i32
        L.direct_force_sym.argtypes = [vp, vp, i64, vp, vp, vp, i64, vp, i32, vp]
        L.direct_force_sym.restype = i32
        L.bh_kick_drift.argtypes = [vp, vp, vp, vp, i64, ctypes.c_float, ctypes.c_float, vp]
        L.bh_kick_drift.restype = i32
        L.bh_tree_force_static.argtypes = [vp, i64, ctypes.POINTER(BhConfig), ctypes.c_float, ctypes.c_float, vp,
                                           ctypes.POINTER(ctypes.c_int), vp]
        L.bh_tree_force_static.restype = i32
        f32p = ctypes.POINTER(ctypes.c_float)
        L.bh_mac_set.argtypes = [vp, f32p, f32p, f32p, ctypes.c_float, ctypes.c_float]
        L.bh_mac_set.restype = i32
        L.bh_mac_label.argtypes = [vp, vp, i64, vp, ctypes.c_float, ctypes.c_float, vp, vp, vp, i64, vp, vp]
        L.bh_mac_label.restype = i32
        L.bh_mlp_train.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, i64, i64, i32, ctypes.c_float,
                                   ctypes.c_float, vp, i64, vp]
        L.bh_mlp_train.restype = i32
        L.bh_mlp_grad.argtypes = [vp, vp, vp, i64, ctypes.c_float, vp, i64, vp, vp, vp]
        L.bh_mlp_grad.restype = i32
        L.bh_mlp_forward.argtypes = [vp, vp, vp, i64, vp, i32, vp]
        L.bh_mlp_forward.restype = i32
        L.bh_batch_layout.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), i32]
        L.bh_batch_layout.restype = i32
        L.bh_force_batched.argtypes = [vp, vp, ctypes.c_float, ctypes.c_float, vp, vp]
        L.bh_force_batched.restype = i32
        L.bh_graph_capture_batched.argtypes = [vp, vp, ctypes.c_float, ctypes.c_float, vp, ctypes.POINTER(vp)]
        L.bh_graph_capture_batched.restype = i32
        L.bh_graph_launch.argtypes = [vp, vp]
        L.bh_graph_launch.restype = i32
        L.bh_graph_destroy.argtypes = [vp]
        L.bh_selftest_wait.argtypes = [vp, i32, vp]
        L.bh_selftest_wait.restype = i32
        L.bh_status.argtypes = [vp, vp]
        L.bh_status.restype = i32
        L.bh_stats.argtypes = [vp, vp, ctypes.POINTER(BhStats)]
        L.bh_stats.restype = i32
        L.bh_export.argtypes = [vp, i32, vp, i64, ctypes.POINTER(ctypes.c_int64), vp]
        L.bh_export.restype = i32
        _lib = L
    return _lib


def _check(rc, what):
    if rc != BH_OK:
        raise BhError(rc, what)


def _stream(stream):
    """cudaStream_t of a torch stream (None = torch's current stream)."""
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def config(**kw):
    c = BhConfig()
    lib().bh_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, int(v))
    return c


def bh_create(cfg, max_n, device=0):
    h = ctypes.c_void_p()
    _check(lib().bh_create(ctypes.byref(h), ctypes.byref(cfg) if cfg is not None else None,
                           int(max_n), int(device)), "bh_create")
    return h


def bh_destroy(h):
    lib().bh_destroy(h)


def tree_build(h, pos, n=None, stream=None):
    n = pos.shape[0] if n is None else n
    return lib().tree_build(h, _dptr(pos), int(n), _stream(stream))


def tree_moments(h, theta, stream=None):
    return lib().tree_moments(h, ctypes.c_float(theta), _stream(stream))


def tree_force(h, eps, out, stream=None):
    return lib().tree_force(h, ctypes.c_float(eps), _dptr(out), _stream(stream))


def tree_force_particles(h, eps, out, unsoftened_cells=False, stream=None, individual_softening=False):
    """The paper's per-particle next/more walk (Fig. 5); with
    individual_softening the lengths set by tree_softening (symmetrized)."""
    flags = (PWALK_UNSOFTENED_CELLS if unsoftened_cells else 0) | \
        (PWALK_INDIVIDUAL_SOFTENING if individual_softening else 0)
    return lib().tree_force_particles(h, ctypes.c_float(eps), int(flags), _dptr(out), _stream(stream))


def tree_softening(h, eps, stream=None):
    """Individual softening lengths (float32 device tensor, caller order) of
    the current tree's particles, for the symmetrized Plummer potential."""
    return lib().tree_softening(h, _dptr(eps), _stream(stream))


def tree_neighbors(h_ctx, h, count=None, rho=None, stream=None):
    """Neighbour counts and SPH densities (Sec. 4.3 general walk): h is a float
    tensor of n radii (caller order) or a positive number."""
    import torch
    if isinstance(h, torch.Tensor):
        return lib().tree_neighbors(h_ctx, _dptr(h), ctypes.c_float(0.0), _dptr(count), _dptr(rho), _stream(stream))
    return lib().tree_neighbors(h_ctx, None, ctypes.c_float(h), _dptr(count), _dptr(rho), _stream(stream))


def direct_force(src, tgt, tgt_self, eps, out, precision, stream=None):
    """Eq. (1) by direct summation: src (n,4) f32, tgt (m,4) f32, tgt_self (m,) int64
    or None, out (m,4) f32 (precision 32) or f64 (precision 64)."""
    return lib().direct_force(_dptr(src), int(src.shape[0]), _dptr(tgt), _dptr(tgt_self),
                              int(tgt.shape[0]), float(eps), _dptr(out), int(precision), _stream(stream))


def direct_force_sym(src, eps_src, tgt, eps_tgt, tgt_self, out, precision, stream=None):
    """direct_force with individual softening lengths (float32, one per source and
    per target) and the symmetrized Plummer potential."""
    return lib().direct_force_sym(_dptr(src), _dptr(eps_src), int(src.shape[0]), _dptr(tgt), _dptr(eps_tgt),
                                  _dptr(tgt_self), int(tgt.shape[0]), _dptr(out), int(precision), _stream(stream))


def bh_kick_drift(h, pos, vel, acc, dt_kick, dt_drift, stream=None):
    return lib().bh_kick_drift(h, _dptr(pos), _dptr(vel), _dptr(acc), int(pos.shape[0]),
                               ctypes.c_float(dt_kick), ctypes.c_float(dt_drift), _stream(stream))


def bh_tree_force_static(pos, theta, eps, out, cfg=None, stream=None, status=True):
    """Force evaluation without any device allocation (fixed scratch, n <= 32768).
    Returns (rc, device status); with status=False the call does not
    synchronise (as inside a CUDA graph capture) and the status is None."""
    st = ctypes.c_int(0)
    rc = lib().bh_tree_force_static(_dptr(pos), int(pos.shape[0]), ctypes.byref(cfg) if cfg is not None else None,
                                    ctypes.c_float(theta), ctypes.c_float(eps), _dptr(out),
                                    ctypes.byref(st) if status else None, _stream(stream))
    return rc, (st.value if status else None)


def _f32host(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def bh_mac_set(h, params=None, fmin=None, fmax=None, tau=1e-3, theta_fb=0.5):
    """Learned criterion on (params: 1313 host floats) or off (params None)."""
    if params is None:
        return lib().bh_mac_set(h, None, None, None, ctypes.c_float(1.0), ctypes.c_float(1.0))
    p, pp = _f32host(params)
    lo, plo = _f32host(fmin)
    hi, phi = _f32host(fmax)
    return lib().bh_mac_set(h, pp, plo, phi, ctypes.c_float(tau), ctypes.c_float(theta_fb))


def bh_mac_label(h, groups, acc_ref, eps, log10_floor, X, Y, count, pairs=None, stream=None):
    return lib().bh_mac_label(h, _dptr(groups), int(groups.numel()), _dptr(acc_ref), ctypes.c_float(eps),
                              ctypes.c_float(log10_floor), _dptr(X), _dptr(Y), _dptr(pairs), int(Y.numel()),
                              _dptr(count), _stream(stream))


def bh_mlp_train(X, Y, order, params, adam_m, adam_v, work, steps, batch, lr, under_weight, loss, t0,
                 stream=None):
    return lib().bh_mlp_train(_dptr(X), _dptr(Y), _dptr(order), int(Y.numel()), _dptr(params), _dptr(adam_m),
                              _dptr(adam_v), _dptr(work), int(work.numel()), int(steps), int(batch),
                              ctypes.c_float(lr), ctypes.c_float(under_weight), _dptr(loss), int(t0),
                              _stream(stream))


def bh_mlp_grad(params, X, Y, under_weight, work, grad, loss, stream=None):
    return lib().bh_mlp_grad(_dptr(params), _dptr(X), _dptr(Y), int(Y.numel()), ctypes.c_float(under_weight),
                             _dptr(work), int(work.numel()), _dptr(grad), _dptr(loss), _stream(stream))


def bh_mlp_forward(h, params, X, y, precision, stream=None):
    return lib().bh_mlp_forward(h, _dptr(params), _dptr(X), int(y.numel()), _dptr(y), int(precision),
                                _stream(stream))


def bh_batch_layout(h, offsets):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    return lib().bh_batch_layout(h, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(off.size - 1))


def bh_force_batched(h, pos, theta, eps, out, stream=None):
    return lib().bh_force_batched(h, _dptr(pos), ctypes.c_float(theta), ctypes.c_float(eps), _dptr(out),
                                  _stream(stream))


class BatchedGraph:
    """bh_force_batched captured once into a CUDA graph, replayed on demand."""

    def __init__(self, ctx, pos, theta, eps, out):
        self.exe = ctypes.c_void_p()
        _check(lib().bh_graph_capture_batched(ctx.h, _dptr(pos), ctypes.c_float(theta), ctypes.c_float(eps),
                                              _dptr(out), ctypes.byref(self.exe)), "bh_graph_capture_batched")
        self.keep = (pos, out)

    def launch(self, stream=None):
        _check(lib().bh_graph_launch(self.exe, _stream(stream)), "bh_graph_launch")

    def close(self):
        if self.exe:
            lib().bh_graph_destroy(self.exe)
            self.exe = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bh_selftest_wait(h, which, stream=None):
    """Launch one bounded device wait that nothing satisfies (SELFTEST_TILE_RING or
    SELFTEST_LOOKBACK); bh_status reports BH_ERR_DEVICE_TIMEOUT afterwards."""
    return lib().bh_selftest_wait(h, int(which), _stream(stream))


def bh_status(h, stream=None):
    return lib().bh_status(h, _stream(stream))


def bh_stats(h, stream=None):
    st = BhStats()
    _check(lib().bh_stats(h, _stream(stream), ctypes.byref(st)), "bh_stats")
    return st


def bh_export(h, what, dst, stream=None):
    nb = ctypes.c_int64(0)
    rc = lib().bh_export(h, EXPORT[what] if isinstance(what, str) else int(what), _dptr(dst),
                         int(dst.numel() * dst.element_size()), ctypes.byref(nb), _stream(stream))
    return rc, nb.value


class Context:
    """One tree context on a CUDA device (owns the library's workspace)."""

    def __init__(self, max_n, device=0, **cfg):
        self.cfg = config(**cfg)
        self.device = int(device)
        self.max_n = int(max_n)
        self.h = bh_create(self.cfg, self.max_n, self.device)

    def close(self):
        if self.h:
            bh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, pos, stream=None):
        _check(tree_build(self.h, pos, stream=stream), "tree_build")

    def moments(self, theta, stream=None):
        _check(tree_moments(self.h, theta, stream), "tree_moments")

    def force(self, eps, out, stream=None):
        _check(tree_force(self.h, eps, out, stream), "tree_force")

    def force_particles(self, eps, out, unsoftened_cells=False, stream=None, individual_softening=False):
        _check(tree_force_particles(self.h, eps, out, unsoftened_cells, stream, individual_softening),
               "tree_force_particles")

    def softening(self, eps, stream=None):
        _check(tree_softening(self.h, eps, stream), "tree_softening")

    def evaluate_symmetrized(self, pos, eps, theta, out=None, unsoftened_cells=False, stream=None):
        """Per-particle walk with individual softening lengths eps (float32,
        caller order) and the symmetrized Plummer potential."""
        import torch
        if out is None:
            out = torch.empty_like(pos)
        self.build(pos, stream)
        self.softening(eps, stream)
        self.moments(theta, stream)
        self.force_particles(0.0, out, unsoftened_cells, stream, individual_softening=True)
        return out

    def evaluate(self, pos, theta, eps, out=None, stream=None, walk="group", unsoftened_cells=False):
        """Whole force evaluation (build, moments, walk); returns (n, 4) f32 on the device.
        walk="group" (warp per group) or "particle" (the paper's per-particle walk)."""
        import torch
        if out is None:
            out = torch.empty_like(pos)
        self.build(pos, stream)
        self.moments(theta, stream)
        if walk == "group":
            self.force(eps, out, stream)
        elif walk == "particle":
            self.force_particles(eps, out, unsoftened_cells, stream)
        else:
            raise ValueError(walk)
        return out

    def neighbors(self, pos, h, stream=None):
        """Build the tree of pos and return (counts int32, densities f32), caller order."""
        import torch
        n = pos.shape[0]
        count = torch.empty(n, dtype=torch.int32, device=pos.device)
        rho = torch.empty(n, dtype=torch.float32, device=pos.device)
        self.build(pos, stream)
        _check(tree_neighbors(self.h, h, count, rho, stream), "tree_neighbors")
        return count, rho

    def kick_drift(self, pos, vel, acc, dt_kick, dt_drift, stream=None):
        _check(bh_kick_drift(self.h, pos, vel, acc, dt_kick, dt_drift, stream), "bh_kick_drift")

    def status(self, stream=None):
        return bh_status(self.h, stream)

    def stats(self, stream=None):
        return bh_stats(self.h, stream).as_dict()

    def export(self, what, stream=None):
        """Copy an internal array to a new host numpy array."""
        import torch
        dt = {"keys": torch.int32, "perm": torch.int32, "spos": torch.float32, "com_m": torch.float32,
              "seff": torch.float32, "quad": torch.float32, "box": torch.float32}.get(what, torch.int32)
        cap = max(self.max_n, 1) * 16 + 64
        if what not in ("keys", "perm", "spos", "group_first", "group_count", "box"):
            cap = (self.max_n + self.cfg.max_level * (self.max_n // (self.cfg.leaf_size + 1)) + 1) * 32
        buf = torch.empty(cap // 4, dtype=dt, device="cuda:%d" % self.device)
        rc, nb = bh_export(self.h, what, buf, stream)
        _check(rc, "bh_export(%s)" % what)
        a = buf[: nb // 4].cpu().numpy()
        if what in ("keys", "perm"):
            a = a.view(np.uint32)
        if what == "keys" and self.cfg.max_level > 10:
            a = a.view(np.uint64)
        if what in ("spos", "com_m"):
            a = a.reshape(-1, 4)
        if what == "quad":
            a = a.reshape(-1, 6)
        return a


def direct(src, tgt=None, tgt_self=None, eps=0.0, precision=32, stream=None):
    """Convenience: direct sum on torch CUDA tensors; with tgt=None every
    particle is a target and skips itself."""
    import torch
    if tgt is None:
        tgt = src
        tgt_self = torch.arange(src.shape[0], device=src.device, dtype=torch.int64)
    out = torch.empty((tgt.shape[0], 4), device=src.device,
                      dtype=torch.float64 if precision == 64 else torch.float32)
    _check(direct_force(src, tgt, tgt_self, eps, out, precision, stream), "direct_force")
    return out
