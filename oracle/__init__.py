"""FP64 CPU oracle of the tree-code force evaluation (numpy + ctypes over oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package; the product library and
its Python binding never do, and share no code with it.

Each wrapper names the passage of N. Nakasato, "Implementation of a Parallel
Tree Method on a GPU", that its C function follows.  Inputs are FP32
particle arrays (x, y, z, m) exactly as the GPU path receives them; all force
arithmetic is FP64.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_i64 = ctypes.c_int64
_vp = ctypes.c_void_p


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_direct.argtypes = [_i64, _f32p, _i64, _f32p, _vp, ctypes.c_double, _f64p]
        L.or_bbox.argtypes = [_i64, _f32p, _f32p]
        L.or_keys.argtypes = [_i64, _f32p, _f32p, _u64p, ctypes.c_int, ctypes.c_int]
        L.or_sph_kernel.argtypes = [ctypes.c_double, ctypes.c_double]
        L.or_sph_kernel.restype = ctypes.c_double
        L.or_sph_density.argtypes = [_i64, _f32p, _f32p, _i32p, _f64p]
        L.or_key_of_cell.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, ctypes.c_int]
        L.or_key_of_cell.restype = ctypes.c_uint64
        L.or_cell_of_key.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _u32p]
        L.or_sort.argtypes = [_i64, _u64p, _u32p]
        L.or_sort.restype = ctypes.c_int
        L.or_tree_build.argtypes = [_i64, _u64p, ctypes.c_int, ctypes.c_int, _i64] + [_i32p] * 5
        L.or_tree_build.restype = _i64
        L.or_moments.argtypes = [_i64, _f32p, _u64p, _i32p, _i32p, _i32p, _f32p,
                                 ctypes.c_double, _f64p, _vp, _f64p, _f64p, ctypes.c_int, ctypes.c_int]
        L.or_groups.argtypes = [_i64, _i32p, _i32p, _i32p, _i32p, ctypes.c_int, _i64, _i32p, _i32p]
        L.or_groups.restype = _i64
        L.or_force_groups.argtypes = [_i64, _f32p, _u32p, _i64, _i32p, _i32p, _i32p, _i32p,
                                      _f64p, _vp, _f64p, _i64, _i32p, _i32p, _vp,
                                      ctypes.c_double, _f64p, _vp, _vp, _vp, _vp]
        L.or_force_groups.restype = ctypes.c_int
        L.or_group_lists.argtypes = [_i64, _f32p, _i32p, _i32p, _i32p, _i32p, _f64p, _f64p,
                                     ctypes.c_int32, ctypes.c_int32, _i32p,
                                     ctypes.POINTER(ctypes.c_int64), _i32p,
                                     ctypes.POINTER(ctypes.c_int64)]
        L.or_group_lists.restype = _i64
        L.or_force_particles.argtypes = [_i64, _f32p, _u32p, _i64, _i32p, _i32p, _i32p, _i32p,
                                         _f64p, _vp, _f64p, _i64, _i64, ctypes.c_double,
                                         ctypes.c_int, _vp, _vp, _f64p, _vp, _vp, _vp, _vp]
        L.or_direct_sym.argtypes = [_i64, _f32p, _f32p, _i64, _f32p, _f32p, _vp, _f64p]
        L.or_cell_softening.argtypes = [_i64, _f32p, _f32p, _i32p, _i32p, _f64p]
        L.or_force_particles.restype = ctypes.c_int
        L.or_pc_eval.argtypes = [_f64p, _f64p, _vp, ctypes.c_double, _f64p]
        L.or_mlp_nparams.restype = ctypes.c_int
        L.or_mlp_forward.argtypes = [_f64p, _i64, _f64p, ctypes.c_int, _f64p]
        L.or_mlp_loss_grad.argtypes = [_f64p, _i64, _f64p, _f64p, ctypes.c_double, _f64p]
        L.or_mlp_loss_grad.restype = ctypes.c_double
        L.or_adam_step.argtypes = [_i64, _f64p, _f64p, _f64p, _f64p, _i64, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double]
        L.or_mac_training_pairs.argtypes = [_f32p, _i64, _i32p, _i32p, _i32p, _i32p, _i32p, _f64p, _vp, _f64p,
                                            _f64p, _i64, _i32p, _i32p, _f64p, ctypes.c_double, ctypes.c_double,
                                            _i64, _f64p, _f64p, _i32p, _i32p]
        L.or_mac_training_pairs.restype = _i64
        L.or_force_groups_learned.argtypes = [_i64, _f32p, _u32p, _i64, _i32p, _i32p, _i32p, _i32p, _i32p,
                                              _f64p, _vp, _f64p, _f64p, ctypes.c_double, ctypes.c_double, _i64,
                                              _i32p, _i32p, _vp, _f64p, _f64p, _f64p, ctypes.c_double,
                                              ctypes.c_double, _f64p, _vp, _vp, _vp, _vp]
        L.or_force_groups_learned.restype = ctypes.c_int
        L.or_kick_drift.argtypes = [_i64, _f64p, _f64p, _f64p, ctypes.c_double, ctypes.c_double]
        L.or_set_cell_rounding.argtypes = [ctypes.c_int]
        L.or_num_threads.restype = ctypes.c_int
        L.or_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _pos(pos):
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    if pos.ndim != 2 or pos.shape[1] != 4:
        raise ValueError("particles must be an (n, 4) array of x, y, z, m")
    return pos


def num_threads():
    return lib().or_num_threads()


def set_threads(t):
    lib().or_set_threads(int(t))


def direct(src, tgt=None, self_idx=None, eps=0.0):
    """Eq. (1): softened direct sum.  Returns (n_tgt, 4) FP64 (ax, ay, az, phi).

    With tgt=None the targets are the sources and target i skips source i.
    """
    src = _pos(src)
    if tgt is None:
        tgt = src
        self_idx = np.arange(src.shape[0], dtype=np.int64)
    tgt = _pos(tgt)
    if self_idx is not None:
        self_idx = np.ascontiguousarray(self_idx, dtype=np.int64)
    out = np.zeros((tgt.shape[0], 4), dtype=np.float64)
    lib().or_direct(src.shape[0], src, tgt.shape[0], tgt, _ptr(self_idx), float(eps), out)
    return out


def bbox(pos):
    """Sec. 4.1 root cube: (xmin, ymin, zmin, L) in FP32."""
    pos = _pos(pos)
    box = np.zeros(4, dtype=np.float32)
    lib().or_bbox(pos.shape[0], pos, box)
    return box


CURVE_MORTON = 0
CURVE_HILBERT = 1


def keys(pos, box, curve=CURVE_MORTON, max_level=10):
    """Sec. 5 ordering: keys of max_level bits per axis (10: 30-bit keys,
    returned as uint32; 21: 63-bit keys, uint64), Morton or Peano-Hilbert."""
    pos = _pos(pos)
    k = np.zeros(pos.shape[0], dtype=np.uint64)
    lib().or_keys(pos.shape[0], pos, np.ascontiguousarray(box, dtype=np.float32), k, int(curve), int(max_level))
    return k.astype(np.uint32) if max_level <= 10 else k


def key_of_cell(x, y, z, curve, nbits=10):
    """Key of one integer cell (nbits bits per axis)."""
    return int(lib().or_key_of_cell(int(x), int(y), int(z), int(curve), int(nbits)))


def cell_of_key(key, curve, nbits=10):
    """Integer cell (x, y, z) of one key."""
    c = np.zeros(3, dtype=np.uint32)
    lib().or_cell_of_key(int(key), int(curve), int(nbits), c)
    return tuple(int(v) for v in c)


def sort(k):
    """Stable sort by key; returns perm with perm[rank] = original index."""
    k = np.ascontiguousarray(k, dtype=np.uint64)
    perm = np.zeros(k.shape[0], dtype=np.uint32)
    if lib().or_sort(k.shape[0], k, perm) != 0:
        raise MemoryError("oracle sort")
    return perm


def node_capacity(n, n_leaf, max_level=10):
    """Upper bound on the node count: <= n leaves plus, on each of levels 0..max_level-1,
    at most n // (n_leaf + 1) internal nodes."""
    return int(n + max_level * (n // (n_leaf + 1)) + 1)


class Tree:
    """Nodes in breadth-first order (sorted by level, then first particle)."""

    def __init__(self, level, first, count, child_first, nchild):
        self.level, self.first, self.count = level, first, count
        self.child_first, self.nchild = child_first, nchild

    @property
    def n_nodes(self):
        return self.level.shape[0]

    def as_dict(self):
        return dict(level=self.level, first=self.first, count=self.count,
                    child_first=self.child_first, nchild=self.nchild)


def tree_build(skeys, n_leaf, max_level=10):
    """Sec. 4.1 octree over sorted keys (leaf: <= n_leaf particles or level max_level)."""
    skeys = np.ascontiguousarray(skeys, dtype=np.uint64)
    n = skeys.shape[0]
    cap = max(node_capacity(n, n_leaf, max_level), 1)
    arrs = [np.zeros(cap, dtype=np.int32) for _ in range(5)]
    nn = lib().or_tree_build(n, skeys, int(n_leaf), int(max_level), cap, *arrs)
    if nn < 0:
        raise RuntimeError("oracle tree_build: capacity exceeded")
    return Tree(*[a[:nn].copy() for a in arrs])


class Moments:
    def __init__(self, com_m, quad, s_eff, side):
        self.com_m, self.quad, self.s_eff, self.side = com_m, quad, s_eff, side


def moments(spos, skeys, tree, box, theta, order=1, curve=CURVE_MORTON, max_level=10):
    """Sec. 4.4 cell data: mass, centre of mass, Eq. (2) S_eff; quadrupole if order 2."""
    spos = _pos(spos)
    nn = tree.n_nodes
    com_m = np.zeros((nn, 4), dtype=np.float64)
    quad = np.zeros((nn, 6), dtype=np.float64) if order >= 2 else None
    s_eff = np.zeros(nn, dtype=np.float64)
    side = np.zeros(nn, dtype=np.float64)
    lib().or_moments(nn, spos, np.ascontiguousarray(skeys, dtype=np.uint64), tree.level,
                     tree.first, tree.count, np.ascontiguousarray(box, dtype=np.float32),
                     float(theta), com_m, _ptr(quad), s_eff, side, int(curve), int(max_level))
    return Moments(com_m, quad, s_eff, side)


def groups(tree, G):
    """Particle groups for the group walk (sibling packing, chunks of oversized leaves)."""
    nn = tree.n_nodes
    if nn == 0:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    n = int(tree.count[0])
    cap = n + 1
    gf = np.zeros(cap, dtype=np.int32)
    gc = np.zeros(cap, dtype=np.int32)
    ng = lib().or_groups(nn, tree.first, tree.count, tree.child_first, tree.nchild, int(G), cap, gf, gc)
    if ng < 0:
        raise RuntimeError("oracle groups: capacity exceeded")
    return gf[:ng].copy(), gc[:ng].copy()


def force_groups(spos, perm, tree, mom, g_first, g_count, eps, group_mask=None, want_quad=None):
    """Group walk with the conservative group form of Eq. (2).

    Returns dict(out=(n,4) caller order, margin=(n,), n_pp=(n,), n_pc=(n,),
    a_abs=(n,) sum of |a| over all terms).
    """
    spos = _pos(spos)
    n = spos.shape[0]
    out = np.zeros((n, 4), dtype=np.float64)
    a_abs = np.zeros(n, dtype=np.float64)
    margin = np.full(n, np.inf, dtype=np.float64)
    n_pp = np.zeros(n, dtype=np.int64)
    n_pc = np.zeros(n, dtype=np.int64)
    quad = mom.quad if want_quad is None or want_quad else None
    if group_mask is not None:
        group_mask = np.ascontiguousarray(group_mask, dtype=np.uint8)
    rc = lib().or_force_groups(n, spos, np.ascontiguousarray(perm, dtype=np.uint32), tree.n_nodes,
                               tree.first, tree.count, tree.child_first, tree.nchild,
                               np.ascontiguousarray(mom.com_m), _ptr(quad), mom.s_eff,
                               g_first.shape[0], g_first, g_count, _ptr(group_mask), float(eps),
                               out, _ptr(margin), _ptr(n_pp), _ptr(n_pc), _ptr(a_abs))
    if rc != 0:
        raise MemoryError("oracle force_groups")
    return dict(out=out, margin=margin, n_pp=n_pp, n_pc=n_pc, a_abs=a_abs)


def group_lists(spos, tree, mom, gfirst, gcount):
    """Accepted nodes and opened leaves of one group."""
    spos = _pos(spos)
    nn = tree.n_nodes
    pc = np.zeros(nn, dtype=np.int32)
    pp = np.zeros(nn, dtype=np.int32)
    npc = ctypes.c_int64(0)
    npp = ctypes.c_int64(0)
    lib().or_group_lists(nn, spos, tree.first, tree.count, tree.child_first, tree.nchild,
                         np.ascontiguousarray(mom.com_m), mom.s_eff, int(gfirst), int(gcount),
                         pc, ctypes.byref(npc), pp, ctypes.byref(npp))
    return pc[:npc.value].copy(), pp[:npp.value].copy()


def force_particles(spos, perm, tree, mom, eps, t0=0, t1=None, unsoftened_pc=False,
                    want_quad=None, eps_s=None, e2bar=None):
    """Per-particle walk of Fig. 3 / Fig. 5 with Eq. (2)'s criterion.  With
    eps_s (softening lengths in Morton order) and e2bar (cell_softening) the
    softening is individual and symmetrized (Sec. 7, after Saitoh & Makino)."""
    spos = _pos(spos)
    if eps_s is not None:
        eps_s = np.ascontiguousarray(eps_s, dtype=np.float32)
        e2bar = np.ascontiguousarray(e2bar, dtype=np.float64)
    n = spos.shape[0]
    t1 = n if t1 is None else t1
    out = np.zeros((n, 4), dtype=np.float64)
    n_pp = np.zeros(n, dtype=np.int64)
    n_pc = np.zeros(n, dtype=np.int64)
    margin = np.full(n, np.inf)
    a_abs = np.zeros(n)
    quad = mom.quad if want_quad is None or want_quad else None
    rc = lib().or_force_particles(n, spos, np.ascontiguousarray(perm, dtype=np.uint32),
                                  tree.n_nodes, tree.first, tree.count, tree.child_first,
                                  tree.nchild, np.ascontiguousarray(mom.com_m), _ptr(quad),
                                  mom.s_eff, int(t0), int(t1), float(eps), int(bool(unsoftened_pc)),
                                  _ptr(eps_s), _ptr(e2bar), out, _ptr(n_pp), _ptr(n_pc), _ptr(margin),
                                  _ptr(a_abs))
    if rc != 0:
        raise MemoryError("oracle force_particles")
    return dict(out=out, n_pp=n_pp, n_pc=n_pc, margin=margin, a_abs=a_abs)


class Built:
    """Everything the oracle derives from one particle set before the walk."""

    def __init__(self, pos, n_leaf, G, theta, order, curve=CURVE_MORTON, max_level=10):
        self.pos = _pos(pos)
        self.box = bbox(self.pos)
        self.curve = curve
        self.max_level = max_level
        self.keys = keys(self.pos, self.box, curve, max_level)
        self.perm = sort(self.keys)
        self.skeys = self.keys[self.perm]
        self.spos = self.pos[self.perm]
        self.tree = tree_build(self.skeys, n_leaf, max_level)
        self.mom = moments(self.spos, self.skeys, self.tree, self.box, theta, order, curve, max_level)
        self.g_first, self.g_count = groups(self.tree, G)
        self.order = order


def tree_force(pos, theta, eps, n_leaf=8, G=32, order=1, walk="group", group_mask=None, curve=CURVE_MORTON,
               max_level=10):
    """Whole force evaluation: box, keys, sort, tree, moments, groups, walk.

    walk="group" (the GPU path's criterion) or "particle" (the paper's).
    Returns (result dict, Built).
    """
    b = Built(pos, n_leaf, G, theta, order, curve, max_level)
    if walk == "group":
        res = force_groups(b.spos, b.perm, b.tree, b.mom, b.g_first, b.g_count, eps,
                           group_mask=group_mask)
    elif walk == "particle":
        res = force_particles(b.spos, b.perm, b.tree, b.mom, eps)
    else:
        raise ValueError(walk)
    return res, b


def kick_drift(pos, vel, acc, dt_kick, dt_drift):
    """Sec. 1's orbit loop, one leapfrog update: v += a dt_kick, then
    x += v dt_drift (with the updated v).  pos, vel, acc: (n, 4); returns new
    FP64 copies of pos and vel (component 3 of each unchanged)."""
    p = np.array(pos, dtype=np.float64, order="C", copy=True)
    v = np.array(vel, dtype=np.float64, order="C", copy=True)
    a = np.ascontiguousarray(acc, dtype=np.float64)
    if not (p.shape == v.shape == a.shape and p.ndim == 2 and p.shape[1] == 4):
        raise ValueError("pos, vel and acc must be (n, 4) arrays")
    lib().or_kick_drift(p.shape[0], p, v, a, float(dt_kick), float(dt_drift))
    return p, v


class cell_rounding:
    """Context manager: cell terms of the walks with (True, the default) or
    without (False) the FP32 rounding of the stored cell's centre and mass."""

    def __init__(self, on):
        self.on = bool(on)

    def __enter__(self):
        lib().or_set_cell_rounding(int(self.on))
        return self

    def __exit__(self, *exc):
        lib().or_set_cell_rounding(1)
        return False


def direct_sym(src, eps_src, tgt=None, eps_tgt=None, self_idx=None):
    """Symmetrized Plummer direct sum (individual softening lengths, pair
    softening (eps_i^2 + eps_j^2)/2).  With tgt=None the targets are the
    sources and target i skips source i."""
    src = _pos(src)
    eps_src = np.ascontiguousarray(eps_src, dtype=np.float32)
    if tgt is None:
        tgt, eps_tgt = src, eps_src
        self_idx = np.arange(src.shape[0], dtype=np.int64)
    tgt = _pos(tgt)
    eps_tgt = np.ascontiguousarray(eps_tgt, dtype=np.float32)
    if self_idx is not None:
        self_idx = np.ascontiguousarray(self_idx, dtype=np.int64)
    out = np.zeros((tgt.shape[0], 4), dtype=np.float64)
    lib().or_direct_sym(src.shape[0], src, eps_src, tgt.shape[0], tgt, eps_tgt, _ptr(self_idx), out)
    return out


def cell_softening(spos, eps_s, tree):
    """Per node: the mass-weighted mean of its particles' eps^2."""
    spos = _pos(spos)
    e2 = np.zeros(tree.n_nodes, dtype=np.float64)
    lib().or_cell_softening(tree.n_nodes, spos, np.ascontiguousarray(eps_s, dtype=np.float32), tree.first,
                            tree.count, e2)
    return e2


def tree_force_sym(pos, eps_len, theta, n_leaf=8, G=32, order=1, curve=CURVE_MORTON, max_level=10,
                   unsoftened_pc=False):
    """Per-particle walk with individual, symmetrized softening: eps_len holds
    each particle's softening length in the caller's order.  Returns (result, Built)."""
    b = Built(pos, n_leaf, G, theta, order, curve, max_level)
    eps_s = np.ascontiguousarray(np.asarray(eps_len, dtype=np.float32)[b.perm])
    e2bar = cell_softening(b.spos, eps_s, b.tree)
    res = force_particles(b.spos, b.perm, b.tree, b.mom, 0.0, unsoftened_pc=unsoftened_pc, eps_s=eps_s,
                          e2bar=e2bar)
    return res, b


def pc_eval(x, com_m, quad=None, eps=0.0):
    """One particle-cell term (monopole, plus quadrupole when quad is given)."""
    out = np.zeros(4, dtype=np.float64)
    q = None if quad is None else np.ascontiguousarray(quad, dtype=np.float64)
    lib().or_pc_eval(np.ascontiguousarray(x, dtype=np.float64),
                     np.ascontiguousarray(com_m, dtype=np.float64), _ptr(q), float(eps), out)
    return out


def rel_err(a, ref):
    """Per-target relative errors of accelerations and potentials (Sec. 5 a_error form)."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    ea = np.linalg.norm(a[:, :3] - ref[:, :3], axis=1) / np.linalg.norm(ref[:, :3], axis=1)
    ep = np.abs(a[:, 3] - ref[:, 3]) / np.abs(ref[:, 3])
    return ea, ep


# ---------------------------------------------------------------- learned MAC
NF = 6


def mlp_nparams():
    return lib().or_mlp_nparams()


def mlp_forward(params, X, bf16=False):
    """Network prediction per sample (FP64; bf16=True emulates the in-walk inference)."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, NF)
    y = np.zeros(X.shape[0])
    lib().or_mlp_forward(P, X.shape[0], X, int(bool(bf16)), y)
    return y


def mlp_loss_grad(params, X, Y, under_weight=4.0):
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, NF)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    g = np.zeros(P.shape[0])
    loss = lib().or_mlp_loss_grad(P, X.shape[0], X, Y, float(under_weight), g)
    return loss, g


def adam_step(params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In place on params, m, v (float64 arrays)."""
    lib().or_adam_step(params.shape[0], params, np.ascontiguousarray(grad, dtype=np.float64), m, v, int(t),
                       lr, b1, b2, eps)


def mac_training_pairs(b, group_idx, a_tot_sorted, eps, descend_above=1e-6, cap=None):
    """(features, labels, group, node) of the guard-passing (group, node) pairs
    of the listed groups; the guard is b's S_eff (b built with theta = theta_guard)."""
    gl_first = np.ascontiguousarray(b.g_first[group_idx], dtype=np.int32)
    gl_count = np.ascontiguousarray(b.g_count[group_idx], dtype=np.int32)
    cap = cap or int(4000 * len(group_idx) + 1000)
    X = np.zeros((cap, NF))
    Y = np.zeros(cap)
    pg = np.zeros(cap, np.int32)
    pn = np.zeros(cap, np.int32)
    t = b.tree
    np_ = lib().or_mac_training_pairs(b.spos, t.n_nodes, t.level, t.first, t.count, t.child_first, t.nchild,
                                      np.ascontiguousarray(b.mom.com_m), _ptr(b.mom.quad), b.mom.side,
                                      b.mom.s_eff, len(group_idx), gl_first, gl_count,
                                      np.ascontiguousarray(a_tot_sorted, dtype=np.float64), float(eps),
                                      float(descend_above), cap, X, Y, pg, pn)
    if np_ < 0:
        raise RuntimeError("mac_training_pairs: capacity exceeded")
    return X[:np_], Y[:np_], pg[:np_], pn[:np_]


def force_groups_learned(b, params, fmin, fmax, tau, eps, theta_guard, theta_fb, group_mask=None):
    """Group walk with the learned criterion (guard = b's S_eff, built with theta_guard)."""
    n = b.spos.shape[0]
    out = np.zeros((n, 4))
    mnet = np.full(n, np.inf)
    mgeo = np.full(n, np.inf)
    n_pp = np.zeros(n, np.int64)
    n_pc = np.zeros(n, np.int64)
    t = b.tree
    if group_mask is not None:
        group_mask = np.ascontiguousarray(group_mask, dtype=np.uint8)
    rc = lib().or_force_groups_learned(n, b.spos, np.ascontiguousarray(b.perm, dtype=np.uint32), t.n_nodes,
                                       t.level, t.first, t.count, t.child_first, t.nchild,
                                       np.ascontiguousarray(b.mom.com_m), _ptr(b.mom.quad), b.mom.side,
                                       b.mom.s_eff, float(theta_guard), float(theta_fb), b.g_first.shape[0],
                                       b.g_first, b.g_count, _ptr(group_mask),
                                       np.ascontiguousarray(params, dtype=np.float64),
                                       np.ascontiguousarray(fmin, dtype=np.float64),
                                       np.ascontiguousarray(fmax, dtype=np.float64), float(tau), float(eps),
                                       out, _ptr(mnet), _ptr(mgeo), _ptr(n_pp), _ptr(n_pc))
    if rc != 0:
        raise MemoryError("oracle force_groups_learned")
    return dict(out=out, margin_net=mnet, margin_geo=mgeo, n_pp=n_pp, n_pc=n_pc)


def mac_features_one(lo, hi, com_m, quad, side, level, count, mtot):
    L = lib()
    L.or_mac_features_one.argtypes = [_f64p, _f64p, _f64p, _vp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, _f64p]
    L.or_mac_features_one.restype = ctypes.c_int
    f = np.zeros(NF)
    q = None if quad is None else np.ascontiguousarray(quad, dtype=np.float64)
    ok = L.or_mac_features_one(np.asarray(lo, np.float64), np.asarray(hi, np.float64),
                               np.asarray(com_m, np.float64), _ptr(q), float(side), int(level), int(count),
                               float(mtot), f)
    return f if ok else None


def sph_kernel(r, h):
    """Cubic spline W(r, h) with support h (Monaghan & Lattanzio 1985)."""
    return float(lib().or_sph_kernel(float(r), float(h)))


def sph_density(pos, h):
    """Neighbour counts (|x_j - x_i| < h_i, j != i, decided in FP32) and SPH
    densities (FP64) by the all-pairs definition.  h: per particle (n,) or a scalar."""
    pos = _pos(pos)
    n = pos.shape[0]
    hh = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float32), (n,)), dtype=np.float32)
    count = np.zeros(n, dtype=np.int32)
    rho = np.zeros(n, dtype=np.float64)
    lib().or_sph_density(n, pos, hh, count, rho)
    return count, rho
