"""ctypes binding of libpd (include/pd.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  The module-level functions carry the C names (pd_create, pd_step,
...); ``Context`` bundles them.  Host buffers are numpy arrays (pinned ones work
and copy faster).  PyTorch supplies the stream and, by default, the device
memory (its caching allocator is passed as the library's allocator callback).

Importing this module does not load the library; the first call does, and it
raises if libpd.so has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the in-tree build of the library (no override: tests and benchmark always load it)
LIB_PATH = os.path.join(_HERE, "_lib", "libpd.so")

PD_OK, PD_EINVAL, PD_ENOMEM, PD_ECUDA, PD_ESTATE = 0, -1, -2, -3, -4
PD_ECAPACITY, PD_ENONFINITE, PD_ETIMEOUT, PD_EWALL = -5, -6, -7, -8
PD_MIXED, PD_FP64 = 0, 1
STATUS_NAMES = {0: "PD_OK", -1: "PD_EINVAL", -2: "PD_ENOMEM", -3: "PD_ECUDA", -4: "PD_ESTATE",
                -5: "PD_ECAPACITY", -6: "PD_ENONFINITE", -7: "PD_ETIMEOUT", -8: "PD_EWALL"}


class PDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Material(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("rho", ctypes.c_double), ("G0", ctypes.c_double),
                ("contact_radius", ctypes.c_double), ("contact_factor", ctypes.c_double),
                ("constants", ctypes.c_int), ("break_mode", ctypes.c_int), ("beta_d", ctypes.c_double),
                ("micromodulus", ctypes.c_int), ("mu", ctypes.c_double), ("wall_overlap", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p), ("precision", ctypes.c_int),
                ("contact", ctypes.c_int), ("contact_every", ctypes.c_int), ("skin", ctypes.c_double),
                ("lanes_per_node", ctypes.c_int), ("graph_chunk", ctypes.c_int), ("tiles", ctypes.c_int),
                ("cand_capacity", ctypes.c_int64), ("pairs", ctypes.c_int), ("persistent", ctypes.c_int),
                ("barrier_absent", ctypes.c_int)]


class Wall(ctypes.Structure):
    _fields_ = [("normal", ctypes.c_double * 3), ("point", ctypes.c_double * 3),
                ("velocity", ctypes.c_double * 3)]


class BondFilter(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", ctypes.c_double * 12)]


_lib = None
_lock = threading.Lock()
P = ctypes.c_void_p


def lib():
    """Loads libpd.so; raises if it is missing (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libpd.so is not built ({LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            i64, f64, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
            sig = {
                "pd_default_options": (None, [P]),
                "pd_create": (i32, [i64, P, P, P, P, P, P, P]),
                "pd_build_bonds": (i32, [P, f64, i32, P]),
                "pd_set_walls": (i32, [P, i32, P]),
                "pd_get_walls": (i32, [P, P]),
                "pd_set_body_force": (i32, [P, P]),
                "pd_stable_dt": (i32, [P, P]),
                "pd_step": (i32, [P, f64, i64]),
                "pd_damage": (i32, [P, P]),
                "pd_bulk_stress": (i32, [P, P, P, P]),
                "pd_bulk_stress_mean": (i32, [P, P, P, P, P]),
                "pd_fragments": (i32, [P, P, P]),
                "pd_fragment_stats": (i32, [P, i64, P, P, P]),
                "pd_num_bonds": (i32, [P, P]),
                "pd_bonds": (i32, [P, P, P]),
                "pd_contacts": (i32, [P, P, P]),
                "pd_forces": (i32, [P, P]),
                "pd_get_state": (i32, [P, P, P, P, P]),
                "pd_get_state_packed": (i32, [P, P, P, P, P]),
                "pd_set_state_packed": (i32, [P, P, P, P, P]),
                "pd_set_state": (i32, [P, P, P, P, P]),
                "pd_tuning": (i32, [P, P, P, P]),
                "pd_last_step_stats": (i32, [P, P, P, P]),
                "pd_step_counters": (i32, [P, P, P, P]),
                "pd_state_counters": (i32, [P, P, P]),
                "pd_set_profiling": (i32, [P, i32]),
                "pd_stable_dt_noalloc": (i32, [i64, P, P, P, P, f64, f64, P, P]),
                "pd_last_error": (ctypes.c_char_p, [P]),
                "pd_destroy": (None, [P]),
                "pd_mlp_create": (i32, [P, i32, ctypes.c_uint64, i32, P, P]),
                "pd_mlp_forward": (i32, [P, P, i64, P]),
                "pd_mlp_forward_device": (i32, [P, P, i64, P]),
                "pd_mlp_train_step": (i32, [P, P, P, i64, ctypes.c_float, P]),
                "pd_mlp_train_step_device": (i32, [P, P, P, i64, ctypes.c_float, P]),
                "pd_mlp_grad": (i32, [P, P, P, i64, P, P]),
                "pd_mlp_num_params": (i32, [P, P]),
                "pd_mlp_get_params": (i32, [P, P]),
                "pd_mlp_set_params": (i32, [P, P]),
                "pd_mlp_last_error": (ctypes.c_char_p, [P]),
                "pd_mlp_destroy": (None, [P]),
                "pd_mlp_set_forward_path": (i32, [P, i32]),
            }
            for name, (res, args) in sig.items():
                if not hasattr(L, name):
                    continue
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(P)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(status, ctx):
    if status != PD_OK:
        msg = lib().pd_last_error(ctx).decode() if ctx else ""
        raise PDError(status, msg)


# ---------------------------------------------------------------- torch plumbing
class _TorchAllocator:
    """Passes PyTorch's caching allocator to the library."""

    def __init__(self, device, stream):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, _ctx):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:  # out of memory: the library reports PD_ENOMEM
            return None

    def _free(self, ptr, _ctx):
        self.torch.cuda.caching_allocator_delete(ptr)


# ---------------------------------------------------------------- C-named calls
def pd_default_options():
    o = Options()
    lib().pd_default_options(ctypes.byref(o))
    return o


def pd_create(x, vol, grain, material, options, v0=None):
    x = _f64(x, (-1, 3))
    vol = _f64(vol)
    grain = np.ascontiguousarray(grain, np.int32)
    v0 = None if v0 is None else _f64(v0, (-1, 3))
    h = P()
    st = lib().pd_create(x.shape[0], _ptr(x), _ptr(vol), _ptr(grain), _ptr(v0), ctypes.byref(material),
                         ctypes.byref(options), ctypes.byref(h))
    if st != PD_OK:
        raise PDError(st, "pd_create failed")
    return h


def pd_build_bonds(h, horizon, filters=()):
    fl = (BondFilter * max(1, len(filters)))()
    for q, (kind, a) in enumerate(filters):
        fl[q].kind = int(kind)
        for t in range(12):
            fl[q].a[t] = float(a[t]) if t < len(a) else 0.0
    _check(lib().pd_build_bonds(h, float(horizon), len(filters), fl), h)


def pd_set_walls(h, walls):
    walls = _f64(walls, (-1, 9))
    arr = (Wall * max(1, walls.shape[0]))()
    for l in range(walls.shape[0]):
        for a in range(3):
            arr[l].normal[a], arr[l].point[a], arr[l].velocity[a] = walls[l, a], walls[l, 3 + a], walls[l, 6 + a]
    _check(lib().pd_set_walls(h, walls.shape[0], arr), h)


def pd_get_walls(h, nw):
    out = np.zeros((nw, 3))
    _check(lib().pd_get_walls(h, _ptr(out)), h)
    return out


def pd_set_body_force(h, b):
    b = _f64(b)
    _check(lib().pd_set_body_force(h, _ptr(b)), h)


def pd_stable_dt(h):
    d = ctypes.c_double()
    _check(lib().pd_stable_dt(h, ctypes.byref(d)), h)
    return d.value


def pd_step(h, dt, nsteps):
    _check(lib().pd_step(h, float(dt), int(nsteps)), h)


def pd_damage(h, n, out=None):
    out = np.zeros(n) if out is None else out
    _check(lib().pd_damage(h, _ptr(out)), h)
    return out


def pd_bulk_stress(h, areas, nw):
    s = np.zeros(6)
    wf = np.zeros((max(nw, 1), 3))
    ar = None if areas is None else _f64(areas)
    _check(lib().pd_bulk_stress(h, _ptr(ar), _ptr(s), _ptr(wf)), h)
    return s, wf[:nw]


def pd_bulk_stress_mean(h, areas, nw):
    s = np.zeros(6)
    wf = np.zeros((max(nw, 1), 3))
    span = ctypes.c_double()
    ar = None if areas is None else _f64(areas)
    _check(lib().pd_bulk_stress_mean(h, _ptr(ar), _ptr(s), _ptr(wf), ctypes.byref(span)), h)
    return s, wf[:nw], span.value


def pd_fragments(h, n):
    label = np.zeros(n, np.int32)
    nf = ctypes.c_int64()
    _check(lib().pd_fragments(h, _ptr(label), ctypes.byref(nf)), h)
    return label, nf.value


def pd_fragment_stats(h, nfrag):
    size = np.zeros(max(nfrag, 1), np.int64)
    vol = np.zeros(max(nfrag, 1))
    dmg = np.zeros(max(nfrag, 1))
    _check(lib().pd_fragment_stats(h, nfrag, _ptr(size), _ptr(vol), _ptr(dmg)), h)
    return size[:nfrag], vol[:nfrag], dmg[:nfrag]


def pd_num_bonds(h):
    B = ctypes.c_int64()
    _check(lib().pd_num_bonds(h, ctypes.byref(B)), h)
    return B.value


def pd_bonds(h, n):
    B = pd_num_bonds(h)
    rp = np.zeros(n + 1, np.int64)
    col = np.zeros(max(B, 1), np.int32)
    _check(lib().pd_bonds(h, _ptr(rp), _ptr(col)), h)
    return rp, col[:B]


def pd_contacts(h):
    cnt = ctypes.c_int64(0)
    _check(lib().pd_contacts(h, ctypes.byref(cnt), None), h)
    m = cnt.value
    ij = np.zeros((max(m, 1), 2), np.int32)
    cnt = ctypes.c_int64(m)
    _check(lib().pd_contacts(h, ctypes.byref(cnt), _ptr(ij)), h)
    return ij[:cnt.value]


def pd_forces(h, n, out=None):
    out = np.zeros((n, 3)) if out is None else out
    _check(lib().pd_forces(h, _ptr(out)), h)
    return out


def pd_get_state(h, n, B, u=None, v=None, broken=None):
    u = np.zeros((n, 3)) if u is None else u
    v = np.zeros((n, 3)) if v is None else v
    broken = np.zeros(max(B, 1), np.uint8) if broken is None else broken
    t = ctypes.c_double()
    _check(lib().pd_get_state(h, _ptr(u), _ptr(v), _ptr(broken), ctypes.byref(t)), h)
    return u, v, broken[:B], t.value


def pd_set_state(h, u=None, v=None, broken=None, t=None):
    u = None if u is None else _f64(u, (-1, 3))
    v = None if v is None else _f64(v, (-1, 3))
    broken = None if broken is None else np.ascontiguousarray(broken, np.uint8)
    tt = None if t is None else ctypes.byref(ctypes.c_double(t))
    _check(lib().pd_set_state(h, _ptr(u), _ptr(v), _ptr(broken), tt), h)


def pd_get_state_packed(h, n, B, u=None, v=None, bits=None):
    """State with the bond memory as ceil(B/32) uint32 words (bit c % 32 of word c // 32)."""
    u = np.zeros((n, 3)) if u is None else u
    v = np.zeros((n, 3)) if v is None else v
    bits = np.zeros(max((B + 31) // 32, 1), np.uint32) if bits is None else bits
    t = ctypes.c_double()
    _check(lib().pd_get_state_packed(h, _ptr(u), _ptr(v), _ptr(bits), ctypes.byref(t)), h)
    return u, v, bits[:(B + 31) // 32], t.value


def pd_set_state_packed(h, u=None, v=None, bits=None, t=None):
    u = None if u is None else _f64(u, (-1, 3))
    v = None if v is None else _f64(v, (-1, 3))
    bits = None if bits is None else np.ascontiguousarray(bits, np.uint32)
    tt = None if t is None else ctypes.byref(ctypes.c_double(t))
    _check(lib().pd_set_state_packed(h, _ptr(u), _ptr(v), _ptr(bits), tt), h)


def pack_broken(broken):
    """uint8 flags per slot -> packed uint32 words (the layout of pd_get_state_packed)."""
    b = np.asarray(broken, np.uint8).astype(bool)
    words = np.zeros((len(b) + 31) // 32, np.uint32)
    idx = np.nonzero(b)[0]
    np.bitwise_or.at(words, idx // 32, (np.uint32(1) << (idx % 32).astype(np.uint32)))
    return words


def pd_tuning(h):
    """(lanes per node, kernel: 0 global gathers / 1 tiles / 2 each bond once,
    ms per candidate: 4 lane counts for each kernel in that order)."""
    lanes, kernel = ctypes.c_int(), ctypes.c_int()
    ms = np.zeros(12)
    _check(lib().pd_tuning(h, ctypes.byref(lanes), ctypes.byref(kernel), _ptr(ms)), h)
    return lanes.value, kernel.value, ms


def pd_step_counters(h):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().pd_step_counters(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), h)
    return a.value, b.value, c.value


def pd_state_counters(h):
    a, u = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().pd_state_counters(h, ctypes.byref(a), ctypes.byref(u)), h)
    return a.value, u.value


def pd_last_step_stats(h):
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(lib().pd_last_step_stats(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), h)
    return a.value, b.value, c.value


def pd_set_profiling(h, on):
    _check(lib().pd_set_profiling(h, 1 if on else 0), h)


def pd_stable_dt_noalloc(n, x_dev, vol_dev, rowptr_dev, col_dev, c, rho, stream, dt_out_dev):
    """Critical time step from device arrays without any allocation (see pd.h).
    Pointer arguments are integers (e.g. torch ``data_ptr()``).  Returns the status."""
    return lib().pd_stable_dt_noalloc(int(n), P(x_dev), P(vol_dev), P(rowptr_dev), P(col_dev), float(c),
                                      float(rho), P(stream) if stream else None, P(dt_out_dev))


def pd_destroy(h):
    lib().pd_destroy(h)


# ---------------------------------------------------------------- convenience class
class Context:
    """One peridynamic problem on one GPU."""

    def __init__(self, x, vol, grain, material, v0=None, precision="mixed", contact=True,
                 contact_every=0, skin=0.0, lanes=0, chunk=64, device=0, stream=None,
                 torch_memory=True, tiles=0, cand_capacity=0, allocator=None, pairs=0, persistent=0,
                 barrier_absent=0):
        import torch
        m = material
        self.material = Material(m.E, m.rho, m.G0, m.contact_radius, m.contact_factor, m.constants,
                                 m.break_mode, getattr(m, "beta_d", 0.0), getattr(m, "micromodulus", 0),
                                 getattr(m, "mu", 0.0), getattr(m, "wall_overlap", 0))
        o = pd_default_options()
        o.device = device
        if stream is None:  # a stream of its own: graphs cannot capture the legacy stream
            stream = torch.cuda.Stream(device)
        self.stream = stream
        o.stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        self._alloc = None
        if allocator is not None:  # an object with ALLOC_FN / FREE_FN callbacks .alloc and .free
            self._alloc = allocator
            o.alloc, o.free = allocator.alloc, allocator.free
        elif torch_memory:
            self._alloc = _TorchAllocator(device, o.stream)
            o.alloc, o.free = self._alloc.alloc, self._alloc.free
        o.precision = PD_FP64 if precision == "fp64" else PD_MIXED
        o.contact = 1 if contact else 0
        o.contact_every = contact_every
        o.skin = skin
        o.lanes_per_node = lanes
        o.graph_chunk = chunk
        o.tiles = tiles
        o.cand_capacity = int(cand_capacity)
        o.pairs = int(pairs)
        o.persistent = int(persistent)
        o.barrier_absent = int(barrier_absent)
        self.options = o
        self.n = int(np.asarray(x).reshape(-1, 3).shape[0])
        self.h = pd_create(x, vol, grain, self.material, o, v0)
        self.nw = 0
        self.B = 0

    @classmethod
    def from_scenario(cls, sc, **kw):
        from . import scenarios as S
        ctx = cls(sc.x, sc.vol, sc.grain, sc.material, v0=sc.v0, **kw)
        if sc.walls:
            ctx.set_walls(S.walls_array(sc.walls))
        if any(sc.body_force):
            ctx.set_body_force(sc.body_force)
        ctx.build_bonds(sc.horizon, sc.filters)
        return ctx

    def build_bonds(self, horizon, filters=()):
        pd_build_bonds(self.h, horizon, filters)
        self.B = pd_num_bonds(self.h)

    def set_walls(self, walls):
        walls = np.asarray(walls, np.float64).reshape(-1, 9)
        pd_set_walls(self.h, walls)
        self.nw = walls.shape[0]

    def get_walls(self):
        return pd_get_walls(self.h, self.nw)

    def set_body_force(self, b):
        pd_set_body_force(self.h, b)

    def stable_dt(self):
        return pd_stable_dt(self.h)

    def step(self, dt, nsteps=1):
        pd_step(self.h, dt, nsteps)

    def damage(self):
        return pd_damage(self.h, self.n)

    def bulk_stress(self, areas=None):
        return pd_bulk_stress(self.h, areas, self.nw)

    def bulk_stress_mean(self, areas=None):
        """(sigma, mean wall forces, span) over the steps since the last call; resets."""
        return pd_bulk_stress_mean(self.h, areas, self.nw)

    def bonds(self):
        return pd_bonds(self.h, self.n)

    def fragments(self):
        """(label (n,) int32, caller order: smallest caller index of the node's fragment, count)."""
        return pd_fragments(self.h, self.n)

    def fragment_stats(self):
        """(size, volume, damage) per fragment in increasing label order."""
        _, nf = pd_fragments(self.h, self.n)
        return pd_fragment_stats(self.h, nf)

    def contacts(self):
        return pd_contacts(self.h)

    def forces(self):
        return pd_forces(self.h, self.n)

    def get_state(self):
        return pd_get_state(self.h, self.n, self.B)

    def set_state(self, u=None, v=None, broken=None, t=None):
        pd_set_state(self.h, u, v, broken, t)

    def tuning(self):
        """(lanes per node, kernel chosen, ms per candidate; see pd_tuning)."""
        return pd_tuning(self.h)

    def set_profiling(self, on):
        pd_set_profiling(self.h, on)

    def last_step_stats(self):
        return pd_last_step_stats(self.h)

    def state_counters(self):
        """(applied, unchanged) pd_set_state* calls since creation."""
        return pd_state_counters(self.h)

    def step_counters(self):
        """(steps, contact-list rebuilds, rolled-back segments) since creation."""
        return pd_step_counters(self.h)

    def close(self):
        if self.h:
            pd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- surrogate MLP
def pd_mlp_create(dims, seed=0, device=0, stream=None):
    d = (ctypes.c_int * len(dims))(*dims)
    h = P()
    st = lib().pd_mlp_create(d, len(dims) - 1, ctypes.c_uint64(seed), device, stream, ctypes.byref(h))
    if st != PD_OK:
        raise PDError(st, "pd_mlp_create failed")
    return h


def _mcheck(status, h):
    if status != PD_OK:
        raise PDError(status, lib().pd_mlp_last_error(h).decode() if h else "")


class MLP:
    """Bulk-stress surrogate network (BF16 tensor-core forward/backward, Adam)."""

    def __init__(self, dims=(109, 256, 256, 256, 256, 6), seed=0, device=0, stream=None):
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.dims = tuple(dims)
        self.h = pd_mlp_create(self.dims, seed, device, stream)
        n = ctypes.c_int64()
        _mcheck(lib().pd_mlp_num_params(self.h, ctypes.byref(n)), self.h)
        self.nparams = n.value

    def forward(self, X):
        X = np.ascontiguousarray(X, np.float32).reshape(-1, self.dims[0])
        Y = np.zeros((X.shape[0], self.dims[-1]), np.float32)
        _mcheck(lib().pd_mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(Y)), self.h)
        return Y

    def forward_device(self, X, Y):
        """X, Y: torch CUDA float32 tensors (contiguous)."""
        _mcheck(lib().pd_mlp_forward_device(self.h, P(X.data_ptr()), X.shape[0], P(Y.data_ptr())), self.h)

    def grad(self, X, T):
        X = np.ascontiguousarray(X, np.float32).reshape(-1, self.dims[0])
        T = np.ascontiguousarray(T, np.float32).reshape(-1, self.dims[-1])
        g = np.zeros(self.nparams, np.float32)
        loss = ctypes.c_float()
        _mcheck(lib().pd_mlp_grad(self.h, _ptr(X), _ptr(T), X.shape[0], _ptr(g), ctypes.byref(loss)), self.h)
        return float(loss.value), g

    def train_step(self, X, T, lr):
        X = np.ascontiguousarray(X, np.float32).reshape(-1, self.dims[0])
        T = np.ascontiguousarray(T, np.float32).reshape(-1, self.dims[-1])
        loss = ctypes.c_float()
        _mcheck(lib().pd_mlp_train_step(self.h, _ptr(X), _ptr(T), X.shape[0], ctypes.c_float(lr),
                                        ctypes.byref(loss)), self.h)
        return float(loss.value)

    def train_step_device(self, X, T, lr, loss_dev=None):
        lp = P(loss_dev.data_ptr()) if loss_dev is not None else None
        _mcheck(lib().pd_mlp_train_step_device(self.h, P(X.data_ptr()), P(T.data_ptr()), X.shape[0],
                                               ctypes.c_float(lr), lp), self.h)

    def set_forward_path(self, path):
        """0: fused tcgen05 forward when possible; 1: mma.sync GEMMs only."""
        _mcheck(lib().pd_mlp_set_forward_path(self.h, int(path)), self.h)

    def get_params(self):
        w = np.zeros(self.nparams, np.float32)
        _mcheck(lib().pd_mlp_get_params(self.h, _ptr(w)), self.h)
        return w

    def set_params(self, w):
        w = np.ascontiguousarray(w, np.float32)
        assert w.size == self.nparams
        _mcheck(lib().pd_mlp_set_params(self.h, _ptr(w)), self.h)

    def close(self):
        if self.h:
            lib().pd_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
