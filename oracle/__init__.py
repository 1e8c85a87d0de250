"""CPU oracle for the PeriDEM hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline``
and reference legs may import this package.  The CUDA library never links it,
and this package imports nothing from the library: the two share no code.

``pd_oracle.c`` holds the peridynamic definitions (FP64, caller node order);
``mlp.py`` holds the surrogate network's forward/backward/Adam in FP64 numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")
_LIB_OMP = os.path.join(_HERE, "_build", "liborc_omp.so")  # the same source with OpenMP (timing only)
_lock = threading.Lock()
_lib = None
_lib_omp = None

ERR_NONFINITE = 1
ERR_WALL = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no FMA contraction, no fast-math; once
    serial (liborc.so, the checker) and once with OpenMP over the node loops
    (liborc_omp.so, same arithmetic per node, for the all-core CPU baseline)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    for out, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
            tmp = out + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", *extra,
                                   "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, out)
    return _LIB


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64),
                ("x", ctypes.c_void_p), ("vol", ctypes.c_void_p), ("grain", ctypes.c_void_p),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("c", ctypes.c_double), ("s0", ctypes.c_double), ("Kn", ctypes.c_double),
                ("Rc", ctypes.c_double), ("rho", ctypes.c_double),
                ("break_mode", ctypes.c_int), ("contact", ctypes.c_int), ("nw", ctypes.c_int),
                ("walls", ctypes.c_void_p), ("b", ctypes.c_double * 3), ("frozen", ctypes.c_int),
                ("beta_d", ctypes.c_double), ("conic", ctypes.c_int), ("delta", ctypes.c_double),
                ("mu", ctypes.c_double), ("dt_f", ctypes.c_double), ("wall_overlap", ctypes.c_int)]


def lib(parallel: bool = False):
    """The serial oracle library, or (parallel=True) its OpenMP build."""
    global _lib, _lib_omp
    with _lock:
        if parallel:
            if _lib_omp is None:
                build()
                _lib_omp = _bind(ctypes.CDLL(_LIB_OMP))
            return _lib_omp
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def set_threads(k: int) -> int:
    """Threads of the OpenMP build; returns the number it will use."""
    return int(lib(parallel=True).orc_set_threads(int(k)))


def _bind(L):
    """Argument and result types of every oracle entry point."""
    P = ctypes.c_void_p
    i64, f64, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
    L.orc_constants.argtypes = [f64, f64, f64, f64, i32, i32, P]
    L.orc_ball_cut.argtypes = [f64, f64, f64, f64, P]
    L.orc_ball_cut.restype = None
    L.orc_bond_row.argtypes = [i64, P, P, f64, i32, P, P, i64, P]
    L.orc_bond_row.restype = i64
    L.orc_bonds_brute.argtypes = [i64, P, P, f64, i32, P, P, P, P]
    L.orc_bonds_brute.restype = i64
    L.orc_bonds_cells.argtypes = [i64, P, P, f64, i32, P, P, P, P]
    L.orc_bonds_cells.restype = i64
    L.orc_contact_pairs.argtypes = [P, P, P, i32, P]
    L.orc_contact_pairs.restype = i64
    L.orc_forces.argtypes = [P, P, P, P, P, P, P]
    L.orc_forces.restype = i32
    L.orc_step.argtypes = [P, P, P, P, P, P, f64, i64, P, P, P]
    L.orc_step.restype = i32
    L.orc_stable_dt.argtypes = [P]
    L.orc_stable_dt.restype = f64
    L.orc_damage.argtypes = [i64, P, P, P]
    L.orc_fragments.argtypes = [i64, P, P, P, P]
    L.orc_fragments.restype = i64
    L.orc_fragment_stats.argtypes = [i64, P, P, P, P, i64, P, P, P]
    L.orc_energy.argtypes = [P, P, P, P]
    L.orc_energy.restype = f64
    L.orc_set_threads.argtypes = [i32]
    L.orc_set_threads.restype = i32
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def ball_cut(R, a, b, c=None):
    """Volume and first moments (V, Mx, My, Mz) of the part of the ball |r| < R
    beyond the planes X = a, Y = b and Z = c (c = None: no Z plane)."""
    out = np.zeros(4)
    lib().orc_ball_cut(float(R), float(a), float(b), -float(R) if c is None else float(c), _p(out))
    return out


def constants(E, G0, delta, contact_factor=5.0, mode=0, micromodulus=0):
    """(K, c, s0, Kn) of the material (see orc_constants)."""
    out = np.zeros(4)
    lib().orc_constants(E, G0, delta, contact_factor, mode, micromodulus, _p(out))
    return tuple(float(v) for v in out)


def _filters(kinds, params):
    kinds = np.ascontiguousarray(kinds, np.int32)
    params = np.ascontiguousarray(params, np.float64).reshape(-1, 12)
    return len(kinds), kinds, params


def fragments(rowptr, col, broken):
    """Connected components over intact bonds (caller order CSR, broken per slot)."""
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    broken = np.ascontiguousarray(broken, np.uint8)
    n = len(rowptr) - 1
    label = np.zeros(max(n, 1), np.int32)
    nf = lib().orc_fragments(n, _p(rowptr), _p(col), _p(broken), _p(label))
    return label[:n], int(nf)


def fragment_stats(rowptr, broken, vol, label, nfrag):
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    broken = np.ascontiguousarray(broken, np.uint8)
    vol = np.ascontiguousarray(vol, np.float64)
    label = np.ascontiguousarray(label, np.int32)
    n = len(rowptr) - 1
    size = np.zeros(max(nfrag, 1), np.int64)
    volume = np.zeros(max(nfrag, 1))
    damage = np.zeros(max(nfrag, 1))
    lib().orc_fragment_stats(n, _p(rowptr), _p(broken), _p(vol), _p(label), nfrag, _p(size), _p(volume), _p(damage))
    return size[:nfrag], volume[:nfrag], damage[:nfrag]


def bond_row(x, grain, delta, i, kinds=(), params=()):
    x = np.ascontiguousarray(x, np.float64)
    grain = np.ascontiguousarray(grain, np.int32)
    nf, kinds, params = _filters(kinds, params)
    out = np.zeros(x.shape[0], np.int32)
    k = lib().orc_bond_row(x.shape[0], _p(x), _p(grain), delta, nf, _p(kinds), _p(params), i, _p(out))
    return out[:k].copy()


def bonds(x, grain, delta, kinds=(), params=(), brute=None):
    """Canonical bond CSR (rowptr int64 (n+1), col int32), caller order, ascending."""
    x = np.ascontiguousarray(x, np.float64)
    grain = np.ascontiguousarray(grain, np.int32)
    n = x.shape[0]
    nf, kinds, params = _filters(kinds, params)
    if brute is None:
        brute = n <= 6000
    fn = lib().orc_bonds_brute if brute else lib().orc_bonds_cells
    rowptr = np.zeros(n + 1, np.int64)
    B = fn(n, _p(x), _p(grain), delta, nf, _p(kinds), _p(params), _p(rowptr), None)
    col = np.zeros(max(B, 1), np.int32)
    fn(n, _p(x), _p(grain), delta, nf, _p(kinds), _p(params), _p(rowptr), _p(col))
    return rowptr, col[:B].copy()


class Model:
    """A problem (geometry, bonds, constants, walls) plus its state, all FP64,
    caller order.  Mirrors the library's state: u, v, a, broken (uint8 per
    directed slot), wall positions and time."""

    def __init__(self, x, vol, grain, rowptr, col, material, horizon, walls=None,
                 body_force=(0.0, 0.0, 0.0), v0=None, contact=True, parallel=False):
        self.L = lib(parallel)  # the OpenMP build only times the CPU baseline
        self.x = np.ascontiguousarray(x, np.float64)
        self.vol = np.ascontiguousarray(vol, np.float64)
        self.grain = np.ascontiguousarray(grain, np.int32)
        self.rowptr = np.ascontiguousarray(rowptr, np.int64)
        self.col = np.ascontiguousarray(col, np.int32)
        n = self.x.shape[0]
        m = material
        self.K, self.c, self.s0, self.Kn = constants(m.E, m.G0, horizon, m.contact_factor, m.constants,
                                                     getattr(m, "micromodulus", 0))
        self.walls = np.ascontiguousarray(walls if walls is not None else np.zeros((0, 9)), np.float64).reshape(-1, 9)
        self.wall_pos = self.walls[:, 3:6].copy()
        self.P = Problem()
        self.P.n = n
        self.P.x, self.P.vol, self.P.grain = _p(self.x), _p(self.vol), _p(self.grain)
        self.P.rowptr, self.P.col = _p(self.rowptr), _p(self.col)
        self.P.c, self.P.s0, self.P.Kn, self.P.Rc, self.P.rho = self.c, self.s0, self.Kn, m.contact_radius, m.rho
        self.P.break_mode = m.break_mode
        self.P.beta_d = getattr(m, "beta_d", 0.0)
        self.P.conic = getattr(m, "micromodulus", 0)
        self.P.mu = getattr(m, "mu", 0.0)
        self.P.wall_overlap = getattr(m, "wall_overlap", 0)
        self.P.dt_f = 0.0  # friction's time step: that of the latest step (0: Coulomb limit)
        self.P.delta = horizon
        self.P.contact = 1 if contact else 0
        self.P.nw = self.walls.shape[0]
        self.P.walls = _p(self.walls)
        self.P.b = (ctypes.c_double * 3)(*body_force)
        self.body_force = np.array(body_force, np.float64)
        self.rho = m.rho
        self.u = np.zeros((n, 3))
        self.v = np.zeros((n, 3)) if v0 is None else np.ascontiguousarray(v0, np.float64).copy()
        self.broken = np.zeros(max(len(self.col), 1), np.uint8)
        self.F = np.zeros((n, 3))
        self.react = np.zeros((self.walls.shape[0], 3))
        self.impulse = np.zeros((self.walls.shape[0], 3))   # sum of dt * react over steps
        self.impulse_span = 0.0
        self.t = 0.0
        self.err = 0
        self.acc = np.zeros((n, 3))

    @classmethod
    def from_scenario(cls, sc, rowptr=None, col=None, contact=True, parallel=False):
        from_sc = sc
        if rowptr is None:
            kinds = [k for k, _ in from_sc.filters]
            params = [list(a) + [0.0] * (12 - len(a)) for _, a in from_sc.filters]
            rowptr, col = bonds(sc.x, sc.grain, sc.horizon, kinds, params)
        walls = np.array([list(w.normal) + list(w.point) + list(w.velocity) for w in sc.walls],
                         np.float64).reshape(-1, 9)
        return cls(sc.x, sc.vol, sc.grain, rowptr, col, sc.material, sc.horizon, walls,
                   sc.body_force, sc.v0, contact, parallel)

    @property
    def n(self):
        return self.x.shape[0]

    def forces(self, frozen=False):
        """F at the current state, sets react; returns F.  Applies breaking unless
        frozen, which evaluates with the current bond memory unchanged."""
        self.P.frozen = 1 if frozen else 0
        self.err |= self.L.orc_forces(ctypes.byref(self.P), _p(self.u), _p(self.v), _p(self.wall_pos),
                                     _p(self.broken), _p(self.F), _p(self.react))
        self.P.frozen = 0
        return self.F

    def init(self):
        """a(t) from the current state, as the first half-kick needs it."""
        self.forces()
        self.acc = (self.F + self.body_force) / self.rho
        return self

    def step(self, dt, nsteps=1):
        if self.P.mu != 0.0 and self.P.dt_f != dt:
            # the friction's stick branch depends on dt: a(t) is evaluated again with it
            self.P.dt_f = dt
            self.init()
        self.err |= self.L.orc_step(ctypes.byref(self.P), _p(self.u), _p(self.v), _p(self.acc),
                                   _p(self.broken), _p(self.wall_pos), dt, nsteps, _p(self.F),
                                   _p(self.react), _p(self.impulse))
        self.t += dt * nsteps
        self.impulse_span += dt * nsteps
        self.P.dt_f = dt
        return self

    def stable_dt(self):
        return float(self.L.orc_stable_dt(ctypes.byref(self.P)))

    def damage(self):
        phi = np.zeros(self.n)
        self.L.orc_damage(self.n, _p(self.rowptr), _p(self.broken), _p(phi))
        return phi

    def fragments(self):
        """(label (n,) int32: smallest node index of the node's fragment, count)."""
        return fragments(self.rowptr, self.col, self.broken)

    def fragment_stats(self):
        """(size, volume, damage) per fragment in increasing label order."""
        label, nf = self.fragments()
        return fragment_stats(self.rowptr, self.broken, self.vol, label, nf)

    def energy(self):
        return float(self.L.orc_energy(ctypes.byref(self.P), _p(self.u), _p(self.v), _p(self.broken)))

    def contact_pairs(self, brute=False):
        """(m,2) int32 ordered contact pairs at the current state, sorted."""
        cnt = self.L.orc_contact_pairs(ctypes.byref(self.P), _p(self.u), _p(self.broken), int(brute), None)
        pr = np.zeros((max(cnt, 1), 2), np.int32)
        self.L.orc_contact_pairs(ctypes.byref(self.P), _p(self.u), _p(self.broken), int(brute), _p(pr))
        return pr[:cnt].copy()

    def bulk_stress(self, areas):
        return bulk_stress(self.walls[:, 0:3], self.react, areas)

    def bulk_stress_mean(self, areas, reset=True):
        """Bulk stress from the wall forces averaged over the steps since the last
        reset (impulse / span), the mean wall forces and the span; then resets."""
        mean = self.impulse / self.impulse_span if self.impulse_span > 0 else np.zeros_like(self.impulse)
        out = (bulk_stress(self.walls[:, 0:3], mean, areas), mean.copy(), self.impulse_span)
        if reset:
            self.impulse[:] = 0.0
            self.impulse_span = 0.0
        return out


def bulk_stress(normals, react, areas):
    """Bulk stress (Voigt xx, yy, zz, yz, xz, xy) from wall reactions.

    Reading of "bulk strength = difference of top and bottom reactions, normalised
    by the top area" (Sec. 6.4): the wall pushes on the aggregate with -R_l over
    area A_l, whose outward normal (of the aggregate) is m_l = -n_l; Cauchy's
    relation sigma m = t gives, per wall, the column sigma e_k = -(R_l / A_l)(m_l . e_k)
    for the axis k that m_l points along.  Columns are averaged over the walls
    that face each axis and the result is symmetrised.
    """
    normals = np.asarray(normals, np.float64).reshape(-1, 3)
    react = np.asarray(react, np.float64).reshape(-1, 3)
    areas = np.asarray(areas, np.float64).reshape(-1)
    S = np.zeros((3, 3))
    cnt = np.zeros(3)
    for l in range(normals.shape[0]):
        m = -normals[l]
        k = int(np.argmax(np.abs(m)))
        S[:, k] += -(react[l] / areas[l]) * np.sign(m[k])
        cnt[k] += 1
    for k in range(3):
        if cnt[k] > 0:
            S[:, k] /= cnt[k]
    S = 0.5 * (S + S.T)
    return np.array([S[0, 0], S[1, 1], S[2, 2], S[1, 2], S[0, 2], S[0, 1]])
