"""Seeded synthetic workloads for the PeriDEM hot path.

This module only lays out nodes, volumes, grain ids, initial velocities,
walls and bond-removal filters.  It holds none of the method's arithmetic
(no micromodulus, stretch, contact law or time step): both the CUDA path and
the CPU oracle receive the arrays produced here and compute everything else
themselves.

Workloads (sizes follow the paper's experiments, Sec. 6-8; the CT grains and
meshes of the paper are not available, so seeded lattices stand in for them):

* ``sphere``      - one glass sphere between two plates (Sec. 6.2 setting).
* ``kalthoff``    - notched steel plate, edge segment given 32 m/s
                    (Kalthoff-Winkler geometry of Sec. 6.1; bonds across the
                    notch faces removed as in Sec. 5.3.1).
* ``hollow``      - hollow glass sphere crushed by two plates (Sec. 6.2,
                    bond removal of Sec. 5.3.2).
* ``aggregate``   - star-shaped grains (seeded spherical-harmonic level sets)
                    in a box, compressed by a top wall (Sec. 6.4 setting).

Every random draw comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# Filter kinds understood by both the library and the oracle.
FILTER_NOTCH = 1    # a[0:4] plane (a,b,c,d); a[4:7] face box min; a[7:10] face box max
FILTER_SPHERE = 2   # a[0:3] centre; a[3] inner radius


@dataclass
class Material:
    E: float            # Young's modulus, Pa (bond-based PD fixes nu = 1/4)
    rho: float          # density, kg/m^3
    G0: float           # critical energy release rate, J/m^2
    contact_radius: float   # R_c, m
    contact_factor: float = 5.0  # K_n = contact_factor * c / delta
    constants: int = 0      # 0 = self-consistent c, s0; 1 = paper's table values
    break_mode: int = 0     # 0 = tension s > s0; 1 = |s| > s0
    beta_d: float = 0.0     # normal contact damping (Sec. 3.3), N s / m^7; 0 = none
    micromodulus: int = 0   # 0 = constant, 1 = conic c (delta - |xi|) (table of Sec. 3.1.1)
    mu: float = 0.0         # stick-slip friction coefficient (Sec. 3.3); 0 = frictionless
    wall_overlap: int = 0   # 1 = inclusion-exclusion over orthogonal walls (Sec. 4.1.1); 0 = sum


@dataclass
class Wall:
    normal: tuple       # unit normal pointing into the domain
    point: tuple        # a point on the plane at t = 0
    velocity: tuple     # rigid velocity of the plane, m/s


@dataclass
class Scenario:
    name: str
    x: np.ndarray           # (n,3) float64 reference positions
    vol: np.ndarray         # (n,) float64 nodal volumes
    grain: np.ndarray       # (n,) int32 grain id
    v0: np.ndarray          # (n,3) float64 initial velocity
    material: Material
    horizon: float          # delta, m
    h: float                # lattice spacing, m
    walls: list = field(default_factory=list)
    filters: list = field(default_factory=list)   # list of (kind, [12 doubles])
    body_force: tuple = (0.0, 0.0, 0.0)
    dt_factor: float = 0.8  # dt = dt_factor * critical step
    steps: int = 200
    wall_area: float = 1.0  # area used to turn the plate reaction into a stress
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def _glass(h: float) -> Material:
    return Material(E=72e9, rho=2440.0, G0=135.0, contact_radius=0.6 * h)


def _steel(h: float) -> Material:
    return Material(E=190e9, rho=8000.0, G0=2.2e4, contact_radius=0.6 * h)


def _jitter(rng, n, h, amp=0.01):
    return rng.uniform(-amp * h, amp * h, size=(n, 3))


def _plates(x: np.ndarray, rc: float, speed: float):
    """Two z-plates just out of reach of the extreme nodes, moving inward."""
    zmax = float(x[:, 2].max())
    zmin = float(x[:, 2].min())
    top = Wall(normal=(0.0, 0.0, -1.0), point=(0.0, 0.0, zmax + rc), velocity=(0.0, 0.0, -speed))
    bot = Wall(normal=(0.0, 0.0, 1.0), point=(0.0, 0.0, zmin - rc), velocity=(0.0, 0.0, speed))
    return [top, bot]


def sphere(seed: int = 0, h: float = 1e-4, radius_cells: int = 10, speed: float = 1.0,
           steps: int = 200) -> Scenario:
    """Single glass sphere, radius 10 h, h = 0.1 mm (4,139 lattice nodes), delta = 3h,
    squeezed between two frictionless plates moving inward at ``speed``."""
    rng = np.random.default_rng(seed)
    r = radius_cells
    i = np.arange(-r, r + 1)
    I, J, K = np.meshgrid(i, i, i, indexing="ij")
    m = (I * I + J * J + K * K) < r * r
    lat = np.stack([I[m], J[m], K[m]], axis=1).astype(np.float64)
    x = lat * h + _jitter(rng, lat.shape[0], h)
    n = x.shape[0]
    mat = _glass(h)
    sc = Scenario(name="sphere", x=x, vol=np.full(n, h ** 3), grain=np.zeros(n, np.int32),
                  v0=np.zeros((n, 3)), material=mat, horizon=3 * h, h=h,
                  walls=_plates(x, mat.contact_radius, speed), steps=steps,
                  wall_area=math.pi * (r * h) ** 2)
    return sc


def kalthoff(seed: int = 0, h: float = 1e-3, length: float = 0.1, height: float = 0.2,
             thickness: float = 0.009, notch_len: float = 0.05, notch_width: float = 1.5e-3,
             notch_gap: float = 0.05, speed: float = 32.0, horizon_cells: int = 4,
             steps: int = 2000, jitter: float = 0.0) -> Scenario:
    """Kalthoff-Winkler-type notched plate (steel).  Nodes sit at cell centres of an
    h-grid over ``length x height x thickness`` (x = impact direction).  Two edge notches
    start at x = 0, run ``notch_len`` along +x, are ``notch_width`` wide in y and lie
    ``notch_gap`` apart, centred in y.  Nodes inside a notch are removed and bonds that
    cross a notch mid-plane inside the notch face are removed (Sec. 5.3.1).  The edge
    column of nodes between the notches starts at ``speed`` along +x."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = int(round(length / h)), int(round(height / h)), int(round(thickness / h))
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    x = np.stack([(I.ravel() + 0.5) * h, (J.ravel() + 0.5) * h, (K.ravel() + 0.5) * h], axis=1)
    yc = [0.5 * height - 0.5 * notch_gap, 0.5 * height + 0.5 * notch_gap]
    keep = np.ones(x.shape[0], bool)
    for c in yc:
        keep &= ~((x[:, 0] < notch_len) & (np.abs(x[:, 1] - c) < 0.5 * notch_width))
    x = x[keep]
    if jitter > 0:
        x = x + _jitter(rng, x.shape[0], h, jitter)
    n = x.shape[0]
    v0 = np.zeros((n, 3))
    seg = (x[:, 0] < h) & (x[:, 1] > yc[0] + 0.5 * notch_width) & (x[:, 1] < yc[1] - 0.5 * notch_width)
    v0[seg, 0] = speed
    filters = []
    for c in yc:
        a = [0.0, 1.0, 0.0, -c,
             -0.5 * h, c - 0.5 * notch_width, -0.5 * h,
             notch_len, c + 0.5 * notch_width, thickness + 0.5 * h]
        filters.append((FILTER_NOTCH, a + [0.0, 0.0]))
    mat = _steel(h)
    return Scenario(name="kalthoff", x=x, vol=np.full(n, h ** 3), grain=np.zeros(n, np.int32),
                    v0=v0, material=mat, horizon=horizon_cells * h, h=h, filters=filters,
                    steps=steps, wall_area=1.0,
                    info={"impacted_nodes": int(seg.sum()), "notch_y": yc})


def hollow(seed: int = 0, h: float = 2e-5, outer_cells: int = 50, inner_cells: int = 35,
           speed: float = 5.0, steps: int = 10000) -> Scenario:
    """Hollow glass sphere, R = 1 mm, r = 0.7 mm, h = 0.02 mm (343,846 lattice nodes),
    delta = 3h, crushed by two plates at ``speed``.  The inner-sphere bond filter of
    Sec. 5.3.2 is passed with radius (inner_cells - 1/2) h, which lies between the
    void and the first shell layer."""
    rng = np.random.default_rng(seed)
    R, r = outer_cells, inner_cells
    i = np.arange(-R, R + 1)
    I, J, K = np.meshgrid(i, i, i, indexing="ij")
    rr = I * I + J * J + K * K
    m = (rr < R * R) & (rr >= r * r)
    lat = np.stack([I[m], J[m], K[m]], axis=1).astype(np.float64)
    x = lat * h + _jitter(rng, lat.shape[0], h)
    n = x.shape[0]
    mat = _glass(h)
    filt = [(FILTER_SPHERE, [0.0, 0.0, 0.0, (r - 0.5) * h] + [0.0] * 8)]
    return Scenario(name="hollow", x=x, vol=np.full(n, h ** 3), grain=np.zeros(n, np.int32),
                    v0=np.zeros((n, 3)), material=mat, horizon=3 * h, h=h,
                    walls=_plates(x, mat.contact_radius, speed), filters=filt, steps=steps,
                    wall_area=math.pi * (R * h) ** 2)


def _real_sph_harm_table(lmax: int, ct: np.ndarray, phi: np.ndarray) -> dict:
    """Real orthonormal spherical harmonics Y_lm(theta, phi) for 0 <= l <= lmax from the
    textbook associated-Legendre recurrence; returns {(l, m): values}."""
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    P = {}
    pmm = np.ones_like(ct)
    for m in range(lmax + 1):
        if m > 0:
            pmm = -pmm * (2 * m - 1) * st
        P[(m, m)] = pmm
        if m + 1 <= lmax:
            P[(m + 1, m)] = ct * (2 * m + 1) * pmm
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * ct * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    Y = {}
    for l in range(lmax + 1):
        for m in range(0, l + 1):
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
            if m == 0:
                Y[(l, 0)] = norm * P[(l, 0)]
            else:
                Y[(l, m)] = math.sqrt(2.0) * norm * P[(l, m)] * np.cos(m * phi)
                Y[(l, -m)] = math.sqrt(2.0) * norm * P[(l, m)] * np.sin(m * phi)
    return Y


def _star_radius(R, coef, dirs):
    ct = dirs[:, 2]
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    Y = _real_sph_harm_table(8, ct, phi)
    r = np.ones(dirs.shape[0])
    for (l, m), a in coef.items():
        r = r + a * Y[(l, m)]
    return R * r


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def star_grain(rng, R: float, h: float, lmax: int = 8, amp: float = 0.04):
    """Lattice nodes of one star-shaped grain r(theta,phi) = R (1 + sum_{l=2..lmax} a_lm Y_lm),
    a_lm ~ N(0, amp/l); redrawn while min r < R/2.  Returns (nodes (k,3) centred at 0,
    max radius)."""
    fib = np.arange(2000) + 0.5
    th = np.arccos(1 - 2 * fib / 2000.0)
    ph = math.pi * (1 + 5 ** 0.5) * fib
    probe = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    while True:
        coef = {(l, m): rng.normal(0.0, amp / l) for l in range(2, lmax + 1) for m in range(-l, l + 1)}
        rp = _star_radius(R, coef, probe)
        if rp.min() >= 0.5 * R:
            break
    rmax = float(rp.max()) * 1.05
    k = int(math.ceil(rmax / h))
    i = np.arange(-k, k + 1)
    I, J, K = np.meshgrid(i, i, i, indexing="ij")
    lat = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1).astype(np.float64) * h
    rad = np.linalg.norm(lat, axis=1)
    cand = lat[(rad < rmax) & (rad > 0)]
    d = cand / np.linalg.norm(cand, axis=1, keepdims=True)
    inside = np.linalg.norm(cand, axis=1) < _star_radius(R, coef, d)
    nodes = np.concatenate([np.zeros((1, 3)), cand[inside]], axis=0)
    return nodes, float(np.linalg.norm(nodes, axis=1).max())


def aggregate(seed: int = 0, n_grains: int = 1000, h: float = 0.5e-3 / 12, rmin: float = 0.4e-3,
              rmax: float = 0.6e-3, gap_cells: float = 1.0, speed: float = 10.0,
              steps: int = 200) -> Scenario:
    """Aggregate of ``n_grains`` star-shaped glass grains (radius R ~ U(rmin, rmax)), each a
    seeded spherical-harmonic level set meshed on a common lattice of spacing h, with a
    random rotation, placed on a jittered cubic lattice of centres inside a box of six
    walls; the top wall moves down at ``speed``.  Grains never overlap at t = 0: the
    centre spacing is the largest grain diameter plus ``gap_cells`` h."""
    rng = np.random.default_rng(seed)
    grains = []
    for g in range(n_grains):
        R = rng.uniform(rmin, rmax)
        nodes, ext = star_grain(rng, R, h)
        grains.append((nodes @ _random_rotation(rng).T, ext))
    ext_max = max(e for _, e in grains)
    pitch = 2 * ext_max + gap_cells * h
    side = int(math.ceil(n_grains ** (1.0 / 3.0)))
    xs, gs = [], []
    for g, (nodes, ext) in enumerate(grains):
        a, b, c = g % side, (g // side) % side, g // (side * side)
        slack = max(0.0, ext_max - ext)
        centre = np.array([a, b, c], np.float64) * pitch + rng.uniform(-slack, slack, 3)
        xs.append(nodes + centre)
        gs.append(np.full(nodes.shape[0], g, np.int32))
    x = np.concatenate(xs)
    grain = np.concatenate(gs)
    n = x.shape[0]
    mat = _glass(h)
    rc = mat.contact_radius
    lo = x.min(axis=0) - rc
    hi = x.max(axis=0) + rc
    walls = [Wall((1.0, 0.0, 0.0), (lo[0], 0.0, 0.0), (0.0, 0.0, 0.0)),
             Wall((-1.0, 0.0, 0.0), (hi[0], 0.0, 0.0), (0.0, 0.0, 0.0)),
             Wall((0.0, 1.0, 0.0), (0.0, lo[1], 0.0), (0.0, 0.0, 0.0)),
             Wall((0.0, -1.0, 0.0), (0.0, hi[1], 0.0), (0.0, 0.0, 0.0)),
             Wall((0.0, 0.0, 1.0), (0.0, 0.0, lo[2]), (0.0, 0.0, 0.0)),
             Wall((0.0, 0.0, -1.0), (0.0, 0.0, hi[2]), (0.0, 0.0, -speed))]
    vol = np.full(n, h ** 3)
    box = np.prod(hi - lo)
    return Scenario(name="aggregate", x=x, vol=vol, grain=grain, v0=np.zeros((n, 3)),
                    material=mat, horizon=3 * h, h=h, walls=walls, steps=steps,
                    wall_area=float((hi[0] - lo[0]) * (hi[1] - lo[1])),
                    info={"n_grains": n_grains, "solid_fraction": float(vol.sum() / box),
                          "nodes_per_grain_min": int(np.bincount(grain).min()),
                          "nodes_per_grain_max": int(np.bincount(grain).max())})


def small_block(seed: int = 0, nx: int = 6, ny: int = 5, nz: int = 4, h: float = 1e-3,
                jitter: float = 0.01) -> Scenario:
    """Tiny jittered brick of glass-like material for unit tests (one grain, no walls)."""
    rng = np.random.default_rng(seed)
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    x = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1).astype(np.float64) * h
    x = x + _jitter(rng, x.shape[0], h, jitter)
    n = x.shape[0]
    return Scenario(name="block", x=x, vol=np.full(n, h ** 3), grain=np.zeros(n, np.int32),
                    v0=np.zeros((n, 3)), material=_glass(h), horizon=3 * h, h=h, steps=10)


def shape_particle(shape: str, R: float, h: float) -> np.ndarray:
    """Lattice nodes (spacing h, centred at 0) of one particle of the shape study
    (Sec. 6.5): "sphere" (|x| < R), "shell" (0.7 R <= |x| < R, the hollow spheres
    of Sec. 6.3), or "jack", a 3-D plus of three orthogonal cylinders reaching R from
    the centre.  Reading: the paper gives no jack dimensions; the arm radius is R/3."""
    k = int(math.ceil(R / h))
    i = np.arange(-k, k + 1)
    I, J, K = np.meshgrid(i, i, i, indexing="ij")
    lat = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1).astype(np.float64) * h
    r2 = (lat * lat).sum(1)
    if shape == "sphere":
        m = r2 < R * R
    elif shape == "shell":
        m = (r2 < R * R) & (r2 >= (0.7 * R) ** 2)
    elif shape == "jack":
        a2 = (R / 3.0) ** 2
        m = np.zeros(len(lat), bool)
        for ax in range(3):
            o = [q for q in range(3) if q != ax]
            m |= (np.abs(lat[:, ax]) < R) & ((lat[:, o] ** 2).sum(1) < a2)
    else:
        raise ValueError(f"unknown shape {shape!r}")
    return lat[m]


def _box_walls(x: np.ndarray, rc: float, top_speed: float):
    """Six walls just out of reach of the extreme nodes; the top (+z) one moves down."""
    lo = x.min(axis=0) - rc
    hi = x.max(axis=0) + rc
    return [Wall((1.0, 0.0, 0.0), (lo[0], 0.0, 0.0), (0.0, 0.0, 0.0)),
            Wall((-1.0, 0.0, 0.0), (hi[0], 0.0, 0.0), (0.0, 0.0, 0.0)),
            Wall((0.0, 1.0, 0.0), (0.0, lo[1], 0.0), (0.0, 0.0, 0.0)),
            Wall((0.0, -1.0, 0.0), (0.0, hi[1], 0.0), (0.0, 0.0, 0.0)),
            Wall((0.0, 0.0, 1.0), (0.0, 0.0, lo[2]), (0.0, 0.0, 0.0)),
            Wall((0.0, 0.0, -1.0), (0.0, 0.0, hi[2]), (0.0, 0.0, -top_speed))], lo, hi


def shape_study(shape: str = "sphere", n_side: int = 5, seed: int = 0, R: float = 1e-3, h: float = 1e-3 / 8,
                gap_cells: float = 1.0, speed: float = 10.0, steps: int = 2000) -> Scenario:
    """The shape study of Sec. 6.5: n_side^3 particles of one shape (radius R = 1 mm)
    on a cubic grid (pitch 2R + gap), glass-like, in a box of six walls whose top wall
    moves down at ``speed`` (10 m/s).  Bulk strength is the difference of the top and
    bottom wall reactions over the top area.  Each particle is its own grain."""
    rng = np.random.default_rng(seed)
    nodes = shape_particle(shape, R, h)
    pitch = 2 * R + gap_cells * h
    xs, gs = [], []
    g = 0
    for a in range(n_side):
        for b in range(n_side):
            for c in range(n_side):
                xs.append(nodes + np.array([a, b, c], np.float64) * pitch + _jitter(rng, len(nodes), h))
                gs.append(np.full(len(nodes), g, np.int32))
                g += 1
    x = np.concatenate(xs)
    n = x.shape[0]
    mat = _glass(h)
    walls, lo, hi = _box_walls(x, mat.contact_radius, speed)
    return Scenario(name=f"shape_{shape}", x=x, vol=np.full(n, h ** 3), grain=np.concatenate(gs),
                    v0=np.zeros((n, 3)), material=mat, horizon=3 * h, h=h, walls=walls, steps=steps,
                    wall_area=float((hi[0] - lo[0]) * (hi[1] - lo[1])),
                    info={"shape": shape, "particles": n_side ** 3, "nodes_per_particle": len(nodes)})


def double_hollow(seed: int = 0, h: float = 4e-5, R: float = 1e-3, gap_cells: float = 1.0, speed: float = 10.0,
                  steps: int = 5000) -> Scenario:
    """Two hollow glass spheres (R = 1 mm, r = 0.7 R) stacked along z in a cubic
    container with fixed lateral and bottom walls and a top wall descending at
    ``speed`` (Sec. 6.3, double hollow sphere).  Reading: the paper gives no mesh
    size; h = 0.04 mm (two grains of ~43,000 nodes)."""
    rng = np.random.default_rng(seed)
    shell = shape_particle("shell", R, h)
    lower = shell + _jitter(rng, len(shell), h)
    upper = shell + np.array([0.0, 0.0, 2 * R + gap_cells * h]) + _jitter(rng, len(shell), h)
    x = np.concatenate([lower, upper])
    grain = np.concatenate([np.zeros(len(shell), np.int32), np.ones(len(shell), np.int32)])
    n = x.shape[0]
    mat = _glass(h)
    # cubic container: as wide as it is tall around the pair
    walls, lo, hi = _box_walls(x, mat.contact_radius, speed)
    half = 0.5 * float((hi - lo).max())
    mid = 0.5 * (lo + hi)
    lo_c, hi_c = mid - half, mid + half
    lo_c[2], hi_c[2] = lo[2], hi[2]
    walls = [Wall(w.normal, tuple(lo_c if sum(w.normal) > 0 else hi_c), w.velocity) for w in walls]
    return Scenario(name="double_hollow", x=x, vol=np.full(n, h ** 3), grain=grain, v0=np.zeros((n, 3)),
                    material=mat, horizon=3 * h, h=h, walls=walls, steps=steps,
                    wall_area=float((hi_c[0] - lo_c[0]) * (hi_c[1] - lo_c[1])))


def walls_array(walls) -> np.ndarray:
    """(nw, 9) float64 rows: normal, point, velocity."""
    if not walls:
        return np.zeros((0, 9))
    return np.array([list(w.normal) + list(w.point) + list(w.velocity) for w in walls], np.float64)


def filters_array(filters):
    """(kinds int32 (k,), params float64 (k,12))."""
    if not filters:
        return np.zeros(0, np.int32), np.zeros((0, 12))
    kinds = np.array([k for k, _ in filters], np.int32)
    params = np.array([list(a) + [0.0] * (12 - len(a)) for _, a in filters], np.float64)
    return kinds, params


BY_NAME = {"sphere": sphere, "kalthoff": kalthoff, "hollow": hollow, "aggregate": aggregate,
           "block": small_block, "shape_study": shape_study, "double_hollow": double_hollow}
