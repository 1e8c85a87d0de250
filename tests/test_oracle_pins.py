"""Pins of the CPU oracle to things other than itself (closed forms, invariants,
brute force, textbook special cases).  CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2506_05362_gb300 import scenarios as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def lattice_block(nx, ny, nz, h, jitter=0.0, seed=0):
    rng = np.random.default_rng(seed)
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    x = np.stack([I.ravel(), J.ravel(), K.ravel()], 1).astype(np.float64) * h
    if jitter:
        x = x + rng.uniform(-jitter * h, jitter * h, x.shape)
    return x


def model_for(x, mat, delta, walls=None, grain=None, vol=None, contact=True, body=(0, 0, 0), v0=None):
    n = x.shape[0]
    grain = np.zeros(n, np.int32) if grain is None else grain
    vol = np.full(n, 1.0) if vol is None else vol
    rp, col = oracle.bonds(x, grain, delta)
    return oracle.Model(x, vol, grain, rp, col, mat, delta, walls, body, v0, contact)


# --------------------------------------------------------------------------- constants
def test_micromodulus_matches_bulk_strain_energy():
    """Sec. 3.1: c is chosen so the PD energy matches the elastic one.  Under an
    isotropic stretch s every bond has stretch s; the PD energy density of a node
    with a full horizon is 1/2 * int_H 1/2 c s^2 |xi| dV, which must equal the
    elastic 1/2 K (tr eps)^2 = 9/2 K s^2.  The integral is done by quadrature."""
    E, G0, delta = 72e9, 135.0, 3e-4
    K, c, s0, Kn = oracle.constants(E, G0, delta)
    assert K == pytest.approx(E / (3 * (1 - 2 * GOLD["poisson_ratio_3d_bond_based"]["value"])), rel=1e-15)
    s = 1e-3
    radial, _ = integrate.quad(lambda r: 0.5 * c * s * s * r * 4 * math.pi * r * r, 0, delta)
    assert 0.5 * radial == pytest.approx(4.5 * K * s * s, rel=1e-12)


def test_critical_stretch_matches_fracture_energy():
    """Sec. 3.1.1: s0 equates G0 with the energy needed to break every bond that
    crosses a unit crack area.  Work to break one bond is 1/2 c s0^2 |xi| per
    unit volume squared; integrating over all bonds crossing the plane (Silling
    and Askari's construction) by quadrature must give G0."""
    E, G0, delta = 72e9, 135.0, 3e-4
    K, c, s0, Kn = oracle.constants(E, G0, delta)
    w = lambda r: 0.5 * c * s0 * s0 * r

    def inner(z):
        # bonds from a point at depth z below the crack plane to points above it
        # within the horizon: integral over |xi| in (z, delta) and polar angle
        # with cos(phi) > z/|xi|, weight 2 pi |xi|^2 sin(phi)
        return integrate.quad(lambda r: w(r) * 2 * math.pi * r * r * (1 - z / r), z, delta)[0]

    G, _ = integrate.quad(inner, 0, delta)
    assert G == pytest.approx(G0, rel=1e-10)


def test_paper_table_constants_switch():
    """The table's printed 3-D constant-micromodulus row, behind constants=1."""
    E, G0, delta = 72e9, 135.0, 3e-4
    _, c0, s00, _ = oracle.constants(E, G0, delta, mode=0)
    _, c1, s01, _ = oracle.constants(E, G0, delta, mode=1)
    assert c1 / c0 == pytest.approx(4.0 / 3.0, rel=1e-14)
    assert s01 / s00 == pytest.approx(math.sqrt(math.pi / 2), rel=1e-14)


# --------------------------------------------------------------------------- lists
@pytest.mark.parametrize("delta,key", [(3.0001, "interior_neighbours_up_to_3h"),
                                       (3.0, "interior_neighbours_strictly_inside_3h"),
                                       (4.0, "interior_neighbours_strictly_inside_4h")])
def test_lattice_neighbour_counts(delta, key):
    h = 1.0
    x = lattice_block(11, 11, 11, h)
    rp, col = oracle.bonds(x, np.zeros(len(x), np.int32), delta * h)
    centre = (5 * 11 + 5) * 11 + 5
    assert rp[centre + 1] - rp[centre] == GOLD[key]["value"]


def test_bonds_cells_equal_brute_and_symmetric():
    sc = S.aggregate(n_grains=2, h=0.5e-3 / 4)
    kinds = np.zeros(0, np.int32)
    a = oracle.bonds(sc.x, sc.grain, sc.horizon, brute=True)
    b = oracle.bonds(sc.x, sc.grain, sc.horizon, brute=False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    rp, col = a
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    fwd = set(zip(rows.tolist(), col.tolist()))
    assert all((j, i) in fwd for i, j in fwd)
    assert all(sc.grain[i] == sc.grain[j] for i, j in fwd)
    # row function agrees with the whole list
    for i in [0, 7, len(rp) - 2]:
        assert np.array_equal(oracle.bond_row(sc.x, sc.grain, sc.horizon, i), col[rp[i]:rp[i + 1]])


def test_notch_filter_cases():
    """Sec. 5.3.1: a bond whose segment meets the notch plane at 0 < t < 1 inside
    the notch face is removed; outside the face, or not crossing, it stays."""
    h = 1.0
    x = np.array([[0.0, -0.5, 0.0], [0.0, 0.5, 0.0],      # crosses y=0 inside the face
                  [5.0, -0.5, 0.0], [5.0, 0.5, 0.0],      # crosses y=0 outside the face
                  [0.0, 0.2, 9.0], [0.0, 1.2, 9.0]])       # does not cross
    grain = np.array([0, 0, 1, 1, 2, 2], np.int32)
    notch = [0.0, 1.0, 0.0, 0.0, -1.0, -0.1, -1.0, 1.0, 0.1, 10.0, 0.0, 0.0]
    rp, col = oracle.bonds(x, grain, 1.5 * h, [S.FILTER_NOTCH], [notch])
    assert list(np.diff(rp)) == [0, 0, 1, 1, 1, 1]


def test_sphere_filter_cases():
    """Sec. 5.3.2: bonds with an end strictly inside the inner sphere are removed."""
    x = np.array([[0.1, 0, 0], [0.9, 0, 0], [1.1, 0, 0], [1.9, 0, 0]])
    rp, col = oracle.bonds(x, np.zeros(4, np.int32), 1.0, [S.FILTER_SPHERE], [[0, 0, 0, 1.0] + [0] * 8])
    rows = {i: list(col[rp[i]:rp[i + 1]]) for i in range(4)}
    assert rows == {0: [], 1: [], 2: [3], 3: [2]}


def test_contact_pairs_grid_equals_brute():
    sc = S.aggregate(n_grains=3, h=0.5e-3 / 4, gap_cells=0.2, seed=3)
    m = oracle.Model.from_scenario(sc)
    rng = np.random.default_rng(1)
    m.u = rng.uniform(-0.5, 0.5, (m.n, 3)) * sc.h
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    pick = rng.random(len(m.col)) < 0.3
    und = set((min(i, j), max(i, j)) for i, j, p in zip(rows, m.col, pick) if p)
    m.broken[:] = [(min(i, j), max(i, j)) in und for i, j in zip(rows, m.col)]
    a = m.contact_pairs(brute=True)
    b = m.contact_pairs(brute=False)
    assert len(a) > 0
    assert np.array_equal(a, b)
    # symmetric, and no pair of the same grain with an intact bond
    sa = set(map(tuple, a.tolist()))
    assert all((j, i) in sa for i, j in sa)


# --------------------------------------------------------------------------- forces
def test_rigid_motion_gives_zero_force():
    """A rigid motion leaves every stretch at zero (Sec. 3.1), so F = 0."""
    mat = S.Material(E=72e9, rho=2440, G0=135, contact_radius=0.6e-3)
    x = lattice_block(6, 5, 4, 1e-3, jitter=0.01)
    m = model_for(x, mat, 3e-3, vol=np.full(len(x), 1e-9))
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    m.u = x @ R.T - x + np.array([0.3, -0.2, 0.1])
    F = m.forces()
    # scale: the force of one bond at unit stretch
    scale = m.c * 1e-9
    assert np.abs(F).max() < 1e-9 * scale
    assert m.broken.sum() == 0


def test_force_is_minus_energy_gradient():
    """Bond force density c s e V_j is the gradient of the PMB pair potential
    1/2 c s^2 |xi| (Sec. 3.1): F_i V_i = -dE/du_i.  Central differences of the
    oracle's energy must reproduce the oracle's force, term by term."""
    mat = S.Material(E=72e9, rho=2440, G0=1e12, contact_radius=0.3e-3)
    x = lattice_block(5, 4, 4, 1e-3, jitter=0.05, seed=2)
    V = np.full(len(x), 1e-9)
    m = model_for(x, mat, 2.5e-3, vol=V, contact=False)
    rng = np.random.default_rng(3)
    m.u = rng.uniform(-1, 1, m.u.shape) * 1e-6
    F = m.forces().copy()
    eps = 1e-10
    for i in [0, 13, 40]:
        for a in range(3):
            up = m.u.copy(); up[i, a] += eps
            dn = m.u.copy(); dn[i, a] -= eps
            m.u = up; Ep = m.energy()
            m.u = dn; Em = m.energy()
            m.u = (up + dn) / 2
            assert -(Ep - Em) / (2 * eps) == pytest.approx(F[i, a] * V[i], rel=2e-5, abs=1e-6 * np.abs(F * V[0]).max())


def test_momentum_balance():
    """Bond and contact forces are pairwise antisymmetric: sum_i F_i V_i = 0."""
    sc = S.aggregate(n_grains=3, h=0.5e-3 / 4, gap_cells=0.2, seed=5)
    m = oracle.Model.from_scenario(sc)
    rng = np.random.default_rng(4)
    m.u = rng.uniform(-0.3, 0.3, (m.n, 3)) * sc.h
    m.walls = np.zeros((0, 9)); m.P.nw = 0
    F = m.forces()
    tot = (F * sc.vol[:, None]).sum(0)
    assert np.abs(tot).max() < 1e-12 * np.abs(F * sc.vol[:, None]).sum()
    assert m.broken.sum() > 0  # large random motion breaks bonds


def test_breaking_threshold_and_memory():
    """gamma = 0 once s > s0 at any time (Sec. 3.1.1) and stays 0."""
    mat = S.Material(E=72e9, rho=2440, G0=135, contact_radius=0.1e-3)
    x = np.array([[0.0, 0, 0], [1e-3, 0, 0]])
    m = model_for(x, mat, 1.5e-3, vol=np.full(2, 1e-9))
    L = 1e-3
    for s, expect in [(m.s0 * (1 - 1e-9), 0), (m.s0 * (1 + 1e-9), 1)]:
        m.broken[:] = 0
        m.u[:] = 0
        m.u[1, 0] = s * L
        m.forces()
        assert list(m.broken) == [expect, expect]
    m.u[:] = 0
    m.forces()
    assert list(m.broken) == [1, 1]
    assert np.all(m.F == 0)
    # compression never breaks in the default tension mode, does in |s| mode
    m2 = model_for(x, mat, 1.5e-3, vol=np.full(2, 1e-9))
    m2.u[1, 0] = -2 * m2.s0 * L
    m2.forces()
    assert m2.broken.sum() == 0
    mat_abs = S.Material(E=72e9, rho=2440, G0=135, contact_radius=0.1e-3, break_mode=1)
    m3 = model_for(x, mat_abs, 1.5e-3, vol=np.full(2, 1e-9))
    m3.u[1, 0] = -2 * m3.s0 * L
    m3.forces()
    assert m3.broken.sum() == 2


def test_damage_counts():
    x = lattice_block(3, 1, 1, 1.0)
    m = model_for(x, S.Material(1, 1, 1, 0.1), 1.5)
    # rows: 0:[1], 1:[0,2], 2:[1]; break slot (1 -> 2)
    k = int(np.where((np.repeat(np.arange(3), np.diff(m.rowptr)) == 1) & (m.col == 2))[0][0])
    m.broken[k] = 1
    assert list(m.damage()) == [0.0, 0.5, 0.0]


# --------------------------------------------------------------------------- walls
@pytest.mark.parametrize("dfrac", [-0.7, -0.3, 0.0, 0.25, 0.6, 0.95])
def test_wall_cap_by_quadrature(dfrac):
    """Sec. 4.1: the wall force is K_n (R_c - |c_l - p|) |S_l| along the inward
    normal, |S_l| the volume of the part of the ball B_Rc(p) behind the wall and
    c_l its centroid.  Both are computed here by slicing the ball."""
    Rc = 2e-4
    mat = S.Material(E=72e9, rho=2440, G0=135, contact_radius=Rc)
    d = dfrac * Rc
    x = np.array([[0.0, 0.0, d]])
    walls = np.array([[0, 0, 1.0, 0, 0, 0, 0, 0, 0]])
    m = model_for(x, mat, 3e-4, walls=walls, vol=np.full(1, 1e-12))
    F = m.forces()
    # slices z' from -Rc to -d below the node (wall side): area pi (Rc^2 - z'^2)
    vol, _ = integrate.quad(lambda z: math.pi * (Rc * Rc - z * z), d, Rc)
    mom, _ = integrate.quad(lambda z: z * math.pi * (Rc * Rc - z * z), d, Rc)
    zbar = mom / vol
    expect = m.Kn * (Rc - zbar) * vol
    assert F[0, 2] == pytest.approx(expect, rel=1e-10)
    assert F[0, 0] == 0 and F[0, 1] == 0
    assert m.react[0, 2] == pytest.approx(-expect * 1e-12, rel=1e-10)
    if dfrac == 0.0:
        assert vol / Rc ** 3 == pytest.approx(GOLD["half_ball_volume_over_Rc3"]["value"], rel=1e-12)
        assert zbar == pytest.approx(3 * Rc / 8, rel=1e-12)


def test_wall_force_vanishes_at_contact_radius_and_flags_penetration():
    Rc = 1e-4
    mat = S.Material(E=72e9, rho=2440, G0=135, contact_radius=Rc)
    walls = np.array([[0, 0, 1.0, 0, 0, 0, 0, 0, 0]])
    m = model_for(np.array([[0, 0, Rc * (1 - 1e-6)]]), mat, 3e-4, walls=walls)
    F = m.forces()
    m0 = model_for(np.array([[0, 0, 0.0]]), mat, 3e-4, walls=walls)
    assert abs(F[0, 2]) < 1e-9 * m0.forces()[0, 2]
    mp = model_for(np.array([[0, 0, -1.01 * Rc]]), mat, 3e-4, walls=walls)
    mp.forces()
    assert mp.err & oracle.ERR_WALL


# --------------------------------------------------------------------------- dynamics
def test_free_fall_is_exact():
    """Velocity-Verlet integrates a constant acceleration exactly (Sec. 5.2)."""
    mat = S.Material(E=72e9, rho=2000.0, G0=135, contact_radius=1e-5)
    g = -9.81
    m = model_for(np.array([[0.0, 0, 0]]), mat, 1e-4, body=(0, 0, 2000.0 * g))
    m.init()
    dt = 1e-3
    m.step(dt, 100)
    t = 100 * dt
    assert m.u[0, 2] == pytest.approx(0.5 * g * t * t, rel=1e-12)
    assert m.v[0, 2] == pytest.approx(g * t, rel=1e-12)


def test_two_node_bond_oscillator_and_stability_limit():
    """Two nodes of volume V joined by one bond of length L oscillate with
    omega^2 = 2 c V / (rho L) (linearised PMB).  Verlet is stable for
    dt < 2/omega, which is exactly the critical step used for dt."""
    mat = S.Material(E=72e9, rho=2440, G0=1e12, contact_radius=1e-6)
    L, V = 1e-3, 1e-9
    x = np.array([[0.0, 0, 0], [L, 0, 0]])
    m = model_for(x, mat, 1.5e-3, vol=np.full(2, V))
    omega = math.sqrt(2 * m.c * V / (mat.rho * L))
    dtc = m.stable_dt()
    assert dtc == pytest.approx(2.0 / omega, rel=1e-12)
    amp = 1e-9
    m.u[1, 0] = amp
    m.init()
    dt = dtc / 200
    nper = int(round(2 * math.pi / omega / dt))
    m.step(dt, nper)
    T = nper * dt
    assert m.u[1, 0] - m.u[0, 0] == pytest.approx(amp * math.cos(omega * T), abs=2e-3 * amp)
    # stability limit
    for f, grows in [(0.98, False), (1.02, True)]:
        mm = model_for(x, mat, 1.5e-3, vol=np.full(2, V))
        mm.u[1, 0] = amp
        mm.init()
        mm.step(f * dtc, 400)
        assert (abs(mm.u[1, 0] - mm.u[0, 0]) > 10 * amp) == grows


def test_two_grain_contact_collision():
    """Two single-node grains meeting head-on: the linear contact spring
    K_n (R_c - |d|) V_i V_j (Sec. 3.2) gives a contact lasting pi sqrt(m_red / k),
    m_red = rho V / 2, k = K_n V^2, and an elastic rebound."""
    Rc, V, delta = 1e-4, 1e-12, 1e-3
    mat = S.Material(E=72e9, rho=2440, G0=135, contact_radius=Rc)
    vel = 0.05
    K, c, s0, Kn = oracle.constants(mat.E, mat.G0, delta)
    k = Kn * V * V
    mred = mat.rho * V / 2
    tc = math.pi * math.sqrt(mred / k)
    dt = tc / 2000
    x = np.array([[0.0, 0, 0], [Rc + 40 * dt * vel, 0, 0]])
    m = model_for(x, mat, delta, grain=np.array([0, 1], np.int32), vol=np.full(2, V),
                  v0=np.array([[vel, 0, 0], [-vel, 0, 0]]))
    assert len(m.col) == 0
    m.init()
    inside, t_in, t_out, t = False, None, None, 0.0
    for _ in range(20000):
        m.step(dt)
        t += dt
        d = (x[1, 0] + m.u[1, 0]) - (x[0, 0] + m.u[0, 0])
        if not inside and d < Rc:
            inside, t_in = True, t
        if inside and d >= Rc:
            t_out = t
            break
    assert t_out is not None
    assert t_out - t_in == pytest.approx(tc, rel=2e-3)
    assert m.v[0, 0] == pytest.approx(-vel, rel=1e-3)
    assert m.v[0, 0] + m.v[1, 0] == pytest.approx(0.0, abs=1e-12)


def test_energy_conserved_without_damage():
    """No breaking (G0 huge), no walls: velocity-Verlet on the conservative PMB
    forces keeps the energy bounded (no drift) with a fluctuation of order dt^2:
    halving dt over the same physical time divides it by about four."""
    mat = S.Material(E=72e9, rho=2440, G0=1e12, contact_radius=0.6e-3)
    x = lattice_block(7, 6, 5, 1e-3, jitter=0.01, seed=7)
    rng = np.random.default_rng(8)
    v0 = rng.normal(0, 0.1, (len(x), 3))
    fluct = []
    for frac, nsteps in [(0.2, 400), (0.1, 800)]:
        m = model_for(x, mat, 3e-3, vol=np.full(len(x), 1e-9), v0=v0)
        m.init()
        E0 = m.energy()
        dt = frac * m.stable_dt()
        es = []
        for _ in range(40):
            m.step(dt, nsteps // 40)
            es.append(m.energy())
        es = np.array(es)
        fluct.append(np.abs(es - E0).max() / E0)
        assert abs(es[-10:].mean() - es[:10].mean()) / E0 < 2 * fluct[-1]
    assert fluct[1] < 2e-3
    assert 3.0 < fluct[0] / fluct[1] < 5.0


def test_bulk_stress_sign_convention():
    """Compression is negative: plates pushed apart by the aggregate."""
    normals = np.array([[0, 0, -1.0], [0, 0, 1.0]])
    react = np.array([[0, 0, 5.0], [0, 0, -5.0]])
    s = oracle.bulk_stress(normals, react, [2.0, 2.0])
    assert s[2] == pytest.approx(-2.5)
    assert np.all(s[[0, 1, 3, 4, 5]] == 0)


def test_wall_impulse_balances_momentum():
    """Newton's second law over a window of steps: bond and contact forces cancel
    in sum_i V_i F_i, so the body's momentum changes only by the wall forces.
    Velocity Verlet integrates them with the trapezoid rule, the accumulated
    impulse J with the rectangle rule at the step ends; hence
    rho sum_i V_i (v_N - v_0) = -(J + dt (R_0 - R_N) / 2), summed over walls."""
    sc = S.sphere()
    m = oracle.Model.from_scenario(sc)
    dt = 0.8 * m.stable_dt()
    m.init()
    m.step(dt, 60)          # walls reach the sphere
    m.bulk_stress_mean([1.0, 1.0])   # reset the accumulator
    R0 = m.react.sum(0)
    p0 = sc.material.rho * (m.v * sc.vol[:, None]).sum(0)
    m.step(dt, 120)
    RN = m.react.sum(0)
    p1 = sc.material.rho * (m.v * sc.vol[:, None]).sum(0)
    J = m.impulse.sum(0)
    assert np.abs(m.impulse).max() > 0, "walls should touch the sphere"
    lhs = p1 - p0
    rhs = -(J + 0.5 * dt * (R0 - RN))
    assert np.abs(lhs).max() > 0.1 * np.abs(J).max()   # the momentum really changed
    assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(m.impulse).sum()
    J_walls = m.impulse.copy()
    sig, mean, span = m.bulk_stress_mean([sc.wall_area] * 2)
    assert span == pytest.approx(120 * dt, rel=1e-15)
    assert np.allclose(mean, J_walls / span, rtol=1e-15, atol=0)
    assert np.all(m.impulse == 0) and m.impulse_span == 0.0
    # the mean stress is the stress of the mean wall forces
    assert np.allclose(sig, oracle.bulk_stress(m.walls[:, 0:3], mean, [sc.wall_area] * 2), rtol=0, atol=0)


@pytest.mark.parametrize("zeta", [0.1, 0.3, 0.6])
def test_damped_contact_restitution(zeta):
    """Normal damping (Sec. 3.3) on two single-node grains meeting head-on: spring
    K_n (R_c - |d|) V V plus dashpot beta_d (v_rel . e) V V is the damped linear
    oscillator with damping ratio zeta = beta_d V^2 / (2 sqrt(k m_red)): contact
    lasts pi / (omega_0 sqrt(1 - zeta^2)) and the rebound keeps the fraction
    exp(-zeta pi / sqrt(1 - zeta^2)) of the approach speed."""
    Rc, V, delta = 1e-4, 1e-12, 1e-3
    K, c, s0, Kn = oracle.constants(72e9, 135, delta)
    rho = 2440.0
    k = Kn * V * V
    mred = rho * V / 2
    beta = zeta * 2 * math.sqrt(k * mred) / (V * V)
    mat = S.Material(E=72e9, rho=rho, G0=135, contact_radius=Rc, beta_d=beta)
    vel = 0.05
    w0 = math.sqrt(k / mred)
    td = math.pi / (w0 * math.sqrt(1 - zeta ** 2))
    dt = td / 4000
    x = np.array([[0.0, 0, 0], [Rc + 40 * dt * vel, 0, 0]])
    m = model_for(x, mat, delta, grain=np.array([0, 1], np.int32), vol=np.full(2, V),
                  v0=np.array([[vel, 0, 0], [-vel, 0, 0]]))
    m.init()
    inside, t_in, t_out, t = False, None, None, 0.0
    for _ in range(40000):
        m.step(dt)
        t += dt
        d = (x[1, 0] + m.u[1, 0]) - (x[0, 0] + m.u[0, 0])
        if not inside and d < Rc:
            inside, t_in = True, t
        if inside and d >= Rc:
            t_out = t
            break
    assert t_out is not None
    assert t_out - t_in == pytest.approx(td, rel=2e-3)
    e = math.exp(-zeta * math.pi / math.sqrt(1 - zeta ** 2))
    assert -m.v[0, 0] / vel == pytest.approx(e, rel=3e-3)
    assert m.v[0, 0] + m.v[1, 0] == pytest.approx(0.0, abs=1e-12)   # momentum


def test_damping_forces_conserve_momentum_and_dissipate():
    """Pair damping is antisymmetric (sum_i V_i F_i = 0) and never does positive
    work on the relative motion: sum_i V_i F_d,i . v_i <= 0."""
    h = 1e-4
    a = lattice_block(5, 5, 4, h, jitter=0.05, seed=1)
    b = lattice_block(5, 5, 4, h, jitter=0.05, seed=2) + np.array([0.2 * h, 0.3 * h, 3.55 * h])
    x = np.concatenate([a, b])
    grain = np.repeat(np.array([0, 1], np.int32), len(a))
    vol = np.full(len(x), h ** 3)
    mat = S.Material(E=72e9, rho=2440, G0=135, contact_radius=0.6 * h, beta_d=1e9)
    m = model_for(x, mat, 3 * h, grain=grain, vol=vol)
    rng = np.random.default_rng(9)
    m.v = rng.normal(0, 1.0, (m.n, 3))
    sc = S.Scenario(name="pair", x=x, vol=vol, grain=grain, v0=m.v, material=mat, horizon=3 * h, h=h)
    F1 = m.forces(frozen=False).copy()
    pairs = len(m.contact_pairs())
    assert pairs > 0
    m.P.beta_d = 0.0
    F0 = m.forces(frozen=True).copy()
    Fd = F1 - F0
    assert np.abs(Fd).max() > 0
    tot = (Fd * sc.vol[:, None]).sum(0)
    assert np.abs(tot).max() < 1e-12 * np.abs(Fd * sc.vol[:, None]).sum()
    assert (Fd * sc.vol[:, None] * m.v).sum() < 0


def test_wall_damping_closed_form():
    """Damping at a wall (Sec. 4.1 substitution): a node at distance d moving with
    v feels beta_d ((v_w - v) . n) n |S| more than without damping, with the cap
    volume |S| = (pi/3)(R_c - d)^2 (2 R_c + d)."""
    Rc = 1e-4
    x = np.array([[0.0, 0.0, 0.4 * Rc]])
    vw = np.array([0.0, 0.0, 0.3])
    walls = np.array([[0, 0, 1.0, 0, 0, 0, *vw]])
    v = np.array([[0.2, -0.1, -1.5]])
    d = 0.4 * Rc
    S_cap = math.pi / 3 * (Rc - d) ** 2 * (2 * Rc + d)
    mat = S.Material(E=72e9, rho=2440, G0=135, contact_radius=Rc)
    m = model_for(x, mat, 3e-4, walls=walls, vol=np.full(1, 1e-12), v0=v)
    F0 = m.forces().copy()
    # a coefficient that makes damping a tenth of the repulsion here
    beta = 0.1 * abs(F0[0, 2]) / (abs((vw - v[0])[2]) * S_cap)
    m.P.beta_d = beta
    F1 = m.forces().copy()
    R1 = m.react.copy()
    expect = beta * ((vw - v[0]) @ np.array([0, 0, 1.0])) * S_cap
    assert expect > 0   # the wall pushes a node that approaches it
    assert F1[0] - F0[0] == pytest.approx([0, 0, expect], rel=1e-12, abs=1e-12 * abs(expect))
    assert R1[0] == pytest.approx(-F1[0] * 1e-12, rel=1e-12)


# --------------------------------------------------------------------------- fragments
def random_bond_graph(n, deg, frac_broken, seed):
    """Symmetric random graph as a caller-order CSR with ascending rows and a
    symmetric broken pattern."""
    rng = np.random.default_rng(seed)
    pairs = set()
    for i in range(n):
        for j in rng.choice(n, deg, replace=False):
            if j != i:
                pairs.add((min(i, j), max(i, j)))
    pairs = sorted(pairs)
    brk_pair = {p: rng.random() < frac_broken for p in pairs}
    rows = [[] for _ in range(n)]
    for (a, b) in pairs:
        rows[a].append(b)
        rows[b].append(a)
    rowptr = np.zeros(n + 1, np.int64)
    col, broken = [], []
    for i in range(n):
        r = sorted(rows[i])
        rowptr[i + 1] = rowptr[i] + len(r)
        col += r
        broken += [brk_pair[(min(i, j), max(i, j))] for j in r]
    return rowptr, np.array(col, np.int32), np.array(broken, np.uint8)


@pytest.mark.parametrize("n,deg,frac,seed", [(1, 0, 0.0, 0), (60, 2, 0.5, 1), (500, 3, 0.6, 2), (2000, 4, 0.45, 3)])
def test_fragments_match_connected_components(n, deg, frac, seed):
    """Fragments are the connected components of the intact-bond graph: the same
    partition as scipy's connected_components, labelled by the smallest member."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    rowptr, col, broken = random_bond_graph(n, deg, frac, seed)
    label, nf = oracle.fragments(rowptr, col, broken)
    data = (broken == 0).astype(np.int8)
    G = csr_matrix((data, col.copy(), rowptr.copy()), shape=(n, n))  # eliminate_zeros works in place
    G.eliminate_zeros()
    ncc, cc = connected_components(G, directed=False)
    assert nf == ncc
    # same partition: the map component -> label is one-to-one
    assert len(set(zip(cc.tolist(), label.tolist()))) == ncc
    # labels are the smallest member of each component
    for c in range(ncc):
        members = np.flatnonzero(cc == c)
        assert np.all(label[members] == members.min())
    # no intact bond crosses two fragments
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    intact = broken == 0
    assert np.all(label[rows[intact]] == label[col[intact]])


def test_fragment_stats_by_hand():
    """Two blocks bonded inside, one bond between them broken: two fragments with
    the right sizes, volumes and broken fractions (counted by hand)."""
    # path 0-1-2 | 3-4 ; bonds (0,1),(1,2),(2,3) broken,(3,4) broken
    rowptr = np.array([0, 1, 3, 5, 7, 8], np.int64)
    col = np.array([1, 0, 2, 1, 3, 2, 4, 3], np.int32)
    broken = np.array([0, 0, 0, 0, 1, 1, 1, 1], np.uint8)
    label, nf = oracle.fragments(rowptr, col, broken)
    assert nf == 3 and label.tolist() == [0, 0, 0, 3, 4]
    size, vol, dmg = oracle.fragment_stats(rowptr, broken, np.array([1.0, 2, 3, 4, 5]), label, nf)
    assert size.tolist() == [3, 1, 1]
    assert vol.tolist() == [6.0, 4.0, 5.0]
    # fragment {0,1,2}: slots 1+2+2 = 5, intact 4 -> 1/5 broken; {3}: 2 slots, none intact; {4}: 1 slot
    assert dmg == pytest.approx([0.2, 1.0, 1.0])


# --------------------------------------------------------------------------- conic micromodulus
def test_conic_micromodulus_energy_and_fracture():
    """Conic micromodulus c (delta - |xi|) (table of Sec. 3.1.1): the coefficient
    matches the bulk strain energy and s0 the crack energy, by the same
    quadratures as the constant case; the printed row sits behind constants=1."""
    E, G0, delta = 72e9, 135.0, 3e-4
    K, c, s0, Kn = oracle.constants(E, G0, delta, micromodulus=1)
    cw = lambda r: c * (delta - r)
    s = 1e-3
    radial, _ = integrate.quad(lambda r: 0.5 * cw(r) * s * s * r * 4 * math.pi * r * r, 0, delta)
    assert 0.5 * radial == pytest.approx(4.5 * K * s * s, rel=1e-12)
    w = lambda r: 0.5 * cw(r) * s0 * s0 * r

    def inner(z):
        return integrate.quad(lambda r: w(r) * 2 * math.pi * r * r * (1 - z / r), z, delta)[0]

    G, _ = integrate.quad(inner, 0, delta)
    assert G == pytest.approx(G0, rel=1e-10)
    _, c1, s01, Kn1 = oracle.constants(E, G0, delta, mode=1, micromodulus=1)
    assert c1 / c == pytest.approx(4.0 / 3.0, rel=1e-14)
    assert s01 / s0 == pytest.approx(math.sqrt(7 * math.pi / 12), rel=1e-14)
    assert Kn1 == Kn  # contact stiffness is defined from K, not from c


def test_conic_bond_force_by_hand():
    """Two nodes, one bond of length L stretched by s: the force density on node
    0 is c (delta - L) s V_1 along the bond."""
    mat = S.Material(E=72e9, rho=2440, G0=1e12, contact_radius=1e-5, micromodulus=1)
    L, delta, V = 1e-4, 3e-4, 1e-12
    m = model_for(np.array([[0.0, 0, 0], [L, 0, 0]]), mat, delta, vol=np.full(2, V), contact=False)
    s = 2e-4
    m.u = np.array([[0.0, 0, 0], [s * L, 0, 0]])
    F = m.forces()
    K, c, s0, _ = oracle.constants(mat.E, mat.G0, delta, micromodulus=1)
    assert F[0, 0] == pytest.approx(c * (delta - L) * s * V, rel=1e-12)
    assert F[1, 0] == pytest.approx(-F[0, 0], rel=1e-15)


# --------------------------------------------------------------------------- self-contact (PD-repulsive branch)
def _self_contact_pair(micromodulus, L=0.4e-4, h=1e-4, V1=2e-12):
    """Two nodes of one grain closer than the contact radius (R_c = 0.6 h), bonded
    (horizon 3 h), unequal volumes."""
    mat = S.Material(E=72e9, rho=2440, G0=135, contact_radius=0.6 * h, micromodulus=micromodulus)
    x = np.array([[0.0, 0, 0], [L, 0, 0]])
    m = model_for(x, mat, 3 * h, vol=np.array([1e-12, V1]))
    assert len(m.col) == 2
    return m, mat


@pytest.mark.parametrize("micromodulus", [0, 1])
@pytest.mark.parametrize("dfrac", [0.3, 0.75, 1.3])
def test_self_contact_repulsive_branch_by_hand(micromodulus, dfrac):
    """Self-contact (Sec. 5, same-grain law): a once-bonded pair of one grain with
    |xi| < R_c whose bond is broken repels only in compression, with the PD law
    c(|xi|) (|d| - |xi|)/|xi| e V_j -- not the inter-grain spring K_n (R_c - |d|).
    Hand values: |xi| = 0.4 h, |d| = dfrac |xi| along x; in tension (|d| > |xi|, still
    inside R_c = 0.6 h) the pair exerts nothing.  Unequal volumes: F_i V_i = -F_j V_j."""
    L = 0.4e-4
    m, mat = _self_contact_pair(micromodulus, L=L)
    delta = 3e-4
    K, c, s0, Kn = oracle.constants(mat.E, mat.G0, delta, micromodulus=micromodulus)
    cw = c * (delta - L) if micromodulus else c
    m.broken[:] = 1
    d = dfrac * L
    m.u = np.array([[0.0, 0, 0], [d - L, 0, 0]])
    F = m.forces(frozen=True)
    expect0 = cw * min(0.0, (d - L) / L) * m.vol[1]  # along +x (e points from node 0 to node 1)
    if dfrac < 1:
        assert expect0 < 0  # node 0 is pushed away from node 1
        assert F[0, 0] == pytest.approx(expect0, rel=1e-12)
        # a spring of the inter-grain law would give -K_n (R_c - |d|) V_j: a different value
        assert abs(-Kn * (mat.contact_radius - d) * m.vol[1] - expect0) > 1e-3 * abs(expect0)
    else:
        assert F[0, 0] == 0.0
    assert np.all(F[:, 1:] == 0.0)
    assert F[0, 0] * m.vol[0] == pytest.approx(-F[1, 0] * m.vol[1], rel=1e-14, abs=0)


@pytest.mark.parametrize("micromodulus", [0, 1])
def test_self_contact_equals_the_intact_bond_in_compression(micromodulus):
    """The self-contact law is the bond law restricted to repulsion: a compressed
    once-bonded pair feels the same force whether its bond is intact or broken,
    and a stretched one only while the bond is intact.  Off the bond axis too."""
    L = 0.4e-4
    m, _ = _self_contact_pair(micromodulus, L=L)
    rng = np.random.default_rng(5)
    for trial in range(6):
        direction = rng.normal(size=3)
        direction /= np.linalg.norm(direction)
        compress = trial % 2 == 0
        d = (0.6 if compress else 1.2) * L
        m.u = np.vstack([np.zeros(3), d * direction - np.array([L, 0, 0])])
        m.broken[:] = 0
        Fb = m.forces(frozen=True).copy()
        m.broken[:] = 1
        Fc = m.forces(frozen=True).copy()
        if compress:
            assert np.allclose(Fc, Fb, rtol=1e-12, atol=0)
            assert np.dot(Fc[0], direction) < 0
        else:
            assert np.all(Fc == 0.0)
            assert np.dot(Fb[0], direction) > 0  # the intact bond pulls


def test_self_contact_spring_branch_beyond_contact_radius():
    """Same grain with |xi| >= R_c (never closer than R_c in the reference): once
    unbonded and pushed inside R_c the pair takes the spring -K_n (R_c - |d|) V_j."""
    h = 1e-4
    mat = S.Material(E=72e9, rho=2440, G0=135, contact_radius=0.6 * h)
    L = 0.9 * h
    m = model_for(np.array([[0.0, 0, 0], [L, 0, 0]]), mat, 3 * h, vol=np.full(2, 1e-12))
    K, c, s0, Kn = oracle.constants(mat.E, mat.G0, 3 * h)
    m.broken[:] = 1
    d = 0.5 * h
    m.u = np.array([[0.0, 0, 0], [d - L, 0, 0]])
    F = m.forces(frozen=True)
    assert F[0, 0] == pytest.approx(-Kn * (mat.contact_radius - d) * 1e-12, rel=1e-12)
    assert F[1, 0] == pytest.approx(-F[0, 0], rel=1e-15)


# --------------------------------------------------------------------------- OpenMP build
def test_openmp_build_gives_the_same_bits():
    """The OpenMP build of the oracle (timed as the all-core CPU baseline) runs
    the same per-node arithmetic: forces with contacts and breaking, and a short
    trajectory, are bit-identical to the serial build's."""
    sc = S.aggregate(n_grains=3, h=0.5e-3 / 4, gap_cells=0.2, seed=3)
    rng = np.random.default_rng(1)
    u = rng.uniform(-0.5, 0.5, (sc.n, 3)) * sc.h
    out = []
    threads = oracle.set_threads(4)
    assert threads == 4
    for par in (False, True):
        m = oracle.Model.from_scenario(sc, parallel=par)
        # a third of the undirected bonds broken (both slots), so that fragments touch
        rows = np.repeat(np.arange(sc.n), np.diff(m.rowptr))
        key = np.minimum(rows, m.col).astype(np.int64) * (sc.n + 1) + np.maximum(rows, m.col)
        uniq, inv = np.unique(key, return_inverse=True)
        m.broken[:] = (np.random.default_rng(2).random(len(uniq)) < 0.3)[inv]
        m.u = u.copy()
        F = m.forces().copy()
        pairs = len(m.contact_pairs())
        m.init()
        m.step(0.5 * m.stable_dt(), 5)
        out.append((F, m.broken.copy(), m.u.copy(), m.v.copy(), m.react.copy(), pairs))
    assert out[0][5] > 0 and out[0][1].sum() > 0
    for a, b in zip(out[0][:5], out[1][:5]):
        assert np.array_equal(a, b)
