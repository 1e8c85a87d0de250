"""Pins of the oracle's stick-slip friction (Sec. 3.3) and of the multi-wall
inclusion-exclusion (Sec. 4.1.1): closed forms, identities the integration
order does not know about, a library quadrature and a voxel count for the
ball-cut volumes, and hand-computed forces."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2506_05362_gb300 import scenarios as S


def model_for(x, mat, delta, walls=None, grain=None, vol=None, v0=None):
    n = x.shape[0]
    grain = np.zeros(n, np.int32) if grain is None else grain
    vol = np.full(n, 1.0) if vol is None else vol
    rp, col = oracle.bonds(x, grain, delta)
    return oracle.Model(x, vol, grain, rp, col, mat, delta, walls, (0, 0, 0), v0, True)


def cap(R, a):
    """Spherical cap {X > a} of the ball: volume and X moment (textbook)."""
    return math.pi / 3 * (R - a) ** 2 * (2 * R + a), math.pi / 4 * (R * R - a * a) ** 2


# --------------------------------------------------------------------------- ball cuts
def test_ball_cut_closed_forms():
    R = 1.7
    V, mx, my, mz = oracle.ball_cut(R, 0.0, 0.0)  # quarter ball, centroid 3R/8 along X and Y
    assert V == pytest.approx(math.pi * R ** 3 / 3, rel=1e-12)
    assert mx / V == pytest.approx(3 * R / 8, rel=1e-11) and my / V == pytest.approx(3 * R / 8, rel=1e-11)
    assert mz == 0.0
    V, mx, my, mz = oracle.ball_cut(R, 0.0, 0.0, 0.0)  # octant
    assert V == pytest.approx(math.pi * R ** 3 / 6, rel=1e-11)
    for m in (mx, my, mz):
        assert m / V == pytest.approx(3 * R / 8, rel=1e-10)
    for a in (-0.9, -0.3, 0.0, 0.25, 0.8):
        Vc, Mc = cap(R, a * R)
        V, mx, my, mz = oracle.ball_cut(R, a * R, -R)
        assert V == pytest.approx(Vc, rel=1e-12) and mx == pytest.approx(Mc, rel=1e-11)
        assert abs(my) < 1e-13 * R ** 4 and mz == 0.0
        V3 = oracle.ball_cut(R, -R, -R, a * R)  # the nested path: cap along Z
        assert V3[0] == pytest.approx(Vc, rel=1e-10) and V3[3] == pytest.approx(Mc, rel=1e-10)
    # beyond the ball's reach: empty
    assert np.all(oracle.ball_cut(R, 0.8 * R, 0.7 * R) == 0)
    assert np.all(oracle.ball_cut(R, 0.6 * R, 0.6 * R, 0.6 * R) == 0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ball_cut_complements_and_permutations(seed):
    """{Y > b} and the mirror image of {Y < b} add up to the cap; the same for Z;
    permuting the axes permutes the moments (the integration order is fixed)."""
    rng = np.random.default_rng(seed)
    R = 1.0
    a, b, c = rng.uniform(-0.8, 0.8, 3)
    Vc, Mc = cap(R, a)
    p, m = oracle.ball_cut(R, a, b), oracle.ball_cut(R, a, -b)
    assert p[0] + m[0] == pytest.approx(Vc, rel=1e-12)
    assert p[1] + m[1] == pytest.approx(Mc, rel=1e-12)
    assert p[2] == pytest.approx(m[2], rel=1e-10, abs=1e-14)
    t, u = oracle.ball_cut(R, a, b, c), oracle.ball_cut(R, a, b, -c)
    assert t[0] + u[0] == pytest.approx(p[0], rel=1e-11, abs=1e-13)
    assert t[1] + u[1] == pytest.approx(p[1], rel=1e-11, abs=1e-13)
    assert t[2] + u[2] == pytest.approx(p[2], rel=1e-11, abs=1e-13)
    assert t[3] == pytest.approx(u[3], rel=1e-10, abs=1e-13)
    q = oracle.ball_cut(R, c, a, b)  # axes (X, Y, Z) <- (c, a, b)
    assert q[0] == pytest.approx(t[0], rel=1e-11, abs=1e-13)
    assert q[1] == pytest.approx(t[3], rel=1e-10, abs=1e-13)
    assert q[2] == pytest.approx(t[1], rel=1e-10, abs=1e-13)
    assert q[3] == pytest.approx(t[2], rel=1e-10, abs=1e-13)
    r = oracle.ball_cut(R, b, a)  # two planes swapped
    assert r[0] == pytest.approx(p[0], rel=1e-12) and r[1] == pytest.approx(p[2], rel=1e-10, abs=1e-14)


def test_ball_cut_against_library_quadrature_and_voxels():
    R, a, b, c = 1.0, 0.15, -0.35, 0.05
    # scipy's adaptive quadrature (QUADPACK) over X then Y of the Z extent
    def zlen(y, x):
        w2 = R * R - x * x - y * y
        if w2 <= 0:
            return 0.0
        w = math.sqrt(w2)
        return max(0.0, w - max(c, -w))
    ymax = lambda x: math.sqrt(max(R * R - x * x, 0.0))
    ylo = lambda x: max(b, -ymax(x))
    V, _ = integrate.dblquad(zlen, a, R, ylo, ymax, epsabs=1e-12, epsrel=1e-12)
    MX, _ = integrate.dblquad(lambda y, x: x * zlen(y, x), a, R, ylo, ymax, epsabs=1e-12, epsrel=1e-12)
    t = oracle.ball_cut(R, a, b, c)
    assert t[0] == pytest.approx(V, rel=1e-8) and t[1] == pytest.approx(MX, rel=1e-8)
    # voxel count (cell centres) on a 200^3 grid over the cube [-R, R]^3
    n = 200
    g = (np.arange(n) + 0.5) / n * 2 * R - R
    h3 = (2 * R / n) ** 3
    vol = 0.0
    mom = np.zeros(3)
    X, Y = np.meshgrid(g, g, indexing="ij")
    for z in g:
        m = (X * X + Y * Y + z * z < R * R) & (X > a) & (Y > b) & (z > c)
        cnt = m.sum()
        vol += cnt * h3
        mom += np.array([X[m].sum(), Y[m].sum(), z * cnt]) * h3
    assert t[0] == pytest.approx(vol, rel=3e-3)
    assert np.allclose(t[1:], mom, rtol=1e-2, atol=3e-3 * R ** 4)


# --------------------------------------------------------------------------- friction
MAT = dict(E=72e9, rho=2440.0, G0=135.0)


def pair_model(mu, Vi=2e-12, Vj=0.5e-12, Rc=1e-4, gap=0.7):
    x = np.array([[0.0, 0.0, 0.0], [gap * Rc, 0.0, 0.0]])
    mat = S.Material(contact_radius=Rc, mu=mu, **MAT)
    return model_for(x, mat, 3e-4, grain=np.array([0, 1], np.int32), vol=np.array([Vi, Vj]))


@pytest.mark.parametrize("vn", [0.0, 0.7])
def test_friction_slip_stick_and_coulomb_limit_by_hand(vn):
    """Relative tangential velocity along y (the contact normal is x):
    slip gives mu f_r V_j against the slip, stick rho |v_t| V_j / (dt (V_i + V_j)),
    dt = 0 the Coulomb limit; a normal velocity changes nothing; momentum holds."""
    Rc, gap, mu = 1e-4, 0.7, 0.4
    m0 = pair_model(0.0)
    m0.v = np.array([[vn, 0.0, 0.0], [0.0, 0.0, 0.0]])
    F0 = m0.forces().copy()
    fr = m0.Kn * (Rc - gap * Rc)  # repulsion per volume squared
    Vi, Vj = 2e-12, 0.5e-12
    rho = MAT["rho"]
    dt = 1e-8
    for vy, stick in ((500.0, False), (1e-9, True)):
        m = pair_model(mu)
        m.v = np.array([[vn, vy, 0.0], [0.0, 0.0, 0.0]])
        m.P.dt_f = dt
        dF = m.forces().copy() - F0
        f_slip = mu * fr
        f_stick = rho * vy / (dt * (Vi + Vj))
        assert (f_stick < f_slip) == stick
        f = min(f_slip, f_stick)
        assert dF[0, 1] == pytest.approx(-f * Vj, rel=1e-12)
        assert dF[1, 1] == pytest.approx(f * Vi, rel=1e-12)
        assert dF[0, 0] == 0 and dF[0, 2] == 0 and dF[1, 0] == 0 and dF[1, 2] == 0
        assert abs(dF[0, 1] * Vi + dF[1, 1] * Vj) < 1e-14 * abs(dF[0, 1] * Vi)
        m.P.dt_f = 0.0  # Coulomb limit: the slip branch at any speed
        dF = m.forces().copy() - F0
        assert dF[0, 1] == pytest.approx(-f_slip * Vj, rel=1e-12)


def test_friction_stops_an_isolated_pair_in_one_step():
    """Stick branch: friction takes away an isolated pair's whole relative
    tangential velocity by the next half step (the property the paper gives for
    eps_f = dt / rho).  The repulsion turns with the contact normal during the
    step; the run without friction takes most of that part out, and a pair
    just inside the contact radius keeps the rest (~1e-7) small."""
    dt = 1e-9
    rel = []
    for mu in (0.5, 0.0):
        m = pair_model(mu, gap=0.999)
        m.v = np.array([[0.0, 2e-7, 0.0], [0.0, -1e-7, 0.0]])
        m.P.dt_f = dt
        m.init()
        m.step(dt, 1)
        vh = m.v + 0.5 * dt * m.acc
        rel.append(vh[0, 1] - vh[1, 1])
    assert MAT["rho"] * 3e-7 / (dt * 2.5e-12) < 0.5 * m.Kn * 1e-7  # the stick branch
    assert rel[0] - rel[1] == pytest.approx(-3e-7, rel=1e-6, abs=0)


def test_friction_conserves_momentum_and_dissipates():
    """Two jittered blocks of different grains with unequal volumes in contact:
    the friction forces sum to zero momentum and do negative work."""
    h = 1e-4
    rng = np.random.default_rng(4)
    a = rng.uniform(0, 4 * h, (60, 3))
    b = rng.uniform(0, 4 * h, (60, 3)) + np.array([0.0, 0.0, 3.7 * h])
    x = np.concatenate([a, b])
    grain = np.repeat(np.array([0, 1], np.int32), 60)
    vol = rng.uniform(0.5, 1.5, len(x)) * h ** 3
    for dt in (1e-8, 1e-12):  # mostly slip; mostly stick
        m0 = model_for(x, S.Material(contact_radius=0.9 * h, **MAT), 3 * h, grain=grain, vol=vol)
        m1 = model_for(x, S.Material(contact_radius=0.9 * h, mu=0.3, **MAT), 3 * h, grain=grain, vol=vol)
        v = rng.normal(0, 1.0, x.shape)
        m0.v, m1.v = v, v.copy()
        m1.P.dt_f = dt
        Ff = m1.forces().copy() - m0.forces().copy()
        assert len(m1.contact_pairs()) > 0 and np.abs(Ff).max() > 0
        tot = (Ff * vol[:, None]).sum(0)
        assert np.abs(tot).max() < 1e-12 * np.abs(Ff * vol[:, None]).sum()
        assert (Ff * vol[:, None] * v).sum() < 0


def test_wall_friction_closed_form():
    """A node at distance d from a wall sliding along it: slip gives
    mu K_n (R_c - zbar) |S| against the slip, stick rho |v_t| / dt; the wall's
    reaction takes the opposite, times V_i; a node moving with the wall feels none."""
    Rc, d, mu, Vi = 1e-4, 0.3e-4, 0.6, 1e-12
    walls = np.array([[0, 0, 1.0, 0, 0, 0, 0.1, 0.0, 0.0]])  # the wall slides along x at 0.1 m/s
    Vcap = math.pi / 3 * (Rc - d) ** 2 * (2 * Rc + d)
    zbar = math.pi / 4 * (Rc * Rc - d * d) ** 2 / Vcap
    dt = 1e-8
    rho = MAT["rho"]
    for vx, stick in ((300.0, False), (0.1 + 1e-9, True), (0.1, None)):
        out = []
        for mu_ in (0.0, mu):
            m = model_for(np.array([[0.0, 0.0, d]]), S.Material(contact_radius=Rc, mu=mu_, **MAT), 3e-4,
                          walls=walls, vol=np.full(1, Vi))
            m.v = np.array([[vx, 0.0, -0.2]])
            m.P.dt_f = dt
            out.append((m.forces().copy(), m.react.copy(), m.Kn))
        dF, dR, Kn = out[1][0] - out[0][0], out[1][1] - out[0][1], out[1][2]
        vt = vx - 0.1
        if stick is None:
            assert np.all(dF == 0)
            continue
        f = min(mu * Kn * (Rc - zbar) * Vcap, rho * abs(vt) / dt)
        assert (rho * abs(vt) / dt < mu * Kn * (Rc - zbar) * Vcap) == stick
        assert dF[0, 0] == pytest.approx(-f * np.sign(vt), rel=1e-9)
        assert dF[0, 1] == 0 and dF[0, 2] == 0
        assert dR[0, 0] == pytest.approx(f * np.sign(vt) * Vi, rel=1e-9)


def test_bulk_stress_shear_from_tangential_reaction():
    """A tangential wall reaction shows up as shear; Cauchy's relation per wall."""
    normals = np.array([[0, 0, -1.0], [0, 0, 1.0]])
    react = np.array([[2.0, 0, 5.0], [-2.0, 0, -5.0]])
    s = oracle.bulk_stress(normals, react, [2.0, 2.0])
    assert s[2] == pytest.approx(-2.5)
    assert s[4] == pytest.approx(-0.5)  # xz: column z = -(R/A)(m . e_z) averaged, symmetrised


# --------------------------------------------------------------------------- several walls
def corner_force(nw, Rc, Kn):
    """Force component along each wall normal at a node touching nw = 1, 2, 3
    mutually orthogonal walls at distance 0 (half ball, quarter ball, octant)."""
    half = Kn * (Rc - 3 * Rc / 8) * (2 * math.pi * Rc ** 3 / 3)
    quarter = Kn * (Rc - 3 * math.sqrt(2) * Rc / 8) * (math.pi * Rc ** 3 / 3) / math.sqrt(2)
    octant = Kn * (Rc - 3 * math.sqrt(3) * Rc / 8) * (math.pi * Rc ** 3 / 6) / math.sqrt(3)
    return {1: half, 2: half - quarter, 3: half - 2 * quarter + octant}[nw]


@pytest.mark.parametrize("nw", [1, 2, 3])
def test_corner_inclusion_exclusion_closed_form(nw):
    Rc, Vi = 1e-4, 1e-12
    normals = np.eye(3)[:nw]
    walls = np.array([list(n) + [0, 0, 0, 0, 0, 0] for n in normals])
    for overlap in (0, 1):
        m = model_for(np.zeros((1, 3)), S.Material(contact_radius=Rc, wall_overlap=overlap, **MAT), 3e-4,
                      walls=walls, vol=np.full(1, Vi))
        F = m.forces()
        expect = corner_force(nw if overlap else 1, Rc, m.Kn)
        for k in range(3):
            want = expect if k < nw else 0.0
            assert F[0, k] == pytest.approx(want, rel=1e-9, abs=1e-30)
        # each wall takes the component along its own normal
        for l in range(nw):
            assert m.react[l] @ normals[l] == pytest.approx(-expect * Vi, rel=1e-9)
        assert np.abs(F[0] * Vi + m.react.sum(0)).max() < 1e-12 * abs(expect * Vi)


def test_overlap_only_for_orthogonal_touching_walls():
    """Walls at 60 degrees keep the plain sum; a node touching one wall is
    unchanged; the correction fades out continuously as the second wall
    leaves the contact radius."""
    Rc = 1e-4
    n2 = np.array([math.cos(math.radians(60)), 0.0, math.sin(math.radians(60))])
    walls = np.array([[0, 0, 1.0, 0, 0, 0, 0, 0, 0], list(n2) + [0, 0, 0, 0, 0, 0]])
    x = np.array([[0.1 * Rc, 0.0, 0.2 * Rc]])
    F = [model_for(x, S.Material(contact_radius=Rc, wall_overlap=o, **MAT), 3e-4, walls=walls).forces().copy()
         for o in (0, 1)]
    assert np.array_equal(F[0], F[1])
    walls = np.array([[0, 0, 1.0, 0, 0, 0, 0, 0, 0], [1.0, 0, 0, 0, 0, 0, 0, 0, 0]])
    x = np.array([[2 * Rc, 0.0, 0.2 * Rc]])
    F = [model_for(x, S.Material(contact_radius=Rc, wall_overlap=o, **MAT), 3e-4, walls=walls).forces().copy()
         for o in (0, 1)]
    assert np.array_equal(F[0], F[1])
    f = []
    for dx in (Rc * (1 - 1e-7), Rc * (1 + 1e-7)):
        m = model_for(np.array([[dx, 0.0, 0.2 * Rc]]), S.Material(contact_radius=Rc, wall_overlap=1, **MAT), 3e-4,
                      walls=walls)
        f.append(m.forces()[0].copy())
    assert np.abs(f[0] - f[1]).max() < 1e-6 * np.abs(f[1]).max()


def test_friction_dissipates_over_a_sliding_collision():
    """Two unbreakable jittered blocks meet obliquely (normal approach plus a
    tangential slip) and separate again.  Without friction the energy after the
    contact equals the energy before (velocity Verlet, spring contact).  With
    friction it drops by a clear amount, and the blocks leave with less slip than
    without friction (rough contact alone changes the slip; friction opposes it).
    Momentum is conserved in both runs."""
    h = 1e-4
    rng = np.random.default_rng(6)
    a = rng.uniform(-0.02, 0.02, (4 * 4 * 3, 3)) * h + np.stack(np.meshgrid(
        np.arange(4), np.arange(4), np.arange(3), indexing="ij"), -1).reshape(-1, 3) * h
    b = a + np.array([0.0, 0.0, 2.0 * h + 0.65 * h])
    x = np.concatenate([a, b])
    grain = np.repeat(np.array([0, 1], np.int32), len(a))
    vol = np.full(len(x), h ** 3)
    v0 = np.zeros_like(x)
    v0[grain == 1] = [5.0, 0.0, -5.0]
    v0[grain == 0] = [-5.0, 0.0, 5.0]
    out = {}
    for mu in (0.0, 0.5):
        m = model_for(x, S.Material(E=72e9, rho=2440.0, G0=1e30, contact_radius=0.6 * h, mu=mu), 3 * h,
                      grain=grain, vol=vol, v0=v0.copy())
        dt = 0.2 * m.stable_dt()
        m.P.dt_f = dt
        m.init()
        e0 = m.energy()
        p0 = (vol[:, None] * m.v).sum(0)
        touched = 0
        for _ in range(400):
            m.step(dt, 1)
            touched += len(m.contact_pairs()) > 0
        assert touched > 50
        assert len(m.contact_pairs()) == 0  # the blocks have separated again
        p1 = (vol[:, None] * m.v).sum(0)
        assert np.abs(p1 - p0).max() <= 1e-12 * np.abs(vol[:, None] * v0).sum()
        slip = m.v[grain == 1, 0].mean() - m.v[grain == 0, 0].mean()
        out[mu] = (e0, m.energy(), slip)
    e0, e1, slip0 = out[0.0]
    assert abs(e1 - e0) < 1e-3 * e0
    e0f, e1f, slipf = out[0.5]
    assert e0f == pytest.approx(e0, rel=1e-12)
    assert e1f < 0.9 * e0f
    assert 0.0 < slipf < 0.5 * slip0
