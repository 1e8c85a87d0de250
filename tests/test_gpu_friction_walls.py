"""Stick-slip friction (Sec. 3.3) and the multi-wall inclusion-exclusion
(Sec. 4.1.1) of the CUDA path against the oracle: forces and wall reactions at
one state, the friction or overlap part alone, and trajectories."""
import numpy as np
import pytest

import oracle
from paper_2506_05362_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    import torch
    assert torch.cuda.is_available()
    from paper_2506_05362_gb300 import pd as _pd
    return _pd


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def lattice(nx, ny, nz, h, jitter, rng):
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    lat = np.stack([I.ravel(), J.ravel(), K.ravel()], 1).astype(np.float64) * h
    return lat + rng.uniform(-jitter, jitter, lat.shape) * h


def sliding_blocks(mu, beta_zeta=0.0):
    """Two jittered blocks of different grains pressed into each other, the lower
    one resting in the range of a wall that slides along x, random velocities."""
    from paper_2506_05362_gb300 import surrogate as SG
    h = 1e-4
    rng = np.random.default_rng(3)
    a = lattice(6, 5, 4, h, 0.05, rng)
    b = lattice(6, 5, 4, h, 0.05, rng) + np.array([0.2 * h, 0.3 * h, 3.55 * h])
    x = np.concatenate([a, b])
    grain = np.repeat(np.array([0, 1], np.int32), len(a))
    vol = np.full(len(x), h ** 3) * rng.uniform(0.7, 1.3, len(x))
    mat = S.Material(E=72e9, rho=2440, G0=135, contact_radius=0.6 * h, mu=mu)
    if beta_zeta:
        mat.beta_d = SG.damping_coefficient(mat, 3 * h, h ** 3, beta_zeta)
    zmin = x[:, 2].min()
    walls = [S.Wall((0.0, 0.0, 1.0), (0.0, 0.0, zmin - 0.5 * mat.contact_radius), (0.4, 0.0, 0.3))]
    v0 = rng.normal(0, 0.5, x.shape)
    return S.Scenario(name="sliding", x=x, vol=vol, grain=grain, v0=v0, material=mat, horizon=3 * h, h=h,
                      walls=walls, wall_area=1e-6)


@pytest.mark.parametrize("dt", [1e-8, 1e-10])  # mostly sticking; mostly slipping
@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-12)])
def test_friction_forces_same_state(pd, precision, tol, dt):
    sc = sliding_blocks(0.3)
    ctx = pd.Context.from_scenario(sc, precision=precision, lanes=8)
    ctx.step(dt, 0)  # the friction's time step
    ref = oracle.Model.from_scenario(sc)
    ref.P.dt_f = dt
    F = ctx.forces()
    ref.forces()
    assert len(ref.contact_pairs()) > 0
    assert rel_l2(F, ref.F) <= tol
    _, wf = ctx.bulk_stress([1e-6])
    assert rel_l2(wf, ref.react) <= max(tol, 1e-9)
    assert abs(ref.react[0, 0]) > 0  # the sliding wall takes a tangential reaction
    # friction alone
    sc0 = sliding_blocks(0.0)
    ctx0 = pd.Context.from_scenario(sc0, precision=precision, lanes=8)
    ref.P.mu = 0.0
    Ff_ref = ref.F.copy() - ref.forces(frozen=True).copy()
    Ff = F - ctx0.forces()
    assert np.abs(Ff_ref).max() > 1e-4 * np.abs(ref.F).max()
    assert rel_l2(Ff, Ff_ref) <= (1e-4 if precision == "mixed" else 1e-9)
    ctx.close(); ctx0.close()


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-9)])
def test_frictional_collision_trajectory(pd, precision, tol):
    """Two grains meeting obliquely (sliding past each other) with friction and
    damping: the trajectory follows the oracle."""
    from paper_2506_05362_gb300 import surrogate as SG
    sc = S.aggregate(n_grains=2, h=0.5e-3 / 4, gap_cells=0.5, seed=4)
    c = sc.x[sc.grain == 0].mean(0) - sc.x[sc.grain == 1].mean(0)
    c /= np.linalg.norm(c)
    t = np.cross(c, [0.0, 0.0, 1.0])
    t /= np.linalg.norm(t)
    sc.v0 = np.where((sc.grain == 0)[:, None], -5.0 * c + 3.0 * t, 5.0 * c - 3.0 * t)
    sc.walls = []
    sc.material.beta_d = SG.damping_coefficient(sc.material, sc.horizon, sc.h ** 3, 0.2)
    sc.material.mu = 0.5
    ctx = pd.Context.from_scenario(sc, precision=precision)
    ref = oracle.Model.from_scenario(sc)
    dt = 0.5 * ref.stable_dt()
    ref.P.dt_f = dt
    ref.init()
    touched, total = 0, 0
    while total < 20000 and touched < 60:
        ref.step(dt, 10)
        ctx.step(dt, 10)
        total += 10
        if touched or len(ref.contact_pairs()) > 0:
            touched += 10
    assert touched > 0, "grains never met"
    u, v, broken, _ = ctx.get_state()
    assert rel_l2(u, ref.u) < tol
    assert rel_l2(v, ref.v) < 10 * tol


def corner_block(overlap, mu=0.0, inward=0.0):
    """A jittered block in the corner of three orthogonal walls; boundary nodes
    sit at -0.2 .. 0.5 R_c from the walls (some slightly behind them)."""
    h = 1e-4
    rng = np.random.default_rng(11)
    x = lattice(5, 5, 5, h, 0.1, rng)
    Rc = 0.6 * h
    mat = S.Material(E=72e9, rho=2440, G0=135, contact_radius=Rc, mu=mu, wall_overlap=overlap)
    lo = x.min(0)
    walls = [S.Wall(tuple(np.eye(3)[k]), tuple(np.where(np.arange(3) == k, lo[k] - 0.15 * Rc, 0.0)),
                    tuple(inward * np.eye(3)[k])) for k in range(3)]
    v0 = rng.normal(0, 0.2, x.shape)
    return S.Scenario(name="corner", x=x, vol=np.full(len(x), h ** 3), grain=np.zeros(len(x), np.int32), v0=v0,
                      material=mat, horizon=3 * h, h=h, walls=walls, wall_area=1e-6)


# FP64: the shared-region integrals differ by quadrature error only (the oracle's
# adaptive Simpson to 1e-12 R_c^3, the library's 32-point Gauss-Legendre rule to
# ~4e-13 R_c^3), a few 1e-12 of the force
@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-10)])
def test_corner_overlap_forces(pd, precision, tol):
    """Nodes touching two or three walls: forces and reactions with the
    inclusion-exclusion terms; the terms alone against the oracle's."""
    sc = corner_block(1)
    ctx = pd.Context.from_scenario(sc, precision=precision, lanes=8)
    ref = oracle.Model.from_scenario(sc)
    rng = np.random.default_rng(2)
    u = rng.normal(0, 0.15 * sc.material.contact_radius, sc.x.shape)
    ctx.set_state(u=u)
    ref.u = u.copy()
    F = ctx.forces()
    ref.forces()
    assert rel_l2(F, ref.F) <= tol
    _, wf = ctx.bulk_stress([1e-6] * 3)
    assert rel_l2(wf, ref.react) <= max(tol, 1e-9)
    # how many nodes touch two and three walls, and one behind a wall
    p = sc.x + u
    d = p - np.array([w.point for w in sc.walls]).diagonal()
    touch = (d < sc.material.contact_radius).sum(1)
    assert (touch >= 2).sum() >= 5 and (touch == 3).sum() >= 1 and (d.min() < 0)
    sc0 = corner_block(0)
    ctx0 = pd.Context.from_scenario(sc0, precision=precision, lanes=8)
    ctx0.set_state(u=u)
    ref.P.wall_overlap = 0
    Fo_ref = ref.F.copy() - ref.forces(frozen=True).copy()
    Fo = F - ctx0.forces()
    assert np.abs(Fo_ref).max() > 1e-3 * np.abs(ref.F).max()
    assert rel_l2(Fo, Fo_ref) <= (1e-4 if precision == "mixed" else 1e-9)
    ctx.close(); ctx0.close()


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-9)])
def test_corner_compression_trajectory(pd, precision, tol):
    """The block pushed into the corner by walls moving in, with friction and
    the inclusion-exclusion terms: the trajectory and the wall impulses follow
    the oracle."""
    sc = corner_block(1, mu=0.4, inward=0.5)
    ctx = pd.Context.from_scenario(sc, precision=precision)
    ref = oracle.Model.from_scenario(sc)
    dt = 0.5 * ref.stable_dt()
    ref.P.dt_f = dt
    ref.init()
    ctx.step(dt, 0)
    ctx.bulk_stress_mean([1e-6] * 3)  # reset the impulses after the set-up evaluations
    ref.impulse[:] = 0
    ref.impulse_span = 0.0
    for _ in range(6):
        ref.step(dt, 25)
        ctx.step(dt, 25)
    u, v, broken, _ = ctx.get_state()
    assert rel_l2(u, ref.u) < tol
    assert rel_l2(v, ref.v) < 10 * tol
    _, wf, span = ctx.bulk_stress_mean([1e-6] * 3)
    _, wf_ref, span_ref = ref.bulk_stress_mean([1e-6] * 3)
    assert span == pytest.approx(span_ref, rel=1e-12)
    assert rel_l2(wf, wf_ref) < 10 * tol
