"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2506_05362_gb300 import scenarios as S

pytestmark = pytest.mark.gpu

MIXED_FORCE_TOL = 1e-5      # rel-L2 of F per evaluation, mixed path
FP64_FORCE_TOL = 1e-12      # rel-L2 of F, all-FP64 path
BAND = 1e-6                 # bonds with |s - s0| < BAND * s0 may decide either way


@pytest.fixture(scope="module")
def pd():
    import torch
    assert torch.cuda.is_available()
    from paper_2506_05362_gb300 import pd as _pd
    _pd.lib()
    return _pd


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def stretches(x, u, rp, col):
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    xi = x[col] - x[rows]
    y = xi + (u[col] - u[rows])
    L = np.linalg.norm(xi, axis=1)
    return (np.linalg.norm(y, axis=1) - L) / L


def small_kalthoff():
    return S.kalthoff(length=0.02, height=0.04, thickness=0.005, notch_len=0.01, notch_width=1.5e-3,
                      notch_gap=0.012, steps=40)


def small_hollow():
    return S.hollow(outer_cells=14, inner_cells=9, steps=40)


# kernels of the mixed path: per-slot gathers from global memory, shared-memory
# tiles, each bond once (two passes)
KERNEL = {"global": dict(tiles=-1, pairs=-1), "tiled": dict(tiles=1, pairs=-1), "pairs": dict(tiles=-1, pairs=1),
          "fp64": {}}

SCENARIOS = {
    "sphere": lambda: S.sphere(),
    "kalthoff_small": small_kalthoff,
    "hollow_small": small_hollow,
    "aggregate_small": lambda: S.aggregate(n_grains=4, h=0.5e-3 / 5, gap_cells=0.3, seed=2),
    "block_ragged": lambda: S.small_block(nx=7, ny=5, nz=3, jitter=0.2),
}


# --------------------------------------------------------------------------- lists
@pytest.mark.parametrize("name", list(SCENARIOS))
def test_bond_lists_bitexact(pd, name):
    sc = SCENARIOS[name]()
    ctx = pd.Context.from_scenario(sc, lanes=8)
    rp, col = ctx.bonds()
    kinds, params = S.filters_array(sc.filters)
    orp, ocol = oracle.bonds(sc.x, sc.grain, sc.horizon, kinds, params)
    assert np.array_equal(rp, orp)
    assert np.array_equal(col, ocol)
    ctx.close()


@pytest.mark.parametrize("name", ["kalthoff", "hollow"])
def test_bond_lists_full_size(pd, name):
    """Full-size plate (178,200 nodes, delta = 4h) and hollow sphere (343,846 nodes):
    whole CSR against the oracle's cell-list build (itself pinned to brute force)."""
    sc = S.BY_NAME[name]()
    ctx = pd.Context.from_scenario(sc, lanes=16, contact=False)
    rp, col = ctx.bonds()
    kinds, params = S.filters_array(sc.filters)
    orp, ocol = oracle.bonds(sc.x, sc.grain, sc.horizon, kinds, params, brute=False)
    assert np.array_equal(rp, orp)
    assert np.array_equal(col, ocol)
    # a few rows by brute force over all nodes
    for i in [0, sc.n // 3, sc.n - 1]:
        assert np.array_equal(col[rp[i]:rp[i + 1]], oracle.bond_row(sc.x, sc.grain, sc.horizon, i, kinds, params))
    ctx.close()


# --------------------------------------------------------------------------- forces
def perturbed_state(sc, rp, col, seed, strain=0.9, noise=0.5):
    """Affine stretch of about `strain` s0 plus noise, so that some bonds break."""
    m = sc.material
    K, c, s0, Kn = oracle.constants(m.E, m.G0, sc.horizon, m.contact_factor, m.constants, m.micromodulus)
    rng = np.random.default_rng(seed)
    A = np.diag([strain * s0, -0.3 * strain * s0, 0.5 * strain * s0]) + rng.normal(0, 0.2 * s0, (3, 3))
    u = (sc.x - sc.x.mean(0)) @ A.T + rng.normal(0, noise * s0 * sc.h, sc.x.shape)
    return u, s0


@pytest.mark.parametrize("precision,tol,kernel", [("mixed", MIXED_FORCE_TOL, "tiled"),
                                                 ("mixed", MIXED_FORCE_TOL, "global"),
                                                 ("mixed", MIXED_FORCE_TOL, "pairs"),
                                                 ("fp64", FP64_FORCE_TOL, "fp64")])
@pytest.mark.parametrize("name", ["sphere", "kalthoff_small", "aggregate_small", "block_ragged"])
@pytest.mark.parametrize("lanes", [4, 32])
def test_forces_same_state(pd, name, precision, tol, kernel, lanes):
    sc = SCENARIOS[name]()
    ctx = pd.Context.from_scenario(sc, precision=precision, lanes=lanes, **KERNEL[kernel])
    assert ctx.tuning()[1] == {"global": 0, "tiled": 1, "pairs": 2, "fp64": 0}[kernel] or kernel == "tiled"
    ref = oracle.Model.from_scenario(sc)
    u, s0 = perturbed_state(sc, ref.rowptr, ref.col, seed=1)
    ctx.set_state(u=u)
    F = ctx.forces()
    _, _, broken, _ = ctx.get_state()
    ref.u = u.copy()
    ref.forces()
    s = stretches(sc.x, u, ref.rowptr, ref.col)
    diff = broken.astype(bool) != ref.broken.astype(bool)
    assert ref.broken.sum() > 0, "test state should break some bonds"
    assert np.all(np.abs(s[diff] - s0) < BAND * s0), "broken sets differ outside the tolerance band"
    # evaluate the oracle with the GPU's decisions on band bonds, then compare F
    ref.broken[:] = broken
    Fo = ref.forces(frozen=True).copy()
    assert rel_l2(F, Fo) <= tol
    ctx.close()


@pytest.mark.parametrize("precision,tol", [("mixed", MIXED_FORCE_TOL), ("fp64", FP64_FORCE_TOL)])
@pytest.mark.parametrize("name", ["sphere", "kalthoff_small"])
@pytest.mark.parametrize("break_mode,constants", [(1, 0), (0, 1), (1, 1)])
def test_forces_breaking_modes(pd, name, precision, tol, break_mode, constants):
    """The |s| > s0 criterion (break_mode 1, the sentence before the table of
    Sec. 3.1.1) and the table's printed constants (constants 1): forces and broken
    sets at a perturbed state.  Under break_mode 1 the state is compressive, so
    that bonds break in compression, which the default criterion never does."""
    sc = SCENARIOS[name]()
    sc.material.break_mode = break_mode
    sc.material.constants = constants
    ctx = pd.Context.from_scenario(sc, precision=precision, lanes=8)
    ref = oracle.Model.from_scenario(sc)
    assert ctx.stable_dt() == pytest.approx(ref.stable_dt(), rel=1e-12)
    u, s0 = perturbed_state(sc, ref.rowptr, ref.col, seed=5, strain=1.1)
    assert s0 == pytest.approx(ref.s0, rel=1e-15)
    if break_mode:
        u = -u
    ctx.set_state(u=u)
    F = ctx.forces()
    _, _, broken, _ = ctx.get_state()
    ref.u = u.copy()
    ref.forces()
    s = stretches(sc.x, u, ref.rowptr, ref.col)
    b = ref.broken.astype(bool)
    assert b.sum() > 0
    if break_mode:
        assert (b & (s < -s0)).sum() > 0, "no bond broke in compression"
    else:
        assert np.all(s[b] > s0 * (1 - BAND))
    diff = broken.astype(bool) != b
    assert np.all(np.abs(np.abs(s[diff]) - s0) < BAND * s0)
    ref.broken[:] = broken
    Fo = ref.forces(frozen=True).copy()
    assert rel_l2(F, Fo) <= tol
    ctx.close()


def test_forces_full_size_sampled(pd):
    """Full-size notched plate in the launch configuration the benchmark times:
    forces at a perturbed state against the oracle (whole field; the oracle
    evaluates 45 M bonds in a few seconds)."""
    sc = S.kalthoff()
    ctx = pd.Context.from_scenario(sc)
    ref = oracle.Model.from_scenario(sc)
    u, s0 = perturbed_state(sc, ref.rowptr, ref.col, seed=3, strain=0.5, noise=0.2)
    ctx.set_state(u=u)
    F = ctx.forces()
    _, _, broken, _ = ctx.get_state()
    ref.u = u.copy()
    ref.forces()
    s = stretches(sc.x, u, ref.rowptr, ref.col)
    diff = broken.astype(bool) != ref.broken.astype(bool)
    assert ref.broken.sum() > 0
    assert np.all(np.abs(s[diff] - s0) < BAND * s0)
    ref.broken[:] = broken
    Fo = ref.forces(frozen=True)
    assert rel_l2(F, Fo) <= MIXED_FORCE_TOL
    ctx.close()


# --------------------------------------------------------------------------- trajectories
# FP64 tolerance: both sides round every operation to 53 bits but sum the bond
# forces in different orders; near equilibrium the net force is a small residual
# of terms ~1e4-1e5 times larger, and 200 steps accumulate it: ~1e-10 observed.
@pytest.mark.parametrize("precision,tol,kernel", [("mixed", 1e-5, "tiled"), ("mixed", 1e-5, "global"),
                                                 ("mixed", 1e-5, "pairs"), ("fp64", 1e-9, "fp64")])
@pytest.mark.parametrize("break_mode,constants", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_sphere_trajectory_200_steps(pd, precision, tol, kernel, break_mode, constants):
    """Glass sphere between plates, 200 steps at 0.8 dt_crit: u, v, wall force;
    under both breaking criteria and both sets of constants (Sec. 3.1.1)."""
    sc = S.sphere()
    sc.material.break_mode = break_mode
    sc.material.constants = constants
    ctx = pd.Context.from_scenario(sc, precision=precision, **KERNEL[kernel])
    ref = oracle.Model.from_scenario(sc)
    dtc = ref.stable_dt()
    assert ctx.stable_dt() == pytest.approx(dtc, rel=1e-12)
    dt = 0.8 * dtc
    ref.init()
    ctx.step(dt, sc.steps)
    ref.step(dt, sc.steps)
    u, v, broken, t = ctx.get_state()
    assert rel_l2(u, ref.u) <= tol
    # velocities carry the same rounding relative to a smaller, noisier field
    # (FP64: 1.1e-8 observed with the table's stiffer constants)
    assert rel_l2(v, ref.v) <= (10 * tol if precision == "mixed" else 5e-8)
    assert t == pytest.approx(ref.t, rel=1e-14)
    walls = ctx.get_walls()
    assert np.allclose(walls, ref.wall_pos, rtol=0, atol=1e-18)
    sig, wf = ctx.bulk_stress([sc.wall_area] * 2)
    assert rel_l2(wf, ref.react) <= max(tol, 1e-9)
    assert np.allclose(sig, ref.bulk_stress([sc.wall_area] * 2), rtol=max(tol, 1e-9))
    # wall forces averaged over the 200 steps (impulse / time)
    sig_m, wf_m, span = ctx.bulk_stress_mean([sc.wall_area] * 2)
    osig_m, owf_m, ospan = ref.bulk_stress_mean([sc.wall_area] * 2)
    assert span == pytest.approx(ospan, rel=1e-14)
    assert np.abs(owf_m).max() > 0
    assert rel_l2(wf_m, owf_m) <= max(tol, 1e-9)
    assert np.allclose(sig_m, osig_m, rtol=max(tol, 1e-9))
    # the call resets the accumulator
    assert ctx.bulk_stress_mean([sc.wall_area] * 2)[2] == 0.0
    ctx.close()


@pytest.mark.parametrize("kernel", ["tiled", "pairs"])
@pytest.mark.parametrize("break_mode,sign", [(0, 1.0), (1, -1.0)])
def test_breaking_trajectory_block(pd, break_mode, sign, kernel):
    """A block torn apart (sign +1) or crushed (sign -1, with the |s| > s0
    criterion, so that bonds break in compression) by opposing initial velocities:
    damage appears, and the step-by-step comparison from a shared state holds
    through the damage."""
    sc = S.small_block(nx=10, ny=6, nz=5, jitter=0.05)
    sc.material.break_mode = break_mode
    sc.v0 = np.zeros_like(sc.x)
    sc.v0[:, 0] = sign * np.where(sc.x[:, 0] > sc.x[:, 0].mean(), 40.0, -40.0)
    ctx = pd.Context.from_scenario(sc, lanes=16, **KERNEL[kernel])
    ref = oracle.Model.from_scenario(sc)
    dt = 0.5 * ref.stable_dt()
    ref.init()
    for _ in range(30):
        ctx.step(dt, 1)
        ref.step(dt, 1)
        u, v, broken, _ = ctx.get_state()
        assert rel_l2(u, ref.u) < 1e-5
        # resynchronise the oracle on the GPU's band decisions (chaos after damage)
        s = stretches(sc.x, u, ref.rowptr, ref.col)
        diff = broken.astype(bool) != ref.broken.astype(bool)
        assert np.all(np.abs(np.abs(s[diff]) - ref.s0) < 1e-3 * ref.s0)
        ref.broken[:] = broken
    assert broken.sum() > 0
    phi = ctx.damage()
    assert np.allclose(phi, ref.damage(), atol=0)
    ctx.close()


@pytest.mark.parametrize("kernel", ["auto", "pairs"])
def test_kalthoff_window(pd, kernel):
    """Small notched plate: impact window of 40 steps, mixed path vs oracle."""
    sc = small_kalthoff()
    ctx = pd.Context.from_scenario(sc, **({} if kernel == "auto" else KERNEL[kernel]))
    ref = oracle.Model.from_scenario(sc)
    dt = 0.8 * ref.stable_dt()
    ref.init()
    ctx.step(dt, sc.steps)
    ref.step(dt, sc.steps)
    u, v, broken, _ = ctx.get_state()
    assert rel_l2(u, ref.u) < 1e-5
    assert rel_l2(v, ref.v) < 1e-5
    ctx.close()


# --------------------------------------------------------------------------- contact
def symmetric_pattern(rp, col, frac, seed):
    """Broken flags (canonical order) for a random set of undirected bonds."""
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    lo, hi = np.minimum(rows, col), np.maximum(rows, col)
    key = lo.astype(np.int64) * (len(rp) + 1) + hi
    rng = np.random.default_rng(seed)
    uniq = np.unique(key)
    pick = set(uniq[rng.random(len(uniq)) < frac].tolist())
    return np.array([k in pick for k in key.tolist()], np.uint8)


def test_contact_pairs_bitexact(pd):
    """Same state on both sides (the oracle takes the GPU's state as returned):
    fragments of broken bonds pushed together, and grains in contact."""
    sc = S.aggregate(n_grains=3, h=0.5e-3 / 4, gap_cells=0.2, seed=3)
    ctx = pd.Context.from_scenario(sc, lanes=8)
    ref = oracle.Model.from_scenario(sc)
    rng = np.random.default_rng(1)
    u = rng.uniform(-0.5, 0.5, (sc.n, 3)) * sc.h
    ctx.set_state(u=u, broken=symmetric_pattern(ref.rowptr, ref.col, 0.3, 2))
    ug, _, broken, _ = ctx.get_state()
    ref.u = ug.copy()
    ref.broken[:] = broken
    pairs = ctx.contacts()
    opairs = ref.contact_pairs()
    assert len(opairs) > 0
    assert np.array_equal(pairs, opairs)
    F = ctx.forces()
    Fo = ref.forces(frozen=True)
    assert rel_l2(F, Fo) < MIXED_FORCE_TOL


@pytest.mark.parametrize("axis,kernel", [(0, "global"), (1, "tiled"), (2, "pairs")])
def test_grain_collision_dynamics(pd, axis, kernel):
    """Two grains flying into each other along ``axis``: contact forces act across
    grains and the trajectory follows the oracle (which rebuilds contacts every
    step).  Each axis in turn, so that the skin bookkeeping sees every velocity
    component."""
    sc = S.aggregate(n_grains=2, h=0.5e-3 / 4, gap_cells=0.5, seed=4)
    sc.x = np.ascontiguousarray(np.roll(sc.x, axis, axis=1))
    c = sc.x[sc.grain == 0].mean(0) - sc.x[sc.grain == 1].mean(0)
    c /= np.linalg.norm(c)
    sc.v0 = np.where((sc.grain == 0)[:, None], -5.0 * c, 5.0 * c)
    sc.walls = []
    ctx = pd.Context.from_scenario(sc, lanes=8, **KERNEL[kernel])
    ref = oracle.Model.from_scenario(sc)
    dt = 0.5 * ref.stable_dt()
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
    assert rel_l2(u, ref.u) < 1e-5
    assert rel_l2(v, ref.v) < 1e-4


@pytest.mark.parametrize("precision,kernel", [("mixed", "global"), ("mixed", "pairs"), ("fp64", "fp64")])
def test_contact_forces_do_not_depend_on_the_list_history(pd, precision, kernel):
    """Contact terms are added in ascending partner order over the touching pairs
    alone, so the skin superset a rebuild happened to produce does not enter the
    result: two grains colliding, once with the automatic rebuild period and once
    rebuilt every step, follow bit-identical trajectories."""
    sc = S.aggregate(n_grains=2, h=0.5e-3 / 4, gap_cells=0.5, seed=4)
    c = sc.x[sc.grain == 0].mean(0) - sc.x[sc.grain == 1].mean(0)
    c /= np.linalg.norm(c)
    sc.v0 = np.where((sc.grain == 0)[:, None], -5.0 * c, 5.0 * c)
    sc.walls = []
    a = pd.Context.from_scenario(sc, precision=precision, lanes=8, **KERNEL[kernel])
    b = pd.Context.from_scenario(sc, precision=precision, lanes=8, contact_every=1, **KERNEL[kernel])
    dt = 0.5 * a.stable_dt()
    touched = 0
    for _ in range(400):
        a.step(dt, 25)
        b.step(dt, 25)
        if len(a.contacts()):
            touched += 1
        if touched > 4:
            break
    assert touched > 0, "grains never met"
    assert a.step_counters()[1] < b.step_counters()[1]  # far fewer rebuilds
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    a.close(); b.close()


# --------------------------------------------------------------------------- invariants
@pytest.mark.parametrize("kernel", ["global", "pairs"])
def test_one_step_calls_carry_the_contact_list(pd, kernel):
    """Calls of one step reuse the contact list while the device's displacement
    bound says it holds: two grains colliding in 1-step calls rebuild far less
    often than once per step, and follow bit for bit a run that rebuilds every
    step; a state sent back unchanged between the calls changes nothing."""
    sc = S.aggregate(n_grains=2, h=0.5e-3 / 4, gap_cells=0.5, seed=4)
    c = sc.x[sc.grain == 0].mean(0) - sc.x[sc.grain == 1].mean(0)
    c /= np.linalg.norm(c)
    sc.v0 = np.where((sc.grain == 0)[:, None], -5.0 * c, 5.0 * c)
    sc.walls = []
    a = pd.Context.from_scenario(sc, lanes=8, persistent=-1, **KERNEL[kernel])
    b = pd.Context.from_scenario(sc, lanes=8, contact_every=1, persistent=-1, **KERNEL[kernel])
    dt = 0.5 * a.stable_dt()
    touched = 0
    for it in range(4000):
        a.step(dt, 1)
        if it % 7 == 3:  # a round trip of the state in between
            up, vp, bits, tp = pd.pd_get_state_packed(a.h, a.n, a.B)
            pd.pd_set_state_packed(a.h, up, vp, bits, tp)
        if it % 25 == 24:
            b.step(dt, 25)
            if len(b.contacts()):
                touched += 1
            if touched > 4:
                break
    assert touched > 0, "grains never met"
    steps_a, rebuilds_a, _ = a.step_counters()
    steps_b, rebuilds_b, _ = b.step_counters()
    assert steps_a == steps_b
    assert rebuilds_a < steps_a / 2 and rebuilds_b >= steps_b
    sa, sb = a.get_state(), b.get_state()
    for x, y in zip(sa[:3], sb[:3]):  # u, v, bond memory
        assert np.array_equal(x, y)
    assert sa[3] == pytest.approx(sb[3], rel=1e-12)  # t: sums of dt over calls of other lengths
    a.close(); b.close()


def test_rigid_motion_zero_force_gpu(pd):
    sc = S.small_block(nx=8, ny=6, nz=5, jitter=0.03)
    ctx = pd.Context.from_scenario(sc, contact=False)
    th = 0.4
    R = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    u = sc.x @ R.T - sc.x + np.array([1e-3, 2e-3, -1e-3])
    ctx.set_state(u=u)
    F = ctx.forces()
    _, _, broken, _ = ctx.get_state()
    assert broken.sum() == 0
    # scale: net force of a surface node under a uniform stretch of s0 / 2
    ref = oracle.Model.from_scenario(sc)
    ref.u = 0.5 * ref.s0 * (sc.x - sc.x.mean(0))
    scale = np.abs(ref.forces()).max()
    assert scale > 0
    assert np.abs(F).max() < 1e-3 * scale
    ctx.close()


def test_momentum_gpu(pd):
    sc = S.aggregate(n_grains=3, h=0.5e-3 / 4, gap_cells=0.2, seed=5)
    sc.walls = []
    ctx = pd.Context.from_scenario(sc)
    u = np.random.default_rng(2).uniform(-0.3, 0.3, sc.x.shape) * sc.h
    ctx.set_state(u=u)
    F = ctx.forces()
    FV = F * sc.vol[:, None]
    assert np.abs(FV.sum(0)).max() < 1e-6 * np.abs(FV).sum()


@pytest.mark.parametrize("kernel", ["tiled", "pairs"])
def test_determinism_and_checkpoint(pd, kernel):
    sc = S.sphere()
    a = pd.Context.from_scenario(sc, lanes=16, **KERNEL[kernel])
    b = pd.Context.from_scenario(sc, lanes=16, **KERNEL[kernel])
    dt = 0.8 * a.stable_dt()
    a.step(dt, 100)
    b.step(dt, 50)
    st = b.get_state()
    walls = b.get_walls()
    c = pd.Context.from_scenario(sc, lanes=16, **KERNEL[kernel])
    c.set_walls(np.concatenate([S.walls_array(sc.walls)[:, :3], walls, S.walls_array(sc.walls)[:, 6:]], 1))
    c.set_state(u=st[0], v=st[1], broken=st[2], t=st[3])
    c.step(dt, 50)
    b.step(dt, 50)
    ua, va, ba, ta = a.get_state()
    for other in (b, c):
        uo, vo, bo, to = other.get_state()
        assert np.array_equal(ua, uo) and np.array_equal(va, vo) and np.array_equal(ba, bo)
        assert ta == to


def test_packed_state_equals_byte_state(pd):
    """The packed bond memory (pd_get/set_state_packed) holds the same state as
    the byte form: identical flags after breaking, and a context restored from
    either form steps to the same bits."""
    sc = S.small_block(nx=9, ny=7, nz=5, jitter=0.05)
    ref = oracle.Model.from_scenario(sc)
    u, _ = perturbed_state(sc, ref.rowptr, ref.col, seed=9, strain=1.2)
    a = pd.Context.from_scenario(sc, lanes=8)
    a.set_state(u=u)
    ua, va, ba, ta = a.get_state()
    assert 0 < ba.sum() < len(ba)
    up, vp, bits, tp = pd.pd_get_state_packed(a.h, a.n, a.B)
    assert np.array_equal(bits, pd.pack_broken(ba))
    assert np.array_equal(up, ua) and np.array_equal(vp, va) and tp == ta
    # restore a fresh context from each form, then step both
    b = pd.Context.from_scenario(sc, lanes=8)
    c = pd.Context.from_scenario(sc, lanes=8)
    b.set_state(u=ua, v=va, broken=ba, t=ta)
    pd.pd_set_state_packed(c.h, ua, va, bits, ta)
    dt = 0.5 * a.stable_dt()
    b.step(dt, 20)
    c.step(dt, 20)
    sb, sc_ = b.get_state(), c.get_state()
    for x, y in zip(sb[:3], sc_[:3]):
        assert np.array_equal(x, y)
    # bits past B are ignored on input (a fresh context restored at the first state,
    # where re-evaluating the forces breaks nothing new)
    assert a.B % 32
    bits2 = bits.copy()
    bits2[-1] |= np.uint32(0xffffffff) << np.uint32(a.B % 32)
    d = pd.Context.from_scenario(sc, lanes=8)
    pd.pd_set_state_packed(d.h, ua, va, bits2, ta)
    assert np.array_equal(d.get_state()[2], ba)


def test_set_state_of_the_current_state_is_skipped(pd):
    """A state sent back unchanged (the byte form, then the packed form) is
    recognised on the device: nothing is applied, the force evaluation is
    skipped, and the run continues bit for bit as one that made no round trip.
    A state that differs in one component is applied."""
    sc = S.sphere()
    a = pd.Context.from_scenario(sc, lanes=16)
    b = pd.Context.from_scenario(sc, lanes=16)
    dt = 0.8 * a.stable_dt()
    a.step(dt, 50)
    b.step(dt, 50)
    u, v, broken, t = a.get_state()
    a.set_state(u=u, v=v, broken=broken, t=t)
    up, vp, bits, tp = pd.pd_get_state_packed(a.h, a.n, a.B)
    pd.pd_set_state_packed(a.h, up, vp, bits, tp)
    assert a.state_counters() == (0, 2)
    a.step(dt, 50)
    b.step(dt, 50)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    sa, wa = a.bulk_stress([sc.wall_area] * 2)
    sb, wb = b.bulk_stress([sc.wall_area] * 2)
    assert np.array_equal(wa, wb)
    u2 = a.get_state()[0].copy()
    u2[sc.n // 2, 1] *= 1.0 + 1e-9  # above the resolution of the double-float state
    a.set_state(u=u2)
    assert a.state_counters() == (1, 2)
    # held as a double-float pair: equal to about 2^-48 relative
    assert np.allclose(a.get_state()[0], u2, rtol=2.0 ** -46, atol=0)
    a.close(); b.close()


@pytest.mark.parametrize("name", ["sphere", "kalthoff_small", "aggregate_small"])
@pytest.mark.parametrize("kernel", ["global", "tiled", "pairs"])
def test_checkpoint_restart_is_exact(pd, name, kernel):
    """A fresh context given a state read out at step k (u, v, bond memory, time
    and wall points) goes on bit for bit as the run it was read from: the live
    double-float pairs lie on the FP64 grid, so the doubles read out are the
    state itself, not a rounding of it.  Sent back to the running context, the
    same state is recognised as unchanged."""
    sc = SCENARIOS[name]()
    kw = dict(lanes=8, **KERNEL[kernel])
    a = pd.Context.from_scenario(sc, **kw)
    dt = 0.8 * a.stable_dt()
    a.step(dt, 37)
    u, v, broken, t = a.get_state()
    w = a.get_walls() if sc.walls else None
    b = pd.Context.from_scenario(sc, **kw)
    if sc.walls:
        wb = S.walls_array(sc.walls)
        wb[:, 3:6] = w
        b.set_walls(wb)
    b.set_state(u=u, v=v, broken=broken, t=t)
    a.set_state(u=u, v=v, broken=broken, t=t)
    assert a.state_counters() == (0, 1)
    a.step(dt, 41)
    b.step(dt, 41)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    if sc.walls:
        assert np.array_equal(a.get_walls(), b.get_walls())
    a.close(); b.close()


def test_damage_and_stable_dt_match(pd):
    sc = S.small_block(nx=9, ny=7, nz=5, jitter=0.05)
    ctx = pd.Context.from_scenario(sc, contact=False)
    ref = oracle.Model.from_scenario(sc)
    u, s0 = perturbed_state(sc, ref.rowptr, ref.col, seed=9, strain=1.2)
    ctx.set_state(u=u)
    ref.u = u.copy()
    ref.forces()
    _, _, broken, _ = ctx.get_state()
    ref.broken[:] = broken
    assert np.array_equal(ctx.damage(), ref.damage())
    assert ctx.stable_dt() == pytest.approx(ref.stable_dt(), rel=1e-12)


# --------------------------------------------------------------------------- errors
def test_error_paths(pd):
    sc = S.small_block()
    with pytest.raises(pd.PDError) as e:
        pd.Context(sc.x, -sc.vol, sc.grain, sc.material)
    ctx = pd.Context(sc.x, sc.vol, sc.grain, sc.material)
    with pytest.raises(pd.PDError) as e:
        ctx.step(1e-9, 1)
    assert e.value.status == pd.PD_ESTATE
    ctx.build_bonds(sc.horizon)
    with pytest.raises(pd.PDError) as e:
        ctx.step(-1.0, 1)
    assert e.value.status == pd.PD_EINVAL
    with pytest.raises(pd.PDError) as e:
        ctx.build_bonds(sc.horizon, [(7, [0] * 12)])
    assert e.value.status == pd.PD_EINVAL
    with pytest.raises(pd.PDError) as e:
        ctx.set_walls(np.array([[0, 0, 2.0, 0, 0, 0, 0, 0, 0]]))
    assert e.value.status == pd.PD_EINVAL
    with pytest.raises(pd.PDError) as e:
        ctx.set_state(u=np.full((sc.n, 3), np.nan))
    assert e.value.status == pd.PD_EINVAL
    # one non-finite entry of v rejects the call, and the (finite) u is not applied either
    before = ctx.get_state()[0]
    v_bad = np.zeros((sc.n, 3))
    v_bad[sc.n // 2, 1] = np.inf
    with pytest.raises(pd.PDError) as e:
        ctx.set_state(u=before + 1e-7, v=v_bad)
    assert e.value.status == pd.PD_EINVAL
    assert np.array_equal(ctx.get_state()[0], before)
    # a wall driven through the body within one step puts nodes a whole contact
    # radius behind it: the device flags it, the call restores the state of its
    # start and latches the error until pd_set_state
    ctx = pd.Context(sc.x, sc.vol, sc.grain, sc.material)
    ctx.build_bonds(sc.horizon)
    u0 = np.random.default_rng(0).normal(0, 1e-6, sc.x.shape)
    ctx.set_state(u=u0)
    u_before = ctx.get_state()[0]
    dt = 0.5 * ctx.stable_dt()
    top = sc.x[:, 2].max() + sc.material.contact_radius
    ctx.set_walls(np.array([[0, 0, -1.0, 0, 0, top, 0, 0, -1e4 * sc.material.contact_radius / dt]]))
    with pytest.raises(pd.PDError) as e:
        ctx.step(dt, 5)
    assert e.value.status == pd.PD_EWALL
    u, _, _, _ = ctx.get_state()
    assert np.array_equal(u, u_before)
    assert np.allclose(ctx.get_walls(), [[0, 0, top]])
    with pytest.raises(pd.PDError) as e:
        ctx.step(dt, 1)
    assert e.value.status == pd.PD_ESTATE
    ctx.set_walls(np.array([[0, 0, -1.0, 0, 0, top, 0, 0, 0.0]]))
    ctx.set_state(u=u0)
    ctx.step(dt, 2)


# --------------------------------------------------------------------------- damping (Sec. 3.3)
def damped_blocks(beta_zeta=0.4):
    """Two jittered blocks of different grains pressed into each other, the lower
    one resting in a wall's contact range, with random velocities."""
    from paper_2506_05362_gb300 import surrogate as SG
    h = 1e-4
    rng = np.random.default_rng(3)
    I, J, K = np.meshgrid(np.arange(6), np.arange(5), np.arange(4), indexing="ij")
    lat = np.stack([I.ravel(), J.ravel(), K.ravel()], 1).astype(np.float64) * h
    a = lat + rng.uniform(-0.05, 0.05, lat.shape) * h
    b = lat + rng.uniform(-0.05, 0.05, lat.shape) * h + np.array([0.2 * h, 0.3 * h, 3.55 * h])
    x = np.concatenate([a, b])
    grain = np.repeat(np.array([0, 1], np.int32), len(a))
    vol = np.full(len(x), h ** 3)
    mat = S.Material(E=72e9, rho=2440, G0=135, contact_radius=0.6 * h)
    mat.beta_d = SG.damping_coefficient(mat, 3 * h, h ** 3, beta_zeta)
    zmin = x[:, 2].min()
    walls = [S.Wall((0.0, 0.0, 1.0), (0.0, 0.0, zmin - 0.5 * mat.contact_radius), (0.0, 0.0, 0.3))]
    v0 = rng.normal(0, 0.5, x.shape)
    return S.Scenario(name="damped", x=x, vol=vol, grain=grain, v0=v0, material=mat, horizon=3 * h, h=h,
                      walls=walls, wall_area=1e-6)


@pytest.mark.parametrize("precision,tol", [("mixed", MIXED_FORCE_TOL), ("fp64", FP64_FORCE_TOL)])
def test_damping_forces_same_state(pd, precision, tol):
    """Pair and wall damping at one state (current velocities) against the oracle;
    the damping term alone is checked too, so it cannot hide under the springs."""
    sc = damped_blocks()
    ctx = pd.Context.from_scenario(sc, precision=precision, lanes=8)
    ref = oracle.Model.from_scenario(sc)
    F = ctx.forces()
    ref.forces()
    assert len(ref.contact_pairs()) > 0
    assert rel_l2(F, ref.F) <= tol
    sig, wf = ctx.bulk_stress([1e-6])
    assert rel_l2(wf, ref.react) <= max(tol, 1e-9)
    # damping alone: the same state without damping
    sc0 = damped_blocks()
    sc0.material.beta_d = 0.0
    ctx0 = pd.Context.from_scenario(sc0, precision=precision, lanes=8)
    ref.P.beta_d = 0.0
    Fd_ref = ref.F.copy() - ref.forces(frozen=True).copy()
    Fd = F - ctx0.forces()
    assert np.abs(Fd_ref).max() > 1e-3 * np.abs(ref.F).max()
    assert rel_l2(Fd, Fd_ref) <= (1e-4 if precision == "mixed" else 1e-9)
    ctx.close(); ctx0.close()


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-9)])
def test_damped_collision_trajectory(pd, precision, tol):
    """Two grains colliding with pair damping (zeta = 0.3) and a damped wall: the
    trajectory follows the oracle, and the collision dissipates energy."""
    from paper_2506_05362_gb300 import surrogate as SG
    sc = S.aggregate(n_grains=2, h=0.5e-3 / 4, gap_cells=0.5, seed=4)
    c = sc.x[sc.grain == 0].mean(0) - sc.x[sc.grain == 1].mean(0)
    c /= np.linalg.norm(c)
    sc.v0 = np.where((sc.grain == 0)[:, None], -5.0 * c, 5.0 * c)
    sc.walls = []
    sc.material.beta_d = SG.damping_coefficient(sc.material, sc.horizon, sc.h ** 3, 0.3)
    ctx = pd.Context.from_scenario(sc, precision=precision)
    ref = oracle.Model.from_scenario(sc)
    dt = 0.5 * ref.stable_dt()
    ref.init()
    ke0 = 0.5 * sc.material.rho * (sc.vol[:, None] * ref.v ** 2).sum()
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
    ke1 = 0.5 * sc.material.rho * (sc.vol[:, None] * ref.v ** 2).sum()
    assert ke1 < ke0


# --------------------------------------------------------------------------- conic micromodulus
@pytest.mark.parametrize("precision,tol", [("mixed", MIXED_FORCE_TOL), ("fp64", FP64_FORCE_TOL)])
@pytest.mark.parametrize("name", ["sphere", "kalthoff_small", "aggregate_small"])
def test_conic_micromodulus_forces_and_dt(pd, name, precision, tol):
    """Conic micromodulus c (delta - |xi|): forces at a perturbed state (with
    breaking) and the critical step against the oracle."""
    sc = SCENARIOS[name]()
    sc.material.micromodulus = 1
    ctx = pd.Context.from_scenario(sc, precision=precision, lanes=8)
    ref = oracle.Model.from_scenario(sc)
    assert ctx.stable_dt() == pytest.approx(ref.stable_dt(), rel=1e-12)
    u, s0 = perturbed_state(sc, ref.rowptr, ref.col, seed=4)
    ctx.set_state(u=u)
    F = ctx.forces()
    _, _, broken, _ = ctx.get_state()
    ref.u = u.copy()
    ref.forces()
    s = stretches(sc.x, u, ref.rowptr, ref.col)
    diff = broken.astype(bool) != ref.broken.astype(bool)
    assert ref.broken.sum() > 0
    assert np.all(np.abs(s[diff] - s0) < BAND * s0)
    ref.broken[:] = broken
    Fo = ref.forces(frozen=True).copy()
    assert rel_l2(F, Fo) <= tol
    ctx.close()


# --------------------------------------------------------------------------- self-contact (PD-repulsive branch)
def self_contact_block():
    """A jittered block of one grain plus one extra node 0.4 h from an interior
    node, i.e. inside the contact radius R_c = 0.6 h of a node of its own grain:
    once their bond is broken, the pair takes the PD-repulsive self-contact law
    c (|d| - |xi|)/|xi| (Sec. 5), which no lattice reaches (nodes start >= 0.98 h
    apart)."""
    sc = S.small_block(nx=6, ny=5, nz=5, jitter=0.05)
    k = int(np.argmin(np.linalg.norm(sc.x - sc.x.mean(0), axis=1)))
    extra = sc.x[k] + np.array([0.38, 0.1, 0.05]) * sc.h
    sc.x = np.vstack([sc.x, extra])
    sc.vol = np.append(sc.vol, 0.5 * sc.h ** 3)
    sc.grain = np.append(sc.grain, np.int32(0)).astype(np.int32)
    sc.v0 = np.zeros_like(sc.x)
    # a tough material (s0 ~ 0.7) so that no bond but the planted one is broken
    sc.material.G0 *= 1e6
    return sc, k, sc.n - 1


def pair_slots(rp, col, i, j):
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return ((rows == i) & (col == j)) | ((rows == j) & (col == i))


@pytest.mark.parametrize("precision,tol,kernel", [("mixed", MIXED_FORCE_TOL, "global"),
                                                 ("mixed", MIXED_FORCE_TOL, "tiled"),
                                                 ("mixed", MIXED_FORCE_TOL, "pairs"),
                                                 ("fp64", FP64_FORCE_TOL, "fp64")])
@pytest.mark.parametrize("micromodulus", [0, 1])
def test_self_contact_repulsion_forces(pd, precision, tol, kernel, micromodulus):
    """The broken pair pushed to |d| = 0.25 h: forces against the oracle, and the
    contact part alone (forces with contact minus without) against the oracle's,
    so that the branch cannot hide under the bond forces."""
    sc, k, e = self_contact_block()
    sc.material.micromodulus = micromodulus
    ref = oracle.Model.from_scenario(sc)
    brk = pair_slots(ref.rowptr, ref.col, k, e).astype(np.uint8)
    assert brk.sum() == 2
    u = np.zeros_like(sc.x)
    d0 = sc.x[e] - sc.x[k]
    u[e] = -d0 + 0.25 * sc.h * d0 / np.linalg.norm(d0)
    outs = []
    for contact in (True, False):
        ctx = pd.Context.from_scenario(sc, precision=precision, lanes=8, contact=contact, **KERNEL[kernel])
        ctx.set_state(u=u, broken=brk)
        F = ctx.forces()
        _, _, broken, _ = ctx.get_state()
        ref.P.contact = 1 if contact else 0
        ref.u = u.copy()
        ref.broken[:] = brk
        ref.forces()
        assert np.array_equal(broken, ref.broken)
        outs.append((F, ref.F.copy()))
        if contact:
            assert rel_l2(F, ref.F) <= tol
            pairs = ctx.contacts()
            assert [k, e] in pairs.tolist() and [e, k] in pairs.tolist()
        ctx.close()
    Fc, Fco = outs[0][0] - outs[1][0], outs[0][1] - outs[1][1]
    K, c, s0, Kn = oracle.constants(sc.material.E, sc.material.G0, sc.horizon, micromodulus=micromodulus)
    L = np.linalg.norm(d0)
    cw = c * (sc.horizon - L) if micromodulus else c
    # hand value on the extra node: c (|d| - |xi|)/|xi| V_k, directed away from node k
    hand = -cw * (0.25 * sc.h - L) / L * sc.vol[k]
    assert np.dot(Fco[e], d0 / L) == pytest.approx(hand, rel=1e-9)
    assert rel_l2(Fc, Fco) <= (1e-4 if precision == "mixed" else 1e-9)


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-9)])
def test_self_contact_repulsion_trajectory(pd, precision, tol):
    """The extra node driven into its broken partner at 30 m/s: it is turned back
    by the PD-repulsive law; 60 steps against the oracle."""
    sc, k, e = self_contact_block()
    ref = oracle.Model.from_scenario(sc)
    brk = pair_slots(ref.rowptr, ref.col, k, e).astype(np.uint8)
    d0 = sc.x[e] - sc.x[k]
    v = np.zeros_like(sc.x)
    v[e] = -30.0 * d0 / np.linalg.norm(d0)
    ctx = pd.Context.from_scenario(sc, precision=precision, lanes=8)
    ctx.set_state(u=np.zeros_like(sc.x), v=v, broken=brk)
    ref.v = v.copy()
    ref.broken[:] = brk
    ref.init()
    dt = 0.5 * ref.stable_dt()
    assert ctx.stable_dt() == pytest.approx(ref.stable_dt(), rel=1e-12)
    closest = np.inf
    for _ in range(12):
        ctx.step(dt, 5)
        ref.step(dt, 5)
        closest = min(closest, np.linalg.norm((sc.x[e] + ref.u[e]) - (sc.x[k] + ref.u[k])))
    u, vg, broken, _ = ctx.get_state()
    assert closest < np.linalg.norm(d0)
    assert rel_l2(u, ref.u) < tol
    assert rel_l2(vg, ref.v) < 10 * tol
    ctx.close()


# --------------------------------------------------------------------------- several steps per launch
def _collision_scenario(zeta=0.0):
    from paper_2506_05362_gb300 import surrogate as SG
    sc = S.aggregate(n_grains=2, h=0.5e-3 / 4, gap_cells=0.5, seed=4)
    c = sc.x[sc.grain == 0].mean(0) - sc.x[sc.grain == 1].mean(0)
    c /= np.linalg.norm(c)
    sc.v0 = np.where((sc.grain == 0)[:, None], -8.0 * c, 8.0 * c)
    sc.walls = []
    if zeta:
        sc.material.beta_d = SG.damping_coefficient(sc.material, sc.horizon, sc.h ** 3, zeta)
    return sc


@pytest.mark.parametrize("case", ["sphere-mixed", "sphere-fp64", "collision", "collision-damped", "friction-walls"])
def test_multi_step_launch_equals_one_launch_per_step(pd, case):
    """The steps between two rebuilds in one cooperative launch (grid-wide barrier
    between steps) give bit for bit the trajectory of one launch per step: state,
    wall points, wall forces and their time average; with walls, contacts and
    rebuilds, pair damping, and the wall-friction kernels."""
    precision = "fp64" if case == "sphere-fp64" else "mixed"
    if case.startswith("sphere"):
        sc, steps, calls = S.sphere(), 150, 2
    elif case == "friction-walls":
        sc = damped_blocks()
        sc.material.mu = 0.4
        steps, calls = 60, 3
    else:
        sc, steps, calls = _collision_scenario(0.3 if case == "collision-damped" else 0.0), 300, 8
    ctxs = [pd.Context.from_scenario(sc, precision=precision, lanes=8, tiles=-1, pairs=-1, persistent=pm)
            for pm in (1, -1)]
    dt = 0.5 * ctxs[0].stable_dt()
    nw = len(sc.walls)
    for _ in range(calls):
        for ctx in ctxs:
            ctx.step(dt, steps)
    a, b = ctxs
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    if nw:
        assert np.array_equal(a.get_walls(), b.get_walls())
        areas = [1e-6] * nw
        assert np.array_equal(a.bulk_stress(areas)[1], b.bulk_stress(areas)[1])
        assert np.array_equal(a.bulk_stress_mean(areas)[1], b.bulk_stress_mean(areas)[1])
    assert a.step_counters() == b.step_counters()
    if case.startswith("collision"):
        assert len(a.contacts()) > 0
    a.close(); b.close()
