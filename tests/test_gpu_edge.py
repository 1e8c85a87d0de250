"""Degenerate inputs on the GPU: a single node, nodes without bonds next to a
bonded body, zero steps, no walls, and the exact free fall under a body force
(velocity Verlet integrates a constant acceleration exactly, Sec. 5.2)."""
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


MAT = S.Material(E=72e9, rho=2000.0, G0=135.0, contact_radius=0.6e-4)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_single_node_free_fall(pd, precision):
    """One node, no bonds, no contact partners, gravity-like body force: the
    state after 100 steps is the closed form; damage and fragments are trivial."""
    g = -9.81
    ctx = pd.Context(np.array([[1e-3, 2e-3, 3e-3]]), np.array([1e-12]), np.array([0], np.int32), MAT,
                     precision=precision)
    ctx.set_body_force([0.0, 0.0, MAT.rho * g])
    ctx.build_bonds(1e-4)
    assert ctx.B == 0
    dt = 1e-4
    ctx.step(dt, 0)  # zero steps: a no-op
    u, v, broken, t = ctx.get_state()
    assert t == 0.0 and np.all(u == 0)
    ctx.step(dt, 100)
    u, v, broken, t = ctx.get_state()
    T = 100 * dt
    # the mixed path holds u, v in double-float pairs but forms the acceleration
    # (F + b) / rho in FP32 (force arithmetic in FP32): 2^-24 relative per step,
    # the same sign every step here
    rel = 1e-12 if precision == "fp64" else 1e-6
    assert u[0, 2] == pytest.approx(0.5 * g * T * T, rel=rel)
    assert v[0, 2] == pytest.approx(g * T, rel=rel)
    assert np.all(u[0, :2] == 0) and np.all(v[0, :2] == 0)
    assert ctx.damage().tolist() == [0.0]
    label, nf = ctx.fragments()
    assert nf == 1 and label.tolist() == [0]
    sig, wf = ctx.bulk_stress()  # no walls: zero stress, no areas needed
    assert np.all(sig == 0) and wf.shape == (0, 3)
    ctx.close()


def test_isolated_nodes_next_to_a_body(pd):
    """A bonded block plus nodes farther than the horizon from everything: the
    lone nodes have no bonds (damage 0, one fragment each), the block's forces
    match the oracle, and every node falls under the body force."""
    sc = S.small_block(nx=6, ny=5, nz=4, jitter=0.05)
    far = np.array([[0.1, 0.1, 0.1], [-0.1, 0.05, 0.0], [0.05, -0.1, 0.02]])
    x = np.concatenate([sc.x, far])
    n = len(x)
    vol = np.full(n, sc.h ** 3)
    grain = np.concatenate([sc.grain, np.array([1, 2, 3], np.int32)])
    ctx = pd.Context(x, vol, grain, sc.material, lanes=8)
    ctx.set_body_force([0.0, 0.0, -50.0])
    ctx.build_bonds(sc.horizon)
    rp, col = ctx.bonds()
    assert np.all(np.diff(rp)[-3:] == 0)
    orp, ocol = oracle.bonds(x, grain, sc.horizon)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    label, nf = ctx.fragments()
    assert nf == 4 and label[-3:].tolist() == [n - 3, n - 2, n - 1]
    rng = np.random.default_rng(5)
    u = rng.normal(0, 1e-3 * sc.h, x.shape)
    ctx.set_state(u=u)
    F = ctx.forces()
    ref = oracle.Model(x, vol, grain, orp, ocol, sc.material, sc.horizon, body_force=(0, 0, -50.0))
    ref.u = u.copy()
    ref.forces()
    assert np.linalg.norm(F - ref.F) / np.linalg.norm(ref.F) < 1e-5
    assert np.all(F[-3:] == 0)
    assert np.all(ctx.damage()[-3:] == 0)
    ctx.close()
