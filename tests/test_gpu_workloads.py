"""The paper's further workloads (shape study of Sec. 6.5: spheres, shells, jacks
on a cubic grid under a descending wall; the double hollow sphere of Sec. 6.3) at
reduced sizes: bond lists bit-exact and trajectories against the oracle."""
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


CASES = {
    "shape_sphere": lambda: S.shape_study("sphere", n_side=2, h=1e-3 / 5),
    "shape_shell": lambda: S.shape_study("shell", n_side=2, h=1e-3 / 6),
    "shape_jack": lambda: S.shape_study("jack", n_side=2, h=1e-3 / 6),
    "double_hollow": lambda: S.double_hollow(h=1e-3 / 8),
}


@pytest.mark.parametrize("name", list(CASES))
def test_workload_lists_and_trajectory(pd, name):
    sc = CASES[name]()
    # start the top wall inside the contact range so the walls act from the first step
    sc.walls[-1] = S.Wall(sc.walls[-1].normal, (0.0, 0.0, sc.walls[-1].point[2] - 0.5 * sc.material.contact_radius),
                          (0.0, 0.0, -50.0))
    ctx = pd.Context.from_scenario(sc, lanes=8)
    ref = oracle.Model.from_scenario(sc)
    rp, col = ctx.bonds()
    assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col)
    dt = 0.8 * ref.stable_dt()
    assert ctx.stable_dt() == pytest.approx(ref.stable_dt(), rel=1e-12)
    ref.init()
    ctx.step(dt, 60)
    ref.step(dt, 60)
    u, v, broken, _ = ctx.get_state()
    assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) < 1e-5
    sig, wf = ctx.bulk_stress([sc.wall_area] * len(sc.walls))
    assert np.abs(ref.react).max() > 0, "the top wall should push"
    assert np.linalg.norm(wf - ref.react) / np.linalg.norm(ref.react) < 1e-5
    ctx.close()


def test_hollow_crush_small_against_oracle(pd):
    """The hollow-sphere crushing run (crush.py) on a reduced shell (R = 14 h, r = 9 h):
    200 steps, before any bond breaks, recorded every 20 steps.  The plate-force
    curve (time-averaged wall forces of each record interval) follows the oracle's,
    and the first 200 steps taken as one captured graph end in the recorded run's
    state bit for bit."""
    from paper_2506_05362_gb300 import crush as C
    sc = S.hollow(outer_cells=14, inner_cells=9)
    ref = oracle.Model.from_scenario(sc)
    dt = 0.8 * ref.stable_dt()
    res = C.crush(sc, dt=dt, graph_steps=200, strain_end=0.0, record_every=20)
    assert res["graph_equal_to_recorded"]
    ref.init()
    F = []
    for _ in range(len(res["t"])):
        ref.step(dt, 20)
        F.append(ref.bulk_stress_mean([sc.wall_area] * 2)[1][:, 2].copy())
    F = np.array(F)
    assert ref.broken.sum() == 0, "the window should end before damage"
    got = np.stack([res["force_top"], res["force_bottom"]], 1)
    assert np.abs(F).max() > 0
    assert np.linalg.norm(got - F) / np.linalg.norm(F) < 1e-5
    assert np.allclose(res["strain"][-1], (2 * 5.0 * 200 * dt) / res["diameter"], rtol=1e-9)
