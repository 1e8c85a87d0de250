"""Failure paths of the hot path, made on the host (no GPU fault): an allocator
that refuses, a contact-candidate list too small for the contacts, and a
contact list that goes stale between rebuilds.  Each must end in the stated
status or be recovered from, with the trajectory still equal to the oracle's."""
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
    _pd.lib()
    return _pd


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def counting_allocator(pd, stream, fail_at=None):
    """PyTorch's caching allocator behind a counter; the fail_at-th request
    (0-based) and every later one return NULL.  live: blocks handed out and not
    yet given back."""

    class Alloc(pd._TorchAllocator):
        def __init__(self):
            super().__init__(0, stream)
            self.calls = 0
            self.live = set()

        def _alloc(self, nbytes, ctx):
            k = self.calls
            self.calls += 1
            if fail_at is not None and k >= fail_at:
                return None
            p = super()._alloc(nbytes, ctx)
            if p:
                self.live.add(int(p))
            return p

        def _free(self, ptr, ctx):
            self.live.discard(int(ptr))
            super()._free(ptr, ctx)

    return Alloc()


def test_allocator_refusal_gives_enomem_and_frees_everything(pd):
    """An allocator callback that returns NULL: pd_create (early, middle, last
    request) and pd_build_bonds fail with PD_ENOMEM, and every block the library
    obtained is handed back (by the failed pd_create itself, or by pd_destroy)."""
    import torch
    sc = S.small_block(nx=9, ny=7, nz=5, jitter=0.05)
    stream = torch.cuda.Stream(0)
    probe = counting_allocator(pd, stream.cuda_stream)
    ctx = pd.Context(sc.x, sc.vol, sc.grain, sc.material, stream=stream, allocator=probe, lanes=8)
    n_create = probe.calls
    ctx.build_bonds(sc.horizon)
    n_total = probe.calls
    ctx.close()
    assert not probe.live
    assert n_create > 10 and n_total > n_create
    for k in (0, n_create // 2, n_create - 1):
        a = counting_allocator(pd, stream.cuda_stream, fail_at=k)
        with pytest.raises(pd.PDError) as e:
            pd.Context(sc.x, sc.vol, sc.grain, sc.material, stream=stream, allocator=a, lanes=8)
        assert e.value.status == pd.PD_ENOMEM
        assert not a.live, f"{len(a.live)} blocks leaked after a refusal at request {k}"
    for k in (n_create, n_create + (n_total - n_create) // 2):
        a = counting_allocator(pd, stream.cuda_stream, fail_at=k)
        ctx = pd.Context(sc.x, sc.vol, sc.grain, sc.material, stream=stream, allocator=a, lanes=8)
        with pytest.raises(pd.PDError) as e:
            ctx.build_bonds(sc.horizon)
        assert e.value.status == pd.PD_ENOMEM
        ctx.close()
        assert not a.live, f"{len(a.live)} blocks leaked after a refusal at request {k}"
    torch.cuda.synchronize()


def colliding_pair(speed=5.0):
    sc = S.aggregate(n_grains=2, h=0.5e-3 / 4, gap_cells=0.5, seed=4)
    c = sc.x[sc.grain == 0].mean(0) - sc.x[sc.grain == 1].mean(0)
    c /= np.linalg.norm(c)
    sc.v0 = np.where((sc.grain == 0)[:, None], -speed * c, speed * c)
    sc.walls = []
    return sc


def run_collision(pd, sc, steps_per_call=10, max_steps=20000, after_touch=80, **kw):
    ctx = pd.Context.from_scenario(sc, **kw)
    ref = oracle.Model.from_scenario(sc)
    dt = 0.5 * ref.stable_dt()
    ref.init()
    touched, total = 0, 0
    while total < max_steps and touched < after_touch:
        ref.step(dt, steps_per_call)
        ctx.step(dt, steps_per_call)
        total += steps_per_call
        if touched or len(ref.contact_pairs()) > 0:
            touched += steps_per_call
    assert touched > 0, "grains never met"
    return ctx, ref


def test_candidate_list_regrows_and_trajectory_holds(pd):
    """An initial candidate capacity of 16 entries: the first rebuild in contact
    overflows it, the segment is rolled back, the list grows, and the run goes on
    to the oracle's trajectory."""
    sc = colliding_pair()
    ctx, ref = run_collision(pd, sc, cand_capacity=16)
    steps, rebuilds, rollbacks = ctx.step_counters()
    assert rollbacks > 0
    u, v, _, _ = ctx.get_state()
    assert rel_l2(u, ref.u) < 1e-5
    assert rel_l2(v, ref.v) < 1e-4
    assert len(ctx.contacts()) == len(ref.contact_pairs())
    ctx.close()


def test_stale_contact_list_rolls_back_and_trajectory_holds(pd):
    """A rebuild period far too long for a thin skin (40 steps; skin 2% of R_c, so
    a node at 5 m/s uses up half the skin in ~14 steps), in calls of 50 steps
    (each call rebuilds at its start): the device flags the stale list, the
    segment is rolled back and rerun with a shorter period, and the trajectory
    equals the oracle's, which rebuilds every step."""
    sc = colliding_pair()
    ctx, ref = run_collision(pd, sc, steps_per_call=50, after_touch=100, contact_every=40,
                             skin=0.02 * sc.material.contact_radius)
    steps, rebuilds, rollbacks = ctx.step_counters()
    assert rollbacks > 0
    assert rebuilds > steps / 40
    u, v, _, _ = ctx.get_state()
    assert rel_l2(u, ref.u) < 1e-5
    assert rel_l2(v, ref.v) < 1e-4
    ctx.close()


def test_bad_candidate_capacity_is_rejected(pd):
    sc = S.small_block()
    with pytest.raises(pd.PDError) as e:
        pd.Context(sc.x, sc.vol, sc.grain, sc.material, cand_capacity=-1)
    assert e.value.status == pd.PD_EINVAL


def test_grid_barrier_wait_runs_out_and_is_reported(pd):
    """The multi-step kernel's grid barrier told to wait for one block more than
    it launches (pd_options.barrier_absent, a test aid): every wait gives up after
    1 s of GPU time, the kernel returns with its error bit, pd_step reports
    PD_ETIMEOUT, the state of the segment's start is restored, the context refuses
    pd_step until pd_set_state, and the device stays usable."""
    import time
    sc = S.sphere()
    ctx = pd.Context.from_scenario(sc, lanes=8, tiles=-1, pairs=-1, persistent=1, barrier_absent=1)
    before = ctx.get_state()
    dt = 0.8 * ctx.stable_dt()
    t0 = time.perf_counter()
    with pytest.raises(pd.PDError) as e:
        ctx.step(dt, 20)
    assert e.value.status == pd.PD_ETIMEOUT and "barrier" in str(e.value)
    assert time.perf_counter() - t0 < 60
    for x, y in zip(ctx.get_state(), before):
        assert np.array_equal(x, y)
    with pytest.raises(pd.PDError) as e:
        ctx.step(dt, 1)
    assert e.value.status == pd.PD_ESTATE
    ctx.close()
    ok = pd.Context.from_scenario(sc, lanes=8, tiles=-1, pairs=-1, persistent=1)
    ok.step(dt, 20)
    assert np.all(np.isfinite(ok.get_state()[0]))
    ok.close()
