"""RVE surrogate pipeline on the GPU: data from the PD hot path, training with the
project's BF16 kernels, and judgement of held-out runs by their own PD results.

What the network gains over the method without it is time: a prediction for a
whole run in a small fraction of the PD run.  Its accuracy on held-out runs is
measured (by rerunning PD) and reported, not asserted against the 5% target:
the wall stress of granular RVEs moves with force-chain rearrangement; on a fixed
held-out set the measured error stays at ~0.15 of the peak stress from 10 to 45
training aggregates (half the mean-history baseline's, far from 5%)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_rve_runs_are_reproducible_and_compacted():
    """An RVE run pre-compresses to a contact network and is bit-reproducible
    (fixed step configuration)."""
    from paper_2506_05362_gb300 import surrogate as SG
    a = SG.rve_run("uniaxial_z", n_grains=8, seed=3, records=24, zeta=0.5)
    b = SG.rve_run("uniaxial_z", n_grains=8, seed=3, records=24, zeta=0.5)
    assert np.array_equal(a.stress, b.stress) and np.array_equal(a.strain, b.strain)
    assert a.precompress_steps > 0
    assert a.sf_confine > 0.45 or a.p_confine >= 2e6
    assert a.desc[0, 8] > 1.0                      # contacts per grain after compaction
    assert np.all(np.isfinite(a.stress))
    assert a.stress[:, :3].mean() < 0              # compression is negative
    assert a.strain[-1, 2] < -0.03                 # the loaded axis shortened


def test_paths_branch_from_one_shared_precompression():
    """Loading paths from one saved pre-compressed state: a path run again after
    another path gives the same record bit for bit (no state leaks between
    branches), and every branch starts from the same compacted box."""
    from paper_2506_05362_gb300 import surrogate as SG
    runs = SG.rve_aggregate(8, seed=5, paths=["uniaxial_z", "isotropic", "uniaxial_z"], records=24, h=0.5e-3 / 6,
                            zeta=0.5, max_precompress=40000)
    a, b, c = runs
    assert np.array_equal(a.stress, c.stress) and np.array_equal(a.strain, c.strain)
    assert np.array_equal(a.desc, c.desc)
    assert a.precompress_steps == b.precompress_steps and a.p_confine == b.p_confine
    assert not np.array_equal(a.stress, b.stress)
    assert a.strain[-1, 2] < -0.03 and b.strain[-1, 0] < -0.03 and abs(a.strain[-1, 0]) < 1e-12
    assert np.all(np.isfinite(b.stress)) and b.stress[:, :3].mean() < 0


def test_twin_runs_repeat_exactly_and_diverge_when_perturbed():
    """The spread measurement behind the surrogate's error floor: a path loaded
    twice from one saved packing gives the same bits; displaced by 1e-6 h it
    gives a different history."""
    from paper_2506_05362_gb300 import surrogate as SG
    recs = SG.twin_spread(8, seed=5, paths=["uniaxial_z"], eps=(0.0, 1e-6), records=24, h=0.5e-3 / 6,
                          max_precompress=40000)
    assert recs[0]["identical"] and recs[0]["spread"] == 0.0
    assert not recs[1]["identical"] and recs[1]["spread"] > 0.0


def test_surrogate_trains_and_is_judged_by_pd():
    from paper_2506_05362_gb300 import surrogate as SG
    runs = []
    for path in ["uniaxial_z", "biaxial_xy"]:
        for r in range(4):
            runs.append(SG.rve_run(path, n_grains=8, seed=100 * r + len(path), records=40, zeta=0.5))
    held = [runs[3], runs[7]]
    train = [r for r in runs if r not in held]
    net, xs, ys, losses = SG.train(train, epochs=400)
    assert losses[-1] < 0.1 * losses[0]
    # the network fits the runs it was trained on
    for r in train[:2]:
        err, _ = SG.judge(net, xs, ys, r)
        assert err < 0.1
    errs, bases = [], []
    for r in held:
        err, t_net = SG.judge(net, xs, ys, r)
        base = SG.baseline_error(train, r)
        print(f"held-out {r.path}: error {err:.4f}, mean-history baseline {base:.4f}")
        assert np.isfinite(err) and err > 0
        errs.append(err)
        bases.append(base)
        # the gain: the whole run's stress history in a small fraction of its PD time
        assert r.pd_seconds / t_net > 100
    # what the network knows beyond the method without it: on average over the
    # held-out runs, stress histories closer than the mean history of the training
    # runs (with 3 training runs per path one held-out run may not be; at the study's
    # scale 23 of 24 are)
    assert np.mean(errs) < np.mean(bases)
    net.close()
