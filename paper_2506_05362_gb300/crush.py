"""Hollow-sphere crushing between two plates (Sec. 6.3 setting): the run as the
hollow-sphere configuration states it, with the plate reaction-force curve and
the damage field written as arrays.

A glass shell (R = 1 mm, r = 0.7 mm, h = 0.02 mm, delta = 3h) sits between two
rigid frictionless plates that close at 5 m/s each.  The first 10,000 steps are
taken by one pd_step call whose steps form one captured CUDA graph (the graph
chunk is set to the call's length); the run then continues to 20% strain (plate
approach over the outer diameter).  The recorded curve comes from a second
context on the same input that steps in short calls: forces do not depend on the
rebuild history, so its state at step 10,000 equals the one-graph run bit for
bit (checked by the command line below).

  python -m paper_2506_05362_gb300.crush --out hollow_crush.npz
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import scenarios as S


def plate_gap(ctx, sc):
    """Distance between the two plates (walls 0 = top, 1 = bottom)."""
    w = ctx.get_walls()
    return float(w[0, 2] - w[1, 2])


def crush(sc, dt=None, graph_steps=10000, strain_end=0.2, record_every=100, device=0, stream=None,
          check_graph=True):
    """Runs the crushing of ``sc`` (a scenario with a top and a bottom plate).

    Returns a dict of arrays: t, approach, strain (approach / outer diameter), the
    plate forces (time-averaged over each record interval, z components, top and
    bottom, N), the bulk stress sigma_zz of the top plate over its disc area, the
    mean damage and broken-bond fraction per record, the damage field phi (caller
    order) at ``graph_steps`` and at the end, the step counts and timings."""
    from . import pd
    import torch
    diam = float(sc.x[:, 2].max() - sc.x[:, 2].min())
    rec = pd.Context.from_scenario(sc, device=device, stream=stream)
    if dt is None:
        dt = 0.8 * rec.stable_dt()
    gap0 = plate_gap(rec, sc)
    rp, _ = rec.bonds()
    nb0 = np.diff(rp).astype(np.float64)
    B = max(float(nb0.sum()), 1.0)
    area = [sc.wall_area, sc.wall_area]
    out = {k: [] for k in ("t", "approach", "strain", "force_top", "force_bottom", "sigma_zz", "damage_mean",
                           "broken_fraction")}
    steps = 0
    phi_graph = None
    t_rec = time.perf_counter()
    while True:
        n = min(record_every, graph_steps - steps) if steps < graph_steps else record_every
        rec.step(dt, n)
        steps += n
        sig, wf, span = rec.bulk_stress_mean(area)
        gap = plate_gap(rec, sc)
        phi = rec.damage()
        out["t"].append(steps * dt)
        out["approach"].append(gap0 - gap)
        out["strain"].append((gap0 - gap) / diam)
        out["force_top"].append(float(wf[0, 2]))
        out["force_bottom"].append(float(wf[1, 2]))
        out["sigma_zz"].append(float(sig[2]))
        out["damage_mean"].append(float(phi.mean()))
        out["broken_fraction"].append(float((phi * nb0).sum() / B))
        if steps == graph_steps:
            phi_graph = phi.copy()
            state_graph = rec.get_state()
        if steps >= graph_steps and out["strain"][-1] >= strain_end:
            break
    torch.cuda.synchronize()
    t_rec = time.perf_counter() - t_rec
    res = {k: np.asarray(v) for k, v in out.items()}
    res.update(phi_graph=phi_graph, phi_end=rec.damage(), steps_total=steps, dt=dt, diameter=diam,
               record_every=record_every, seconds_recorded_run=t_rec,
               fragments_end=rec.fragments()[1])
    rec.close()
    if check_graph:
        # the first graph_steps steps as one call whose steps form one captured graph:
        # a rebuild period that divides the call (50 steps; at the plates' 5 m/s a
        # node uses up a fifth of the skin in that time) and a graph chunk of the
        # call's length
        kw = dict(device=device, stream=stream, chunk=graph_steps, contact_every=50)
        one = pd.Context.from_scenario(sc, **kw)
        one.step(dt, graph_steps)  # captures and runs the graph (a warm context is not needed)
        u1, v1, b1, t1 = one.get_state()
        same = all(np.array_equal(a, b) for a, b in zip((u1, v1, b1), state_graph[:3]))
        # time a second one-graph run on a fresh context (graph captured during its call)
        two = pd.Context.from_scenario(sc, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        two.step(dt, graph_steps)
        torch.cuda.synchronize()
        res.update(graph_equal_to_recorded=bool(same), seconds_one_graph=time.perf_counter() - t0,
                   graph_launches=two.last_step_stats()[2])
        one.close()
        two.close()
    return res


def describe(res):
    """A short text summary of the curve's shape (for the profiles)."""
    f = 0.5 * (np.abs(res["force_top"]) + np.abs(res["force_bottom"]))
    k = int(np.argmax(f))
    lines = [
        f"steps {res['steps_total']}, dt {res['dt']:.3e} s, final strain {res['strain'][-1]:.3f}",
        f"peak mean plate force {f[k]:.4g} N at strain {res['strain'][k]:.4f} (t = {res['t'][k]:.3e} s)",
        f"force at the end {f[-1]:.4g} N ({f[-1] / max(f[k], 1e-300):.2f} of the peak)",
        f"damage mean: {res['damage_mean'][len(f) // 4]:.4f} at a quarter of the run, "
        f"{res['damage_mean'][-1]:.4f} at the end; broken bonds {res['broken_fraction'][-1]:.4f}",
        f"fragments at the end: {res['fragments_end']}",
    ]
    if "graph_equal_to_recorded" in res:
        lines.append(f"one-graph run of the first steps equal to the recorded run: {res['graph_equal_to_recorded']}; "
                     f"{res['seconds_one_graph']:.3f} s for the one-graph call")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser(description="hollow-sphere crushing to 20% strain")
    ap.add_argument("--out", default="hollow_crush.npz")
    ap.add_argument("--graph-steps", type=int, default=10000)
    ap.add_argument("--strain", type=float, default=0.2)
    ap.add_argument("--record-every", type=int, default=100)
    ap.add_argument("--outer-cells", type=int, default=50)
    ap.add_argument("--inner-cells", type=int, default=35)
    args = ap.parse_args()
    sc = S.hollow(outer_cells=args.outer_cells, inner_cells=args.inner_cells)
    res = crush(sc, graph_steps=args.graph_steps, strain_end=args.strain, record_every=args.record_every)
    np.savez_compressed(args.out, **{k: v for k, v in res.items()})
    print(describe(res))
    print(json.dumps({k: (float(v) if np.isscalar(v) and not isinstance(v, (bool, np.bool_)) else v)
                      for k, v in res.items() if np.isscalar(v) or isinstance(v, (bool, int, float))}))


if __name__ == "__main__":
    main()
