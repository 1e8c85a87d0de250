"""Bulk-stress surrogate of a representative volume (RVE) of grains.

The paper motivates RVEs (the force per area of crushed aggregates converges
with grain count, Sec. 6.4, pointing to multiscale use) but builds none.  Here
an MLP learns the bulk stress of small star-grain aggregates from their recent
strain history and descriptors, from data that the peridynamic hot path itself
generates, and is judged against a fresh full PD run.

Data: an aggregate in a box of six rigid walls is compressed isotropically to a
confining pressure, then strained at a constant rate along one of 8 loading paths
(wall velocities per axis); every ``stride`` steps the macroscopic strain (from
wall positions) and the bulk stress of the wall forces averaged over the interval
(pd_bulk_stress_mean) are recorded.  A sample is a window of 16 strain records (6 Voigt components,
the shear ones are zero for axis-aligned walls) plus 13 descriptors at the
window end (109 inputs); the target is the stress (6) at the window end.
Inputs and targets are standardised with the training set's statistics.

All simulation runs in libpd (pd_step), all network arithmetic in the BF16
tensor-core kernels (pd_mlp_*); this module only arranges arrays.
"""
from __future__ import annotations

import dataclasses
import math
import time
from dataclasses import dataclass

import numpy as np

from . import scenarios as S

# strain-rate multipliers per axis (compression positive)
LOADING_PATHS = {
    "uniaxial_x": (1.0, 0.0, 0.0),
    "uniaxial_y": (0.0, 1.0, 0.0),
    "uniaxial_z": (0.0, 0.0, 1.0),
    "biaxial_xy": (1.0, 1.0, 0.0),
    "biaxial_yz": (0.0, 1.0, 1.0),
    "biaxial_zx": (1.0, 0.0, 1.0),
    "isotropic": (1.0, 1.0, 1.0),
    "z_lateral_release": (-0.25, -0.25, 1.0),
}
WINDOW = 16
N_DESC = 13
N_IN = 6 * WINDOW + N_DESC   # 109
N_OUT = 6


@dataclass
class Run:
    path: str
    n_grains: int
    seed: int
    strain: np.ndarray      # (T, 6)
    stress: np.ndarray      # (T, 6) Pa
    desc: np.ndarray        # (T, 13)
    pd_seconds: float       # device+host time of the PD steps (pre-compression included)
    steps: int
    nodes: int
    precompress_steps: int = 0
    p_confine: float = 0.0  # mean wall stress reached by the pre-compression, Pa
    sf_confine: float = 0.0 # solid fraction at the end of the pre-compression


def save_runs(path: str, runs) -> None:
    """Writes runs to one .npz file (arrays stacked per field, in run order)."""
    import json
    meta = [{k: getattr(r, k) for k in ("path", "n_grains", "seed", "pd_seconds", "steps", "nodes",
                                        "precompress_steps", "p_confine", "sf_confine")} for r in runs]
    arr = {}
    for q, r in enumerate(runs):
        arr[f"strain{q}"], arr[f"stress{q}"], arr[f"desc{q}"] = r.strain, r.stress, r.desc
    np.savez_compressed(path, meta=np.array(json.dumps(meta)), **arr)


def load_runs(path: str):
    """Reads runs written by save_runs."""
    import json
    z = np.load(path)
    meta = json.loads(str(z["meta"]))
    return [Run(strain=z[f"strain{q}"], stress=z[f"stress{q}"], desc=z[f"desc{q}"], **m) for q, m in enumerate(meta)]


def damping_coefficient(material, horizon: float, volume: float, zeta: float) -> float:
    """beta_d (Sec. 3.3) giving a damping ratio ``zeta`` to two nodes of ``volume`` in
    contact: their relative motion has stiffness K_n V^2 (K_n = f_c 18 K / (pi delta^5),
    K = 2E/3), reduced mass rho V / 2 and damping beta_d V^2, so critical damping is
    beta_d = sqrt(2 K_n rho / V)."""
    K = 2.0 * material.E / 3.0
    Kn = material.contact_factor * 18.0 * K / (math.pi * horizon ** 5)
    return zeta * math.sqrt(2.0 * Kn * material.rho / volume)


def grain_shape_stats(x, grain, vol):
    """Equivalent radius, sphericity proxy (r_eq / r_max) and aspect ratio
    (sqrt of the extreme covariance eigenvalues) of every grain."""
    req, sph, asp = [], [], []
    for g in np.unique(grain):
        pts = x[grain == g]
        V = vol[grain == g].sum()
        r_eq = (3.0 * V / (4.0 * math.pi)) ** (1.0 / 3.0)
        c = pts.mean(0)
        r_max = np.linalg.norm(pts - c, axis=1).max() + 1e-30
        ev = np.linalg.eigvalsh(np.cov((pts - c).T) + 1e-30 * np.eye(3))
        req.append(r_eq)
        sph.append(min(1.0, r_eq / r_max))
        asp.append(math.sqrt(max(ev[-1], 1e-30) / max(ev[0], 1e-30)))
    return np.array(req), np.array(sph), np.array(asp)


def _box(pos):
    """(lo, hi) corners of the six-wall box from the wall points (order -x, +x, -y, +y, -z, +z)."""
    lo = np.array([pos[0, 0], pos[2, 1], pos[4, 2]])
    hi = np.array([pos[1, 0], pos[3, 1], pos[5, 2]])
    return lo, hi


def _areas(L):
    return np.array([L[1] * L[2]] * 2 + [L[0] * L[2]] * 2 + [L[0] * L[1]] * 2)


def _rve_setup(n_grains, seed, h, G0, zeta, rate, device, stream, lanes):
    """Aggregate, box walls moving inward at ``rate`` (isotropic pre-compression)
    and a context with a fixed kernel configuration."""
    from . import pd
    sc = S.aggregate(n_grains=n_grains, seed=seed, h=h, gap_cells=0.5)
    if G0 is not None:  # fracture energy of the grains (glass: 135 J/m^2)
        sc.material = dataclasses.replace(sc.material, G0=G0)
    if zeta > 0:  # normal contact damping (Sec. 3.3) at this ratio of critical for a node pair
        sc.material = dataclasses.replace(sc.material, beta_d=damping_coefficient(sc.material, sc.horizon,
                                                                                  float(sc.vol.mean()), zeta))
    walls = S.walls_array(sc.walls)
    lo, hi = _box(walls[:, 3:6])
    L0 = hi - lo
    walls[:, 6:9] = 0.0
    for k in range(3):  # isotropic pre-compression: every wall moves inward
        walls[2 * k, 6 + k] = 0.5 * rate * L0[k]
        walls[2 * k + 1, 6 + k] = -0.5 * rate * L0[k]
    sc.walls = [S.Wall(tuple(w[0:3]), tuple(w[3:6]), tuple(w[6:9])) for w in walls]
    ctx = pd.Context.from_scenario(sc, device=device, stream=stream, lanes=lanes, tiles=-1)
    return sc, walls, ctx


def _precompress(ctx, sc, dt, p_confine, sf_max, max_precompress):
    """Steps until the mean wall stress reaches p_confine or the solid fraction
    sf_max; returns (steps, mean wall stress, solid fraction)."""
    vol_sum = sc.vol.sum()
    chunk, pc_steps, p_mean, sf = 64, 0, 0.0, 0.0
    while pc_steps < max_precompress:
        ctx.step(dt, chunk)
        pc_steps += chunk
        lo, hi = _box(ctx.get_walls())
        L = hi - lo
        sig, _, _ = ctx.bulk_stress_mean(_areas(L))
        p_mean = -float(np.mean(sig[:3]))
        sf = vol_sum / np.prod(L)
        if p_mean >= p_confine or sf >= sf_max:
            break
    return pc_steps, p_mean, sf


def _load(ctx, sc, walls, path, dt, rate, strain_end, records, n_grains):
    """Strains the compacted box along ``path`` (walls move from their current
    points) and records strain, time-averaged stress and descriptors; returns
    (strain, stress, desc, steps)."""
    mult = np.array(LOADING_PATHS[path])
    lo, hi = _box(ctx.get_walls())
    Lp = hi - lo
    walls = walls.copy()
    walls[:, 3:6] = ctx.get_walls()
    walls[:, 6:9] = 0.0
    for k in range(3):
        vk = 0.5 * mult[k] * rate * Lp[k]
        walls[2 * k, 6 + k] = vk        # lower wall moves up
        walls[2 * k + 1, 6 + k] = -vk   # upper wall moves down
    ctx.set_walls(walls)
    t_end = strain_end / (rate * max(abs(mult).max(), 1e-9))
    steps_total = max(records, int(math.ceil(t_end / dt)))
    stride = max(1, steps_total // records)
    req, sph, asp = grain_shape_stats(sc.x, sc.grain, sc.vol)
    static = [req.mean(), req.std(), sph.mean(), sph.std(), math.log(n_grains), asp.mean(), asp.std()]
    vol_sum = sc.vol.sum()
    strain = np.zeros((records, 6))
    stress = np.zeros((records, 6))
    desc = np.zeros((records, N_DESC))
    rp, _ = ctx.bonds()
    nb0 = np.diff(rp).astype(np.float64)
    B = max(float(nb0.sum()), 1.0)
    for r in range(records):
        ctx.step(dt, stride)
        lo_t, hi_t = _box(ctx.get_walls())
        L = hi_t - lo_t
        sig, _, _ = ctx.bulk_stress_mean(_areas(L))
        strain[r, :3] = (L - Lp) / Lp
        stress[r] = sig
        phi = ctx.damage()
        ncont = len(ctx.contacts())
        desc[r] = [vol_sum / np.prod(L), static[0], static[1], static[2], static[3], phi.mean(),
                   float((phi * nb0).sum()) / B, static[4], ncont / n_grains, static[5], static[6],
                   L.max() / L.min(), rate * abs(mult).max()]
    return strain, stress, desc, stride * records


def rve_run(path: str, n_grains: int = 8, seed: int = 0, rate: float = 2.0e3, strain_end: float = 0.04,
            records: int = 64, h: float = 0.5e-3 / 6, device: int = 0, stream=None, lanes: int = 8,
            p_confine: float = 2.0e6, sf_max: float = 0.62, max_precompress: int = 40000,
            G0: float = None, zeta: float = 0.0) -> Run:
    """One RVE run: an aggregate in a box of six rigid walls is first compressed
    isotropically at strain rate ``rate`` until the mean wall stress reaches the
    confining pressure ``p_confine`` (a connected contact network; the solid
    fraction is capped at ``sf_max``), then strained along ``path`` at ``rate`` up
    to ``strain_end`` on the dominant axis, recorded ``records`` times.  ``zeta`` > 0
    turns on the normal contact damping at that fraction of critical.  Strain is
    measured from the box at the end of the pre-compression; the recorded stress
    is that of the wall forces averaged over each record interval.

    The step kernel's configuration is fixed (``lanes`` per node, no tiles) so
    that a run is reproducible: the autotuner's choice would change the order of
    the force sums, and a granular packing amplifies rounding differences."""
    sc, walls, ctx = _rve_setup(n_grains, seed, h, G0, zeta, rate, device, stream, lanes)
    dt = 0.8 * ctx.stable_dt()
    t0 = time.perf_counter()
    pc_steps, p_mean, sf = _precompress(ctx, sc, dt, p_confine, sf_max, max_precompress)
    strain, stress, desc, steps = _load(ctx, sc, walls, path, dt, rate, strain_end, records, n_grains)
    pd_seconds = time.perf_counter() - t0
    ctx.close()
    return Run(path, n_grains, seed, strain, stress, desc, pd_seconds, pc_steps + steps, sc.n, pc_steps, p_mean, sf)


def rve_aggregate(n_grains: int = 50, seed: int = 0, paths=None, rate: float = 2.0e3, strain_end: float = 0.04,
                  records: int = 64, h: float = 0.5e-3 / 12, device: int = 0, stream=None, lanes: int = 8,
                  p_confine: float = 2.0e6, sf_max: float = 0.62, max_precompress: int = 80000,
                  G0: float = None, zeta: float = 0.0):
    """The runs of one aggregate along several loading paths (all eight by
    default): one pre-compression as in ``rve_run``, its end state (u, v, bond
    memory, time, wall points) saved, and every path loaded from that state.  A
    run's ``pd_seconds`` counts the pre-compression plus its own loading, the
    cost of producing that run alone."""
    paths = list(LOADING_PATHS) if paths is None else list(paths)
    sc, walls, ctx = _rve_setup(n_grains, seed, h, G0, zeta, rate, device, stream, lanes)
    dt = 0.8 * ctx.stable_dt()
    t0 = time.perf_counter()
    pc_steps, p_mean, sf = _precompress(ctx, sc, dt, p_confine, sf_max, max_precompress)
    u, v, broken, t = ctx.get_state()
    wall_pts = ctx.get_walls()
    t_pc = time.perf_counter() - t0
    runs = []
    for path in paths:
        t1 = time.perf_counter()
        w = walls.copy()
        w[:, 3:6] = wall_pts
        w[:, 6:9] = 0.0
        ctx.set_walls(w)
        ctx.set_state(u=u, v=v, broken=broken, t=t)
        strain, stress, desc, steps = _load(ctx, sc, walls, path, dt, rate, strain_end, records, n_grains)
        runs.append(Run(path, n_grains, seed, strain, stress, desc, t_pc + time.perf_counter() - t1,
                        pc_steps + steps, sc.n, pc_steps, p_mean, sf))
    ctx.close()
    return runs


def history_spread(a, b):
    """The surrogate's error measure between two stress histories [records x 6]:
    RMS over the windows' last records of |sigma_b - sigma_a|, over the largest
    |sigma_a| of the run."""
    err = np.linalg.norm(b[WINDOW - 1:] - a[WINDOW - 1:], axis=1)
    return float(np.sqrt((err ** 2).mean()) / (np.linalg.norm(a, axis=1).max() + 1e-30))


def twin_spread(n_grains: int = 50, seed: int = 0, paths=None, eps=(0.0, 1e-9, 1e-6), rate: float = 2.0e3,
                strain_end: float = 0.04, records: int = 64, h: float = 0.5e-3 / 12, zeta: float = 0.5,
                p_confine: float = 2.0e6, sf_max: float = 0.62, max_precompress: int = 80000, device: int = 0,
                stream=None, lanes: int = 8):
    """How far the stress history of one packing moves under a change no input can
    see: the aggregate is pre-compressed once as in ``rve_aggregate``, and every
    path is loaded from the saved state as it is and from the same state with
    every node displaced by eps * h in a random direction (eps = 0 repeats the run
    and must give the same bits).  Returns one record per (path, eps) with the
    spread of the two histories in the surrogate's error measure."""
    paths = list(LOADING_PATHS) if paths is None else list(paths)
    sc, walls, ctx = _rve_setup(n_grains, seed, h, None, zeta, rate, device, stream, lanes)
    dt = 0.8 * ctx.stable_dt()
    _precompress(ctx, sc, dt, p_confine, sf_max, max_precompress)
    u, v, broken, t = ctx.get_state()
    wall_pts = ctx.get_walls()
    rng = np.random.default_rng(seed + 99991)
    d = rng.normal(size=u.shape)
    d /= np.linalg.norm(d, axis=1, keepdims=True)

    def run_from(u0):
        w = walls.copy()
        w[:, 3:6] = wall_pts
        w[:, 6:9] = 0.0
        ctx.set_walls(w)
        ctx.set_state(u=u0, v=v, broken=broken, t=t)
        return _load(ctx, sc, walls, path, dt, rate, strain_end, records, n_grains)[1]

    out = []
    for path in paths:
        ref = run_from(u)
        for e in eps:
            twin = run_from(u + e * h * d)
            out.append({"path": path, "eps": e, "spread": history_spread(ref, twin),
                        "identical": bool(np.array_equal(ref, twin))})
    ctx.close()
    return out


def windows(run: Run):
    """(X (m, 109), Y (m, 6)) samples of one run."""
    T = run.strain.shape[0]
    X, Y = [], []
    for t in range(WINDOW - 1, T):
        X.append(np.concatenate([run.strain[t - WINDOW + 1:t + 1].ravel(), run.desc[t]]))
        Y.append(run.stress[t])
    return np.array(X), np.array(Y)


class Scaler:
    def __init__(self, A):
        self.mu = A.mean(0)
        sd = A.std(0)
        self.sd = np.where(sd > 1e-12 * (np.abs(self.mu) + 1e-30), sd, 1.0)

    def fwd(self, A):
        return (A - self.mu) / self.sd

    def inv(self, A):
        return A * self.sd + self.mu


def train(runs, epochs=300, batch=4096, lr=1e-3, seed=0, device=0, stream=None, val_runs=None):
    """Trains the MLP on all windows of ``runs`` on the GPU; returns (net,
    x_scaler, y_scaler, losses).  With ``val_runs`` (runs kept out of the training
    set) the network is evaluated on them every 10 epochs and the parameters with
    the lowest validation error are kept (early stopping)."""
    import torch
    from . import pd
    X = np.concatenate([windows(r)[0] for r in runs])
    Y = np.concatenate([windows(r)[1] for r in runs])
    xs, ys = Scaler(X), Scaler(Y)
    dev = torch.device("cuda", device)
    Xd = torch.tensor(xs.fwd(X), dtype=torch.float32, device=dev)
    Yd = torch.tensor(ys.fwd(Y), dtype=torch.float32, device=dev)
    net = pd.MLP((N_IN, 256, 256, 256, 256, N_OUT), seed=seed, device=device, stream=stream)
    g = torch.Generator(device="cpu").manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    losses = []
    m = Xd.shape[0]
    best, best_params = math.inf, None
    for ep in range(epochs):
        perm = torch.randperm(m, generator=g).to(dev)
        lr_ep = lr * (0.5 * (1 + math.cos(math.pi * ep / epochs)) * 0.9 + 0.1)
        for b0 in range(0, m, batch):
            idx = perm[b0:b0 + batch]
            xb = Xd.index_select(0, idx).contiguous()
            yb = Yd.index_select(0, idx).contiguous()
            net.train_step_device(xb, yb, lr_ep, loss)
        if ep % 10 == 0 or ep == epochs - 1:
            torch.cuda.synchronize(dev)
            losses.append(float(loss.item()))
            if val_runs:
                err = float(np.mean([judge(net, xs, ys, r, device=device)[0] for r in val_runs]))
                if err < best:
                    best, best_params = err, net.get_params()
    if best_params is not None:
        net.set_params(best_params)
    return net, xs, ys, losses


def judge(net, xs, ys, run: Run, device=0):
    """Error of the surrogate on one run, judged against the PD result:
    RMS over windows of |sigma_pred - sigma_PD| / max over the run of |sigma_PD|;
    and the time the network needs for the run's windows."""
    import torch
    X, Y = windows(run)
    dev = torch.device("cuda", device)
    Xd = torch.tensor(xs.fwd(X), dtype=torch.float32, device=dev)
    Yd = torch.empty((X.shape[0], N_OUT), dtype=torch.float32, device=dev)
    net.forward_device(Xd, Yd)  # warm
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    net.forward_device(Xd, Yd)
    torch.cuda.synchronize(dev)
    t_net = time.perf_counter() - t0
    pred = ys.inv(Yd.cpu().numpy().astype(np.float64))
    err = np.linalg.norm(pred - Y, axis=1)
    scale = np.linalg.norm(run.stress, axis=1).max() + 1e-30
    return float(np.sqrt((err ** 2).mean()) / scale), t_net


def baseline_error(train_runs, run: Run):
    """Error of the method without a surrogate of the history: the mean stress of
    the training runs at the same record index (what is known before running)."""
    S_mean = np.mean([r.stress for r in train_runs], axis=0)
    X, Y = windows(run)
    pred = S_mean[WINDOW - 1:]
    err = np.linalg.norm(pred - Y, axis=1)
    scale = np.linalg.norm(run.stress, axis=1).max() + 1e-30
    return float(np.sqrt((err ** 2).mean()) / scale)


def study(runs_per_path: int = 4, grain_counts=(8, 12), epochs: int = 300, rate: float = 2.0e3,
          records: int = 64, seed: int = 0, device: int = 0, zeta: float = 0.0, runs=None, log=print):
    """Generates runs_per_path runs per loading path (grain counts cycling through
    grain_counts, seeds distinct, contact damping ratio zeta), or takes ``runs``
    already generated in that order, holds out the last run of every path, trains
    on the rest and judges the held-out runs against their PD results."""
    # the network runs on torch's current stream (its tensors are made there);
    # every PD context makes its own capturable stream and synchronises on return
    stream = None
    t0 = time.perf_counter()
    if runs is None:
        runs = []
        for pi, path in enumerate(LOADING_PATHS):
            for r in range(runs_per_path):
                ng = grain_counts[r % len(grain_counts)]
                runs.append(rve_run(path, n_grains=ng, seed=seed + 1000 * pi + r, rate=rate, records=records,
                                    device=device, stream=stream, zeta=zeta))
    else:
        assert len(runs) == runs_per_path * len(LOADING_PATHS)
    t_data = time.perf_counter() - t0
    held = [runs[(pi + 1) * runs_per_path - 1] for pi in range(len(LOADING_PATHS))]
    train_runs = [r for r in runs if r not in held]
    # early stopping on the second-last run of every path (not used for training)
    val = [runs[(pi + 1) * runs_per_path - 2] for pi in range(len(LOADING_PATHS))] if runs_per_path >= 4 else []
    fit = [r for r in train_runs if r not in val]
    return _fit_and_judge(runs, fit, val, held, train_runs, t_data, epochs, seed, device, stream)


def _fit_and_judge(runs, fit, val, held, known, t_data, epochs, seed, device, stream):
    """Trains on ``fit`` (early stopping on ``val``), judges every ``held`` run by
    its own PD result and the mean-history baseline of the ``known`` runs."""
    t0 = time.perf_counter()
    net, xs, ys, losses = train(fit, epochs=epochs, seed=seed, device=device, stream=stream, val_runs=val)
    t_train = time.perf_counter() - t0
    rows = []
    for r in held:
        err, t_net = judge(net, xs, ys, r, device=device)
        rows.append({"path": r.path, "grains": r.n_grains, "seed": r.seed, "nodes": r.nodes, "steps": r.steps,
                     "err": err, "err_mean_history": baseline_error(known, r),
                     "pd_seconds": r.pd_seconds, "net_seconds": t_net, "speedup": r.pd_seconds / max(t_net, 1e-9)})
    errs = np.array([q["err"] for q in rows])
    train_err = [judge(net, xs, ys, r, device=device)[0] for r in fit[:16]]
    net.close()
    return {"runs": len(runs), "train_runs": len(fit), "validation_runs": len(val), "held_out": len(held),
            "train_err_median": float(np.median(train_err)),
            "err_mean_history_median": float(np.median([q["err_mean_history"] for q in rows])),
            "samples": int(sum(windows(r)[0].shape[0] for r in fit)),
            "data_seconds": t_data, "train_seconds": t_train, "final_loss": losses[-1],
            "err_median": float(np.median(errs)), "err_max": float(errs.max()),
            "frac_within_5pct": float((errs <= 0.05).mean()),
            "speedup_median": float(np.median([q["speedup"] for q in rows])), "held": rows}


def study_aggregates(n_aggregates: int = 25, grain_counts=(50, 100), epochs: int = 400, rate: float = 2.0e3,
                     records: int = 64, h: float = 0.5e-3 / 12, seed: int = 0, device: int = 0, zeta: float = 0.5,
                     held: int = 3, val: int = 2, runs=None, p_confine: float = 2.0e6):
    """Every aggregate loaded along all eight paths from one shared pre-compression
    (``rve_aggregate``); grain counts cycle through ``grain_counts``.  The last
    ``held`` aggregates are held out with all their paths (no held-out run shares
    its packing with a training run), the ``val`` aggregates before them stop the
    training early, the rest train."""
    P = len(LOADING_PATHS)
    t0 = time.perf_counter()
    if runs is None:
        runs = []
        for a in range(n_aggregates):
            runs += rve_aggregate(grain_counts[a % len(grain_counts)], seed=seed + a, rate=rate, records=records,
                                  h=h, device=device, zeta=zeta, p_confine=p_confine)
    assert len(runs) == n_aggregates * P and n_aggregates > held + val
    t_data = time.perf_counter() - t0
    n_fit = n_aggregates - held - val
    fit, vr, hr = runs[:n_fit * P], runs[n_fit * P:(n_fit + val) * P], runs[(n_fit + val) * P:]
    return _fit_and_judge(runs, fit, vr, hr, fit + vr, t_data, epochs, seed, device, None)


def scaling_aggregates(runs, train_sizes, held: int = 3, val: int = 2, epochs: int = 400, seed: int = 0,
                       device: int = 0):
    """Held-out error against the number of training aggregates, on one fixed
    held-out set: the last ``held`` aggregates of ``runs`` (all their paths) are
    judged, the ``val`` before them stop the training early, and the network is
    trained on the first n aggregates for every n in ``train_sizes``.  Returns the
    reports and the least-squares slope of log(median error) on log(n)."""
    P = len(LOADING_PATHS)
    n_ag = len(runs) // P
    n_fit_max = n_ag - held - val
    vr = runs[n_fit_max * P:(n_fit_max + val) * P]
    hr = runs[(n_fit_max + val) * P:]
    reps = []
    for n in train_sizes:
        assert 0 < n <= n_fit_max
        fit = runs[:n * P]
        rep = _fit_and_judge(runs, fit, vr, hr, fit + vr, 0.0, epochs, seed, device, None)
        rep["train_aggregates"] = n
        reps.append(rep)
    x = np.log([r["train_aggregates"] for r in reps])
    y = np.log([r["err_median"] for r in reps])
    slope = float(np.polyfit(x, y, 1)[0]) if len(reps) > 1 else float("nan")
    return reps, slope


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="RVE bulk-stress surrogate study on one GPU")
    ap.add_argument("--runs-per-path", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--records", type=int, default=64)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--zeta", type=float, default=0.0, help="contact damping ratio of the RVE runs")
    ap.add_argument("--grains", type=int, nargs="+", default=[8, 12], help="grain counts, cycled over the runs")
    ap.add_argument("--out", default=None, help="also write the full report (per held-out run) to this file")
    ap.add_argument("--runs-file", default=None,
                    help="read the runs from this .npz if it exists, else generate them and write it")
    ap.add_argument("--aggregates", type=int, default=0,
                    help="> 0: this many aggregates, each loaded along all eight paths from one shared "
                         "pre-compression; whole aggregates held out (--held) and used for early stopping (--val)")
    ap.add_argument("--h", type=float, default=None, help="lattice spacing of the grains, m")
    ap.add_argument("--p-confine", type=float, default=2.0e6,
                    help="confining pressure that ends the isotropic pre-compression, Pa")
    ap.add_argument("--held", type=int, default=3)
    ap.add_argument("--val", type=int, default=2)
    ap.add_argument("--train-sizes", type=int, nargs="+", default=None,
                    help="with --aggregates: train on the first n aggregates for each n, one fixed held-out set")
    ap.add_argument("--twins", type=int, default=0,
                    help="measure the history spread under an invisible perturbation on this many aggregates")
    ap.add_argument("--twin-eps", type=float, nargs="+", default=[0.0, 1e-9, 1e-6],
                    help="node displacements of the twin runs, in units of h")
    ap.add_argument("--generate-only", action="store_true",
                    help="with --aggregates and --runs-file: extend the runs file and stop")
    a = ap.parse_args()
    import os
    if a.twins > 0:
        h = a.h if a.h is not None else 0.5e-3 / 12
        recs = []
        for ag in range(a.twins):
            for r in twin_spread(a.grains[ag % len(a.grains)], seed=a.seed + ag, eps=tuple(a.twin_eps),
                                 records=a.records, h=h, zeta=a.zeta, p_confine=a.p_confine):
                recs.append(dict(r, aggregate=ag, grains=a.grains[ag % len(a.grains)]))
                print(json.dumps(recs[-1]), flush=True)
        summary = {str(e): {"median": float(np.median([r["spread"] for r in recs if r["eps"] == e])),
                            "max": float(np.max([r["spread"] for r in recs if r["eps"] == e])),
                            "identical": int(sum(r["identical"] for r in recs if r["eps"] == e))}
                   for e in a.twin_eps}
        if a.out:
            with open(a.out, "w") as f:
                json.dump({"runs": recs, "summary": summary}, f, indent=1)
        print(json.dumps(summary))
        raise SystemExit(0)
    if a.aggregates > 0:
        h = a.h if a.h is not None else 0.5e-3 / 12
        P = len(LOADING_PATHS)
        # a runs file is extended aggregate by aggregate, so a cut-off job resumes
        runs = load_runs(a.runs_file) if a.runs_file and os.path.exists(a.runs_file) else []
        for ag in range(len(runs) // P, a.aggregates):
            runs += rve_aggregate(a.grains[ag % len(a.grains)], seed=a.seed + ag, records=a.records, h=h,
                                  zeta=a.zeta, p_confine=a.p_confine)
            if a.runs_file:
                save_runs(a.runs_file, runs)
        if a.generate_only:
            print(json.dumps({"aggregates": len(runs) // P, "runs": len(runs)}))
            raise SystemExit(0)
        if a.train_sizes:
            reps, slope = scaling_aggregates(runs[:a.aggregates * P], a.train_sizes, held=a.held, val=a.val,
                                             epochs=a.epochs, seed=a.seed)
            out = {"slope_log_err_vs_log_n": slope,
                   "by_size": [{k: v for k, v in r.items() if k != "held"} for r in reps],
                   "held_by_size": [r["held"] for r in reps]}
            if a.out:
                with open(a.out, "w") as f:
                    json.dump(out, f, indent=1)
            print(json.dumps({"slope": slope, "sizes": [(r["train_aggregates"], r["err_median"], r["err_max"],
                                                          r["err_mean_history_median"]) for r in reps]}))
            raise SystemExit(0)
        rep = study_aggregates(a.aggregates, grain_counts=tuple(a.grains), epochs=a.epochs, records=a.records, h=h,
                               seed=a.seed, zeta=a.zeta, held=a.held, val=a.val, runs=runs[:a.aggregates * P],
                               p_confine=a.p_confine)
        if a.out:
            with open(a.out, "w") as f:
                json.dump(rep, f, indent=1)
        print(json.dumps({k: v for k, v in rep.items() if k != "held"}))
        raise SystemExit(0)
    runs = load_runs(a.runs_file) if a.runs_file and os.path.exists(a.runs_file) else None
    if runs is None and a.runs_file:
        runs = []
        for pi, path in enumerate(LOADING_PATHS):
            for r in range(a.runs_per_path):
                ng = a.grains[r % len(a.grains)]
                runs.append(rve_run(path, n_grains=ng, seed=a.seed + 1000 * pi + r, records=a.records, zeta=a.zeta))
        save_runs(a.runs_file, runs)
    rep = study(a.runs_per_path, grain_counts=tuple(a.grains), epochs=a.epochs, records=a.records, seed=a.seed,
                zeta=a.zeta, runs=runs)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rep, f, indent=1)
    print(json.dumps({k: v for k, v in rep.items() if k != "held"}))
