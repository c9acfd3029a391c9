"""Training data, training and evaluation of the learned warm start.

The paper starts the first frame of a sequence from zero flows and names a
smarter first-frame initialisation as future work (Section 7). Here a small
convolutional network (sf_net in include/sf.h) predicts, from the four
coarsest-level images of a quadruple, the coarsest level's initial delta
fields; the plain hierarchy then runs as before from that start.

Workload (640 x 480, grid stride 8, four levels, Figure-2 weights): the
coarsest level is 80 x 60 pixels with an 8 x 10 warp grid.

* Data: quadruples of the seeded stereo videos (``scenes.SceneVideo``,
  rendered on the device by ``scenes_device``), each solved from a cold start
  by the plain method (3 Gauss-Newton x 20 PCG per level). The target is that
  solve's own coarsest-level total fields (the state the coarsest level
  reaches); the finest totals restricted to the coarsest grid (finest node
  (8i, 8j) for coarsest node (i, j), divided by 8) are kept as an
  alternative target.
* Training: mean squared error, Adam, cosine learning-rate decay; the GPU
  runs every step (sf_net_train_step).
* Evaluation: on held-out first frames, the final energy of the cold-start
  solve with the full schedule against warm-started solves with cheaper
  schedules (fewer Gauss-Newton steps per level). A schedule is accepted when
  every evaluation frame ends within 1e-4 relative of its cold-start energy.
* Time to energy: per frame, the cheapest schedule of a family (more or
  fewer Gauss-Newton steps per level) whose final energy reaches the cold
  start's within 1e-4, from the zero start, from the network's prediction,
  and from the prediction kept only where it lowers the coarsest level's
  energy (guarded); the Gauss-Newton cost and frames/s to get there.
"""

from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import scenes, scenes_device, sf

W0, H0, STRIDE, LEVELS = 640, 480, 8, 4
FULL = (3, 3, 3, 3)  # Gauss-Newton steps per level, finest first
PCG = 20
# cheaper schedules tried by the evaluation, finest first
SCHEDULES = ((3, 3, 3, 3), (3, 3, 3, 1), (3, 3, 3, 0), (3, 3, 2, 0), (2, 2, 2, 1), (2, 2, 2, 0), (2, 2, 1, 0),
             (2, 1, 1, 0), (1, 1, 1, 1), (1, 1, 1, 0))
ACCEPT_REL = 1e-4


def solver_params(gn=FULL, pcg: int = PCG, use_graph: int = 1) -> sf.Params:
    return sf.preset(sf.PRESET_FIG2, gn_iters=list(gn), pcg_iters=[pcg] * len(gn), use_graph=use_graph)


def schedule_cost(gn) -> float:
    """Relative cost of a schedule: Gauss-Newton steps weighted by level pixels."""
    return float(sum(g * 4.0 ** -l for l, g in enumerate(gn)))


def make_dataset(n_videos: int, frames_per_video: int, seed0: int, device="cuda", render_dtype=torch.float32):
    """Inputs [N, 4, 60, 80] and two targets [N, 6, 8, 10] on the device: the
    cold solve's finest totals restricted to the coarsest grid, and the cold
    solve's own coarsest-level totals."""
    solver = sf.Solver(W0, H0, STRIDE, LEVELS, solver_params())
    xs, yf, yc = [], [], []
    for v in range(n_videos):
        video = scenes.SceneVideo(W0, H0, frames_per_video, seed=seed0 + v)
        q = scenes_device.frames(video, frames_per_video, device, dtype=render_dtype)
        for f in range(frames_per_video):
            solver.reset()
            F = solver.solve(q[f])
            xs.append(sf.coarsest_images(solver, q[f]))
            yf.append(F[:, 0:57:8, 0:73:8] / 8.0)
            yc.append(solver.state(LEVELS - 1)[1])
    return torch.stack(xs), torch.stack(yf).contiguous(), torch.stack(yc).contiguous()


def init_params(seed: int) -> torch.Tensor:
    """He-normal weights and zero biases in the standard parameter layout."""
    rng = np.random.default_rng(seed)
    chans = ((4, 32), (32, 64), (64, 64), (64, 64), (64, 32), (32, 6))
    parts = []
    for cin, cout in chans:
        parts.append(rng.standard_normal(cout * cin * 9) * math.sqrt(2.0 / (9 * cin)))
        parts.append(np.zeros(cout))
    return torch.from_numpy(np.concatenate(parts).astype(np.float32)).cuda()


def train(net: sf.Net, x: torch.Tensor, y: torch.Tensor, epochs: int, batch: int = 256, lr: float = 2e-3,
          lr_min: float = 2e-5, seed: int = 0):
    """Trains on (x, y) with Adam and cosine decay; returns the mean loss per epoch."""
    n = x.shape[0]
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    steps = epochs * max(1, n // batch)
    step = 0
    loss = torch.zeros(1, device="cuda")
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        tot = torch.zeros(1, device="cuda")
        nb = 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            rate = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * step / max(1, steps)))
            net.train_step(x[idx].contiguous(), y[idx].contiguous(), rate, loss)
            tot += loss
            nb += 1
            step += 1
        hist.append(float(tot.item() / max(1, nb)))
    net.status()
    return hist


def evaluate(net: sf.Net | None, n_videos: int, seed0: int, schedules=SCHEDULES, device="cuda"):
    """Final energies of the first frames of n_videos held-out videos: cold start
    with the full schedule, warm start with each schedule."""
    quads = [scenes_device.frames(scenes.SceneVideo(W0, H0, 1, seed=seed0 + v), 1, device)[0] for v in range(n_videos)]
    cold = sf.Solver(W0, H0, STRIDE, LEVELS, solver_params())
    e_cold = []
    for q in quads:
        cold.reset()
        cold.solve(q)
        e_cold.append(cold.stats().energy)
    e_cold = np.array(e_cold)
    res = {"cold_energy": e_cold.tolist(), "schedules": []}
    for gn in schedules:
        s = sf.Solver(W0, H0, STRIDE, LEVELS, solver_params(gn))
        e_warm, e_zero = [], []
        for q in quads:
            s.reset()
            if net is not None:
                net.warm_start(s, q)
            s.solve(q)
            e_warm.append(s.stats().energy)
            s.reset()
            s.solve(q)
            e_zero.append(s.stats().energy)
        e_warm, e_zero = np.array(e_warm), np.array(e_zero)
        rel_w = (e_warm - e_cold) / e_cold
        rel_z = (e_zero - e_cold) / e_cold
        res["schedules"].append({"gn": list(gn), "cost": schedule_cost(gn),
                                 "warm_max_rel": float(rel_w.max()), "warm_mean_rel": float(rel_w.mean()),
                                 "cold_max_rel": float(rel_z.max()), "cold_mean_rel": float(rel_z.mean()),
                                 "warm_accepted": bool(np.all(rel_w <= ACCEPT_REL)),
                                 "cold_accepted": bool(np.all(rel_z <= ACCEPT_REL))})
        s.close()
    acc_w = [r for r in res["schedules"] if r["warm_accepted"]]
    acc_z = [r for r in res["schedules"] if r["cold_accepted"]]
    res["cheapest_warm"] = min(acc_w, key=lambda r: r["cost"])["gn"] if acc_w else None
    res["cheapest_cold"] = min(acc_z, key=lambda r: r["cost"])["gn"] if acc_z else None
    return res


# the schedule family of the time-to-energy evaluation, cheapest first by cost
# (Gauss-Newton steps weighted by level pixels): the schedules above and ones
# with more steps on the finest level
TTE_SCHEDULES = tuple(sorted(set(SCHEDULES) | {(g0,) + tail for g0 in range(4, 9)
                                               for tail in ((3, 3, 3), (2, 2, 1), (1, 1, 0), (2, 2, 0))},
                             key=schedule_cost))


def guarded_init(net: sf.Net, solver: sf.Solver, q: torch.Tensor) -> bool:
    """Predicts the coarsest initial delta and keeps it only where it lowers
    the coarsest level's energy against the zero start (both with W taken at
    their own state and the feature weights of the zero start); returns
    whether the prediction was kept. The same safeguard as the step
    acceptance of the solve, applied to the start."""
    img = sf.coarsest_images(solver, q)  # also builds the context's pyramid
    pred = net.forward(img[None].contiguous())[0].contiguous()
    lc = solver.levels - 1
    _, _, nx, ny = solver.dims(lc)
    zero = torch.zeros((6, ny * nx), device="cuda", dtype=torch.float32)
    wf = solver.probe_feature_weights(lc, zero)
    e_pred = solver.probe_energy(lc, zero, pred.view(6, -1).contiguous(), wf)[0].item()
    e_zero = solver.probe_energy(lc, zero, zero, wf)[0].item()
    if e_pred < e_zero:
        solver.set_init(pred.view(6, -1).contiguous())
        return True
    return False


def evaluate_time_to_energy(net: sf.Net, n_videos: int, seed0: int, schedules=TTE_SCHEDULES, device="cuda",
                            rel=ACCEPT_REL):
    """The spec evaluation of the warm start: on the first frames of
    n_videos held-out videos, E_cold is the final energy of the cold start
    with the full schedule; for each start (zero, network, guarded network)
    and frame, the cheapest schedule of the family whose final energy is
    within `rel` of E_cold (E <= (1 + rel) E_cold), its cost (Gauss-Newton
    steps weighted by level pixels) and its solve time (CUDA events, the
    network's pass included). A frame that no schedule brings there counts as
    not reached."""
    quads = [scenes_device.frames(scenes.SceneVideo(W0, H0, 1, seed=seed0 + v), 1, device)[0] for v in range(n_videos)]
    solvers = {gn: sf.Solver(W0, H0, STRIDE, LEVELS, solver_params(gn)) for gn in set(schedules) | {FULL}}

    def run(gn, q, start):
        s = solvers[gn]
        s.reset()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        if start == "warm":
            net.warm_start(s, q)
        elif start == "guarded":
            guarded_init(net, s, q)
        s.solve(q)
        b.record()
        b.synchronize()
        return s.stats().energy, a.elapsed_time(b)

    for q in quads[:2]:  # warm-up (graph capture of every schedule)
        for gn in solvers:
            run(gn, q, "zero")
    e_cold = [run(FULL, q, "zero")[0] for q in quads]
    out = {"frames": n_videos, "bar": f"E <= (1 + {rel:g}) E_cold, E_cold the cold start with {list(FULL)}",
           "family": [list(gn) for gn in schedules], "cold_full_cost": schedule_cost(FULL), "starts": {}}
    for start in ("zero", "warm", "guarded"):
        costs, times, reached, picks = [], [], 0, []
        for q, ec in zip(quads, e_cold):
            pick = None
            for gn in schedules:
                e, ms = run(gn, q, start)
                if e <= (1.0 + rel) * ec:
                    pick = (gn, ms)
                    break
            if pick is not None:
                reached += 1
                costs.append(schedule_cost(pick[0]))
                times.append(pick[1])
                picks.append(list(pick[0]))
            else:
                picks.append(None)
        out["starts"][start] = {
            "reached": reached, "mean_cost": float(np.mean(costs)) if costs else None,
            "frames_per_s_to_reach": len(times) * 1e3 / float(np.sum(times)) if times else None,
            "schedules": picks}
    for s in solvers.values():
        s.close()
    z, w = out["starts"]["zero"], out["starts"]["warm"]
    out["warm_accepted"] = bool(w["reached"] == n_videos and z["mean_cost"] is not None and
                                w["mean_cost"] is not None and w["mean_cost"] < z["mean_cost"])
    return out


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--videos", type=int, default=2000)
    t.add_argument("--frames", type=int, default=10)
    t.add_argument("--epochs", type=int, default=60)
    t.add_argument("--seed", type=int, default=20000)
    t.add_argument("--out", required=True)
    t.add_argument("--eval-videos", type=int, default=32)
    t.add_argument("--target", choices=("coarse", "fine"), default="coarse")
    a = ap.parse_args(argv)
    if a.cmd == "train":
        t0 = time.time()
        x, yf, yc = make_dataset(a.videos, a.frames, a.seed)
        y = yc if a.target == "coarse" else yf
        t1 = time.time()
        net = sf.Net(max_batch=256)
        net.set_params(init_params(a.seed))
        hist = train(net, x, y, a.epochs)
        t2 = time.time()
        p = net.get_params().cpu().numpy()
        ev = evaluate(net, a.eval_videos, seed0=900000)
        t3 = time.time()
        info = {"samples": int(x.shape[0]), "videos": a.videos, "frames_per_video": a.frames, "seed": a.seed,
                "target": a.target, "epochs": a.epochs, "data_s": t1 - t0, "train_s": t2 - t1, "eval_s": t3 - t2,
                "loss_first": hist[0], "loss_last": hist[-1], "eval": ev}
        np.savez(a.out, params=p, loss=np.array(hist), info=json.dumps(info))
        print(json.dumps(info))


if __name__ == "__main__":
    main()
