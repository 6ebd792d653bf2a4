"""Task-level runs: CE-MPPI against standard MPPI.

Synthetic unicycle scenes in the spirit of the paper's evaluation (Sec.
III-B): a static obstacle near the straight path to the goal and the same
exactly on it (Scenario 1), and an obstacle crossing the robot's path
(Scenario 2).  Many seeded episodes of each method run as one device-resident batch: every
replan's first control moves the robot through the planner's own model step
(`x_next` aliases `x0`), the obstacles follow recorded streams, and after the
episode the robot's path is checked against the true obstacles.  Standard
MPPI (Eq. 6-7 over all K) carries a collision penalty w[7] in its cost; CE-MPPI
prunes colliding rollouts instead (w[7] = 0).  Planner settings are the
paper's unicycle values (Table III: K, T, dt, lambda, sigma, input box, eps,
minPts); the scene geometry is ours (the paper does not give it).

    python -m paper_2607_06499_b300.scenarios --episodes 64 --steps 400

The approach study (`--study`) isolates the averaging of Eq. 7: one replan of
each method on the same perturbations while the robot drives straight at the
blocking disc.
"""
import argparse
import json
import math

import numpy as np

from . import workloads as W

GOAL_TOL = 0.3   # m: the goal counts as reached within this distance


def scene(kind: str, seed: int, n_steps: int) -> dict:
    """Obstacle streams and start / goal of one episode (seeded jitter)."""
    rng = np.random.default_rng(1000 + seed)
    start = np.array([0.0, rng.uniform(-0.15, 0.15), 0.0])
    goal = np.array([4.0, 0.0, 0.0])
    H = 5
    n_rows = n_steps + H
    dt = 0.03
    if kind == "static":
        # one disc on the straight path (within 2 cm of it): the rollouts split
        # to both sides, and their weighted average points at the disc
        c = np.array([[2.0, rng.uniform(-0.02, 0.02)]])
        r = np.array([0.35])
        obs = np.repeat(c[None], n_rows, axis=0)
    elif kind == "blocking":
        # the symmetric case: start, disc and goal exactly on one line, so
        # the free rollouts pass on both sides in equal measure
        start = np.array([0.0, 0.0, 0.0])
        c = np.array([[2.0, 0.0]])
        r = np.array([0.35])
        obs = np.repeat(c[None], n_rows, axis=0)
    elif kind == "crossing":
        # one disc crossing the path from below, meeting the robot near x = 2
        v = rng.uniform(0.45, 0.6)
        c0 = np.array([2.0 + rng.uniform(-0.2, 0.2), -2.0])
        tt = np.arange(n_rows)[:, None] * dt
        obs = (c0[None] + tt * np.array([0.0, v])[None])[:, None, :]
        r = np.array([0.3])
    else:
        raise KeyError(kind)
    return dict(start=start, goal=goal, obs=np.asarray(obs, float), radius=r, dt=dt, H=H)


def planner_cfg(goal, mppi: bool, seed: int, lam: float = 0.7) -> dict:
    cfg = W.base_params(W.DYN_UNICYCLE, 300, 30, 0.03, lam=lam, sigma=(0.4, 3.0),
                        u_min=(-0.8, -7.0), u_max=(0.8, 7.0), goal=tuple(goal),
                        w=(10, 10, 0, 50, 50, 50), eps=0.3, min_pts=5, seed=seed,
                        robot_radius=0.1, mppi_only=int(mppi))
    if mppi:
        cfg["w"] = list(cfg["w"]) + [0.0, 1e4]   # w[7]: collision penalty
    return cfg


def run(kind: str, mppi: bool, episodes: int, steps: int, device: str = "cuda") -> dict:
    """Run `episodes` seeded episodes of one method on one scene kind."""
    import torch
    from . import Batch, Planner

    scs = [scene(kind, e, steps) for e in range(episodes)]
    pls, reqs = [], []
    for e, sc in enumerate(scs):
        cfg = planner_cfg(sc["goal"], mppi, seed=e)
        pl = Planner(cfg, n_obs_max=sc["radius"].shape[0])
        pl.set_nominal(np.zeros((cfg["T"], 2)))
        n_o = sc["radius"].shape[0]
        rq = dict(x0=torch.tensor(sc["start"], dtype=torch.float32, device=device),
                  hist=torch.tensor(sc["obs"], dtype=torch.float32, device=device).contiguous(),
                  radius=torch.tensor(sc["radius"], dtype=torch.float32, device=device),
                  obs_step=n_o * 2)
        rq["x_next"] = rq["x0"]
        pls.append(pl)
        reqs.append(rq)
    b = Batch(pls, reqs, use_graph=True)
    path = torch.zeros((steps + 1, episodes, 3), dtype=torch.float32, device=device)
    xs = [r["x0"] for r in reqs]
    path[0] = torch.stack(xs)
    for t in range(steps):
        b.run()
        path[t + 1] = torch.stack(xs)
    torch.cuda.synchronize()
    path = path.cpu().numpy()
    b.close()
    for pl in pls:
        pl.close()
    return evaluate(scs, path)


def evaluate(scs: list, path: np.ndarray) -> dict:
    """Collision (robot disc against the true obstacles at each step), goal
    arrival before any collision, time to goal, least clearance."""
    steps = path.shape[0] - 1
    out = dict(episodes=len(scs), collided=0, reached=0, time_to_goal=[], min_clear=[])
    for e, sc in enumerate(scs):
        H = sc["H"]
        p = path[:, e, :2]
        # replan t reads observation rows t .. t+H-1; the obstacle at the time
        # of state t+1 is row t+H (one obs_dt later than the newest observation)
        o = sc["obs"][H - 1:H - 1 + steps + 1]
        d = np.linalg.norm(p[:, None, :] - o, axis=2) - (sc["radius"][None] + 0.1)
        clear = d.min(axis=1)
        hit = np.flatnonzero(clear < 0.0)
        first_hit = hit[0] if hit.size else steps + 1
        at_goal = np.flatnonzero(np.linalg.norm(p - sc["goal"][None, :2], axis=1) < GOAL_TOL)
        first_goal = at_goal[0] if at_goal.size else steps + 1
        out["collided"] += int(hit.size > 0)
        if first_goal <= steps and first_goal < first_hit:
            out["reached"] += 1
            out["time_to_goal"].append(float(first_goal * sc["dt"]))
        out["min_clear"].append(float(clear.min()))
    out["time_to_goal_median_s"] = (float(np.median(out["time_to_goal"]))
                                    if out["time_to_goal"] else None)
    out["min_clear_median_m"] = float(np.median(out["min_clear"]))
    del out["time_to_goal"], out["min_clear"]
    return out


def nominal_path(x0, U, dt: float) -> np.ndarray:
    """States x_1..x_T of the unicycle (Eq. 21) driven by the nominal U."""
    x = np.array(x0, dtype=np.float64)
    out = []
    for u in np.asarray(U, dtype=np.float64):
        x = x + dt * np.array([u[0] * math.cos(x[2]), u[0] * math.sin(x[2]), u[1]])
        out.append(x.copy())
    return np.array(out)


def approach_study(seeds: int = 64, lams=(0.7, 5.0), Ks=(300, 2048), x_start: float = 1.1,
                   v: float = 0.8) -> dict:
    """The averaging-induced failure of Eq. 7 (Sec. I, Fig. 1; Sec. III-B,
    Scenario 1) on the symmetric blocking scene: the robot is on the line
    through the disc and the goal, 0.9 m before the disc's centre, driving
    straight at it at full speed (nominal v, omega = 0), so the straight
    rollouts hit the disc and the free ones pass on either side or stop short.
    For each seed, one CE-MPPI replan and one standard MPPI replan (collision
    penalty w[7]) from the same seed and replan counter -- the same
    perturbations, the same trajectories -- and each new nominal driven
    through the model: does its path meet the disc, and where does it end
    laterally."""
    from . import Planner
    sc = scene("blocking", 0, 8)
    c, rad, H = sc["obs"][0, 0], sc["radius"], sc["H"]
    x0 = np.array([x_start, 0.0, 0.0])
    out = {}
    for K in Ks:
        for lam in lams:
            res, ncl = {}, []
            for name, mppi in (("ce-mppi", False), ("mppi", True)):
                meets, lat, two = 0, [], 0
                for e in range(seeds):
                    cfg = planner_cfg(sc["goal"], mppi, seed=e, lam=lam)
                    cfg["K"] = K
                    pl = Planner(cfg, n_obs_max=1)
                    pl.set_nominal(np.tile([v, 0.0], (cfg["T"], 1)))
                    u, diag = pl.replan(x0, sc["obs"][:H], rad)
                    pl.close()
                    path = nominal_path(x0, u, sc["dt"])
                    cl = (np.linalg.norm(path[:, :2] - c[None], axis=1) - (rad[0] + 0.1)).min()
                    meets += int(cl < 0.0)
                    lat.append(abs(float(path[-1, 1])))
                    if not mppi:
                        ncl.append(diag["n_clusters"])
                res[name] = {"nominal_meets_disc": meets,
                             "median_abs_lateral_m": float(np.median(lat))}
            res["seeds"] = seeds
            res["ce_two_or_more_clusters"] = int(np.sum(np.array(ncl) >= 2))
            out[f"K={K}/lam={lam}"] = res
    return out


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--episodes", type=int, default=64)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--study", action="store_true",
                    help="the single-replan approach study instead of the episodes")
    ap.add_argument("--seeds", type=int, default=64, help="seeds of the study")
    args = ap.parse_args()
    if args.study:
        print(json.dumps(approach_study(args.seeds)))
        return
    res = {}
    for kind in ("static", "blocking", "crossing"):
        for name, mppi in (("ce-mppi", False), ("mppi", True)):
            res[f"{kind}/{name}"] = run(kind, mppi, args.episodes, args.steps)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
