"""Seeded synthetic workloads for the CE-MPPI replanning iteration.

This module is the one piece shared by the CUDA path's tests and benchmark and
the oracle's: it draws scenes, obstacle motion and parameter sets, and holds
none of the method's arithmetic (no dynamics, costs, kinematics, sampling of
the method's perturbations, or clustering).  All draws come from numpy's
counter-based Philox bit generator keyed by the scene seed, in a fixed order,
so a seed names the same scene on every machine.

The paper's own scenes are not specified, so these stand in for them:

* ``di_static``      2-D double integrator, 10 static discs in a 10x10 m field.
* ``di_blocked``     the same robot moving toward a disc on its path, so that
                     rollouts collide and split around it (exercises every stage).
* ``unicycle``       differential drive (Sec. III-A), 50 moving discs that
                     reflect off the walls of a 20x20 m field; K=16384, T=50.
* ``unicycle_paper`` the paper's simulation parameters (Table I: K=300, N=30,
                     dt=0.03, |v|<=0.8, |omega|<=7, lambda=0.7) with one static
                     disc straight ahead of the robot (Scenario-1-like).
* ``arm``            6-DoF UR5e-like arm, joint-velocity integrator, 20 moving
                     spheres in a 1.2 m cube in front of the base; K=4096, T=32.
* ``arm_paper``      the paper's real-robot parameters (Table III: K=50, N=12,
                     dt=0.1, |qdot|<=0.1, lambda=0.05, DBSCAN eps 0.3).
* ``batch_instance`` one instance of the uneven batch: unicycle with K
                     log-uniform in [512, 16384], T in [20, 60], 5-100 discs,
                     static or moving with probability 1/2.
"""
from __future__ import annotations

import math

import numpy as np

DYN_DI, DYN_UNICYCLE, DYN_ARM, DYN_ARM12 = 0, 1, 2, 3
DIMS = {DYN_DI: (4, 2, 2), DYN_UNICYCLE: (3, 2, 2), DYN_ARM: (6, 6, 3),
        DYN_ARM12: (12, 6, 3)}  # (n, m, p)

# Start pose of the arm (base turned to face +x) and the positions of its
# seven DH frame origins there, in metres; obstacles are kept clear of them.
ARM_Q0 = (math.pi, -math.pi / 2, math.pi / 2, -math.pi / 2, -math.pi / 2, 0.0)
_ARM_Q0_JOINTS = ((0.0, 0.0, 0.0), (0.0, 0.0, 0.1625), (0.0, 0.0, 0.5875),
                  (0.3922, 0.0, 0.5875), (0.3922, 0.1333, 0.5875),
                  (0.4919, 0.1333, 0.5875), (0.4919, 0.1333, 0.4879))


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, stream]))


def base_params(dyn: int, K: int, T: int, dt: float, *, lam: float, sigma, u_min, u_max,
                goal, w, eps: float, min_pts: int, seed: int, hist_len: int = 5,
                robot_radius: float = 0.0, obs_dt: float | None = None,
                norm_eps: float = 1e-6, v_static_thresh: float = 0.05,
                ref_mode: int = 0, check_j0: int = 0, noise_regen: int = 0,
                mppi_only: int = 0) -> dict:
    """A parameter set with the fields both the library and the oracle take."""
    return dict(dyn=dyn, K=int(K), T=int(T), dt=float(dt),
                obs_dt=float(dt if obs_dt is None else obs_dt), **{"lambda": float(lam)},
                dbscan_eps=float(eps), min_pts=int(min_pts),
                sigma=[float(s) for s in sigma], u_min=[float(s) for s in u_min],
                u_max=[float(s) for s in u_max], goal=[float(g) for g in goal],
                w=[float(x) for x in w], hist_len=int(hist_len),
                robot_radius=float(robot_radius), norm_eps=float(norm_eps),
                v_static_thresh=float(v_static_thresh), seed=int(seed),
                ref_mode=int(ref_mode), check_j0=int(check_j0), noise_regen=int(noise_regen),
                mppi_only=int(mppi_only))


def _place_discs(rng, n, field, r_lo, r_hi, keep_out, margin):
    """Disc radii U[r_lo, r_hi]; centres uniform inside the field, redrawn while
    within margin + radius of any keep-out point."""
    radius = rng.uniform(r_lo, r_hi, size=n)
    centres = np.zeros((n, len(field)))
    for o in range(n):
        for _ in range(1000):
            c = np.array([rng.uniform(lo + radius[o], hi - radius[o]) for lo, hi in field])
            if all(np.linalg.norm(c - np.asarray(q)) >= margin + radius[o] for q in keep_out):
                break
        centres[o] = c
    return centres, radius


def _move(rng, centres, radius, field, speed_lo, speed_hi, n_steps, step_dt, static):
    """Obstacle positions at n_steps observation times: constant speed in a
    uniformly random direction, reflecting off the field walls."""
    n, p = centres.shape
    speed = np.zeros(n) if static else rng.uniform(speed_lo, speed_hi, size=n)
    if p == 2:
        ang = rng.uniform(0.0, 2 * math.pi, size=n)
        direction = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    else:
        d = rng.normal(size=(n, 3))
        direction = d / np.linalg.norm(d, axis=1, keepdims=True)
    vel = direction * speed[:, None]
    lo = np.array([f[0] for f in field])[None, :] + radius[:, None]
    hi = np.array([f[1] for f in field])[None, :] - radius[:, None]
    pos = centres.copy()
    out = np.zeros((n_steps, n, p))
    for s in range(n_steps):
        out[s] = pos
        pos = pos + vel * step_dt
        over, under = pos > hi, pos < lo
        pos = np.where(over, 2 * hi - pos, pos)
        pos = np.where(under, 2 * lo - pos, pos)
        vel = np.where(over | under, -vel, vel)
    return out, vel


def make(name: str, seed: int = 0, n_replans: int = 1, **over) -> dict:
    """Build a named workload: returns dict(cfg, x0, U0, radius, obs), where
    obs[r : r + H] is the observation history (oldest first) of replan r and U0
    the initial nominal (a constant control u0 over the horizon)."""
    rng = _rng(seed)
    u0 = None
    if name in ("di_static", "di_blocked"):
        K, T = over.pop("K", 1024), over.pop("T", 30)
        cfg = base_params(DYN_DI, K, T, 0.05, lam=1.0, sigma=(0.5, 0.5), u_min=(-2, -2),
                          u_max=(2, 2), goal=(9.5, 9.5), w=(1.0, 0.01, 1.0), eps=0.3,
                          min_pts=10, seed=seed, **over)
        start, goal = (0.5, 0.5), (9.5, 9.5)
        centres, radius = _place_discs(rng, 10, [(0, 10), (0, 10)], 0.2, 0.5,
                                       [start, goal], 1.0)
        x0 = np.array([0.5, 0.5, 0.0, 0.0])
        if name == "di_blocked":
            # moving at 1.2 m/s along the diagonal toward a small disc 1.5 m ahead
            x0 = np.array([0.5, 0.5, 1.2 / math.sqrt(2), 1.2 / math.sqrt(2)])
            centres = np.vstack([centres, [[0.5 + 1.5 / math.sqrt(2)] * 2]])
            radius = np.append(radius, 0.08)
        obs, _ = _move(rng, centres, radius, [(0, 10), (0, 10)], 0, 0,
                       n_replans + cfg["hist_len"] - 1, cfg["obs_dt"], static=True)
    elif name in ("unicycle", "unicycle_blocked", "batch_instance"):
        static = False
        n_obs = over.pop("n_obs", 50)
        K, T = over.pop("K", 16384), over.pop("T", 50)
        if name == "batch_instance":
            K = int(round(math.exp(rng.uniform(math.log(512), math.log(16384)))))
            T = int(rng.integers(20, 61))
            n_obs = int(rng.integers(5, 101))
            static = bool(rng.uniform() < 0.5)
        sig = (0.5, 1.0) if name == "unicycle_blocked" else (0.5, 0.5)
        cfg = base_params(DYN_UNICYCLE, K, T, 0.05, lam=1.0, sigma=sig,
                          u_min=(0.0, -2.0), u_max=(2.0, 2.0),
                          goal=(19.0, 19.0, math.pi / 4), w=(10, 10, 0, 50, 50, 50),
                          eps=0.25, min_pts=20, seed=seed, **over)
        start = (1.0, 1.0)
        centres, radius = _place_discs(rng, n_obs, [(0, 20), (0, 20)], 0.2, 0.6,
                                       [start, (19.0, 19.0)], 1.0)
        x0 = np.array([1.0, 1.0, math.pi / 4])
        obs, _ = _move(rng, centres, radius, [(0, 20), (0, 20)], 0.0, 1.5,
                       n_replans + cfg["hist_len"] - 1, cfg["obs_dt"], static=static)
        if name == "unicycle_blocked":
            # one more disc 1.4 m ahead on the start heading, crossing at 0.2 m/s
            c = np.array([1.0 + 1.4 / math.sqrt(2), 1.0 + 1.4 / math.sqrt(2)])
            v = np.array([0.2 / math.sqrt(2), -0.2 / math.sqrt(2)])
            tt = np.arange(obs.shape[0])[:, None] * cfg["obs_dt"]
            track = c[None, :] + v[None, :] * (tt - tt[cfg["hist_len"] - 1])
            obs = np.concatenate([obs, track[:, None, :]], axis=1)
            radius = np.append(radius, 0.3)
            u0 = (1.0, 0.0)
    elif name == "unicycle_paper":
        lam = over.pop("lam", 0.7)
        cfg = base_params(DYN_UNICYCLE, over.pop("K", 300), over.pop("T", 30), 0.03, lam=lam,
                          sigma=(0.4, 3.0), u_min=(-0.8, -7.0), u_max=(0.8, 7.0),
                          goal=(4.0, 0.0, 0.0), w=(10, 10, 0, 50, 50, 50), eps=0.3,
                          min_pts=5, seed=seed, **over)
        centres = np.array([[0.75, 0.0]])
        radius = np.array([0.3])
        obs, _ = _move(rng, centres, radius, [(-5, 5), (-5, 5)], 0, 0,
                       n_replans + cfg["hist_len"] - 1, cfg["obs_dt"], static=True)
        x0 = np.array([0.0, 0.0, 0.0])
        u0 = (0.6, 0.0)  # already driving forward at 0.6 m/s
    elif name in ("arm", "arm_blocked", "arm_paper", "arm12", "arm12_blocked"):
        q0 = np.array(ARM_Q0)
        q_goal = q0 + rng.uniform(-1.0, 1.0, size=6)
        if name in ("arm12", "arm12_blocked"):
            # 12-D state (q, qdot) with joint-acceleration input, config-3 sizes
            cfg = base_params(DYN_ARM12, over.pop("K", 4096), over.pop("T", 32), 0.02, lam=1.0,
                              sigma=[1.0] * 6, u_min=[-3.0] * 6, u_max=[3.0] * 6,
                              goal=(), w=(10, 3, 1000), eps=0.2, min_pts=16, seed=seed,
                              robot_radius=0.06, **over)
            n_obs, speed_hi = 20, 0.3
        elif name in ("arm", "arm_blocked"):
            cfg = base_params(DYN_ARM, over.pop("K", 4096), over.pop("T", 32), 0.02, lam=1.0,
                              sigma=[0.3] * 6, u_min=[-1.0] * 6, u_max=[1.0] * 6,
                              goal=(), w=(10, 3, 1000), eps=0.2, min_pts=16, seed=seed,
                              robot_radius=0.06, **over)
            n_obs, speed_hi = 20, 0.3
        else:
            cfg = base_params(DYN_ARM, over.pop("K", 50), over.pop("T", 12), 0.1, lam=0.05,
                              sigma=[0.05] * 6, u_min=[-0.1] * 6, u_max=[0.1] * 6,
                              goal=(), w=(10, 3, 1000), eps=0.3, min_pts=5, seed=seed,
                              robot_radius=0.06, **over)
            n_obs, speed_hi = 4, 0.0
        cfg["goal_q"] = [float(v) for v in q_goal]
        field = [(0.2, 1.4), (-0.6, 0.6), (0.0, 1.2)]
        centres, radius = _place_discs(rng, n_obs, field, 0.05, 0.15, _ARM_Q0_JOINTS, 0.2)
        if name not in ("arm", "arm12"):
            # one static sphere just beside the end effector, 0.03 m clear of it
            ee = np.array(_ARM_Q0_JOINTS[6])
            centres = np.vstack([centres, ee + np.array([0.0, 0.0, -0.17])])
            radius = np.append(radius, 0.08)
        obs, _ = _move(rng, centres, radius, field, 0.0, speed_hi,
                       n_replans + cfg["hist_len"] - 1, cfg["obs_dt"],
                       static=(speed_hi == 0.0))
        if name in ("arm_blocked", "arm12_blocked"):
            obs[:, -1, :] = obs[0, -1, :]
        x0 = q0 if cfg["dyn"] == DYN_ARM else np.concatenate([q0, np.zeros(6)])
    else:
        raise KeyError(name)
    n, m, p = DIMS[cfg["dyn"]]
    U0 = np.zeros((cfg["T"], m)) if u0 is None else np.tile(np.asarray(u0, float), (cfg["T"], 1))
    return dict(cfg=cfg, x0=np.asarray(x0, float), U0=U0,
                radius=np.asarray(radius, float), obs=np.asarray(obs, float))


def history(scene: dict, r: int) -> np.ndarray:
    """Observation history [H][n_obs][p] (oldest first) for replan r."""
    H = scene["cfg"]["hist_len"]
    return np.ascontiguousarray(scene["obs"][r:r + H])


def batch(n_inst: int = 256, seed0: int = 0, n_replans: int = 1) -> list:
    """The uneven batch: instance i is ``batch_instance`` with seed seed0 + i."""
    return [make("batch_instance", seed0 + i, n_replans) for i in range(n_inst)]


def session_arrivals(rate_hz: float = 200.0, duration_s: float = 60.0, seed: int = 0):
    """Poisson session arrivals for the served loop: list of dicts with arrival
    time, lifetime U[2, 20] s and kind (70 % unicycle K in {1024, 4096, 16384},
    T=50; 30 % arm K in {2048, 4096}, T=32)."""
    rng = _rng(seed, stream=1)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return out
        if rng.uniform() < 0.7:
            kind, K = "unicycle", int(rng.choice([1024, 4096, 16384]))
        else:
            kind, K = "arm", int(rng.choice([2048, 4096]))
        out.append(dict(t=t, lifetime=float(rng.uniform(2.0, 20.0)), kind=kind, K=K,
                        seed=int(rng.integers(0, 2**31))))
