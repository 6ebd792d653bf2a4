"""Benchmark of the CE-MPPI replan on B300.

Workload: 2-D unicycle closed loop with moving obstacles -- K=16384 rollouts,
horizon T=50, dt=0.05, 50 discs (radius U[0.2,0.6], speed U[0,1.5] m/s,
reflecting off the walls of a 20x20 m field), DBSCAN eps 0.25 / minPts 20,
obstacle-motion selection; 16 seeded episodes (seeds 0..15).  Synthetic scenes
from paper_2607_06499_b300.workloads; observation streams and robot states are
resident on the device and the loop is closed on the device (x_next = x0).

One step = one replan of each of the 16 episodes, one launch per stage for all
of them, replayed from a captured CUDA graph.  value = rollout-steps/s
(16 * K * T per step).  The same replans run one instance at a time through the
blocking host-buffer call (the plain form) for comparison.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2607_06499_b300 import workloads as W  # noqa: E402

N_EPISODES = 16
WORKLOAD = dict(workload="ce-mppi replan, unicycle closed loop, moving obstacles", dyn="unicycle",
                K=16384, T=50, n_obs=50, episodes=N_EPISODES, dbscan_eps=0.25, min_pts=20,
                lam=1.0, sigma=[0.5, 0.5], l2="flushed between timed steps (256 MB write)")
METRIC = "CE-MPPI replan throughput (rollout-steps/s)"
UNIT = "rollout-steps/s"
STAGES = ("tracks", "rollout", "prune", "dbscan", "select", "update")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return pk, "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


def alu_peak_tflops(sm_count: int, mhz: float) -> float:
    """FP32 lanes x 2 flops per FMA x clock: 128 lanes per SM on sm_103."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def rollout_flops_per_step(n_obs: int) -> int:
    """Algorithmic FP32 operations of one unicycle rollout-step: 6 per circle
    test (2 sub, mul, fma counted 2, compare) and 60 for sampling clip, cost
    and the model step (Eq. 3-5, Eq. 21-23)."""
    return 6 * n_obs + 60


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for nm, v in zip(names, r[3:7]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(scenes, max_threads: int, budget_s: float = 20.0) -> dict:
    """The FP64 oracle on the host cores: independent replans of the workload's
    episodes (first replan each), one per thread, repeated while within budget."""
    import oracle
    nthr = max(1, min(max_threads, os.cpu_count() or 1))
    Ps = [oracle.make_params(s["cfg"]) for s in scenes]
    args = ([s["x0"] for s in scenes], [s["U0"] for s in scenes],
            [W.history(s, 0) for s in scenes], [s["radius"] for s in scenes])
    done, secs = 0, 0.0
    t0 = time.perf_counter()
    while True:
        n = min(nthr, len(scenes))
        _, dt = oracle.replan_many(Ps[:n], *[a[:n] for a in args], n_threads=n)
        done += n
        secs += dt
        if time.perf_counter() - t0 > budget_s or done >= len(scenes):
            break
    cfg = scenes[0]["cfg"]
    return {"value": done * cfg["K"] * cfg["T"] / secs, "unit": UNIT, "cores": min(nthr, len(scenes)),
            "kind": "oracle", "seconds": secs,
            "sample": f"{done} full replans (first replan of episodes 0..{done - 1}), one per host "
                      f"thread; FP64, O(|V|^2) DBSCAN"}


def run_reference(args) -> None:
    """Reference arm: the FP64 oracle timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    nthr = max(1, min(os.cpu_count() or 1, 8))
    scenes = [W.make("unicycle", seed=s) for s in range(nthr)]
    Ps = [oracle.make_params(s["cfg"]) for s in scenes]
    inputs = ([s["x0"] for s in scenes], [s["U0"] for s in scenes],
              [W.history(s, 0) for s in scenes], [s["radius"] for s in scenes])
    for _ in range(args.warmup):
        oracle.replan_many(Ps, *inputs, n_threads=nthr)
    t = []
    for _ in range(args.steps):
        _, dt = oracle.replan_many(Ps, *inputs, n_threads=nthr)
        t.append(dt)
    tot = float(np.sum(t))
    cfg = scenes[0]["cfg"]
    value = len(scenes) * cfg["K"] * cfg["T"] * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": WORKLOAD,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthr, "kind": "oracle",
                             "sample": f"each step: {nthr} full replans (episodes 0..{nthr - 1}), "
                                       f"one per host thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--plain-steps", type=int, default=10)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import paper_2607_06499_b300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(dev)

    total_replans = args.warmup + args.steps + args.plain_steps + args.steps + 8
    seeds = [rank * N_EPISODES + i for i in range(N_EPISODES)]
    scenes = [W.make("unicycle", seed=s, n_replans=total_replans) for s in seeds]
    cfg0 = scenes[0]["cfg"]
    K, T = cfg0["K"], cfg0["T"]
    planners, reqs = [], []
    for sc in scenes:
        pl = pkg.Planner(sc["cfg"], n_obs_max=sc["radius"].shape[0])
        pl.set_nominal(np.tile([1.0, 0.0], (T, 1)))
        n_obs = sc["radius"].shape[0]
        reqs.append(dict(
            x0=torch.tensor(sc["x0"], dtype=torch.float32, device=dev),
            hist=torch.tensor(sc["obs"], dtype=torch.float32, device=dev).contiguous(),
            radius=torch.tensor(sc["radius"], dtype=torch.float32, device=dev),
            u_out=torch.zeros((T, 2), dtype=torch.float32, device=dev),
            diag=torch.zeros(128, dtype=torch.uint8, device=dev), obs_step=n_obs * 2))
        reqs[-1]["x_next"] = reqs[-1]["x0"]
        planners.append(pl)
    batch = pkg.Batch(planners, reqs, stream=stream, use_graph=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        batch.run()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    clk = clocks.stop()
    tot_ms = float(step_ms.sum())
    if dist:
        t = torch.tensor([tot_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
        dist.barrier()
    units = world * N_EPISODES * K * T * args.steps
    value = units / (tot_ms / 1e3)

    # per-stage device times (stage-by-stage replans, same workload, L2 flushed)
    prof = {s: [] for s in STAGES}
    for i in range(args.steps):
        flush.fill_(float(i))
        for s, ms in batch.profile().items():
            prof[s].append(ms)
    stage_ms = {s: float(np.mean(v)) for s, v in prof.items()}
    roll_ms = stage_ms["rollout"]
    n_obs = scenes[0]["radius"].shape[0]
    flops = N_EPISODES * K * T * rollout_flops_per_step(n_obs)
    achieved = flops / (roll_ms * 1e-3) / 1e12
    pk, pk_kind = peaks()
    peak = alu_peak_tflops(props.multi_processor_count, pk.get("sm_max_mhz", 2032.0))

    # diagnostics of the last replan of each episode
    modes = []
    for r in reqs:
        d = np.frombuffer(r["diag"].cpu().numpy().tobytes()[:32], dtype=np.int32)
        modes.append(int(d[0]))
        assert d[7] == 0, f"device status {d[7]}"

    # end to end through the public API with host buffers: per step, the
    # observation windows go host -> device, the new nominals come back.
    H = cfg0["hist_len"]
    e2e_pl, e2e_req = [], []
    for sc in scenes:
        pl = pkg.Planner(sc["cfg"], n_obs_max=sc["radius"].shape[0])
        pl.set_nominal(np.tile([1.0, 0.0], (T, 1)))
        n_o = sc["radius"].shape[0]
        e2e_req.append(dict(
            x0=torch.tensor(sc["x0"], dtype=torch.float32, device=dev),
            hist=torch.zeros((H, n_o, 2), dtype=torch.float32, device=dev),
            radius=torch.tensor(sc["radius"], dtype=torch.float32, device=dev),
            u_out=torch.zeros((T, 2), dtype=torch.float32, device=dev)))
        e2e_req[-1]["x_next"] = e2e_req[-1]["x0"]
        e2e_pl.append(pl)
    e2e_batch = pkg.Batch(e2e_pl, e2e_req, stream=stream, use_graph=True)
    host_obs = [torch.tensor(sc["obs"], dtype=torch.float32).pin_memory() for sc in scenes]
    host_u = torch.zeros((N_EPISODES, T, 2), dtype=torch.float32).pin_memory()
    h2d = sum(r["hist"].numel() * 4 for r in e2e_req)
    d2h = host_u.numel() * 4

    def e2e_step(r):
        for i, q in enumerate(e2e_req):
            q["hist"].copy_(host_obs[i][r:r + H], non_blocking=True)
        e2e_batch.run()
        for i, q in enumerate(e2e_req):
            host_u[i].copy_(q["u_out"], non_blocking=True)
        stream.synchronize()

    for r in range(args.warmup):
        e2e_step(r)
    t0 = time.perf_counter()
    for r in range(args.steps):
        e2e_step(args.warmup + r)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * N_EPISODES * K * T * args.steps / e2e_s

    # plain form: one instance per launch chain, blocking host-buffer call
    plain_pl = [pkg.Planner(sc["cfg"], n_obs_max=sc["radius"].shape[0]) for sc in scenes]
    for pl in plain_pl:
        pl.set_nominal(np.tile([1.0, 0.0], (T, 1)))
    lat = []
    for r in range(args.plain_steps):
        for i, sc in enumerate(scenes):
            t1 = time.perf_counter()
            plain_pl[i].replan(sc["x0"], W.history(sc, r), sc["radius"])
            lat.append(time.perf_counter() - t1)
    lat = np.array(lat[N_EPISODES:]) * 1e3  # first round is warm-up
    plain = {"replans_per_s": 1e3 / float(lat.mean()), "p50_ms": float(np.percentile(lat, 50)),
             "p99_ms": float(np.percentile(lat, 99)),
             "rollout_steps_per_s": K * T * 1e3 / float(lat.mean())}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD, parallelism=f"replicas x{world}, episodes sharded by rank"),
        "replans_per_s": world * N_EPISODES * args.steps / (tot_ms / 1e3),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99)),
                       "note": "batched step: all 16 replans complete"},
        "plain": plain,
        "stage_ms": stage_ms,
        "modes_last_step": {pkg.MODES[m]: modes.count(m) for m in sorted(set(modes))},
        "roofline": {"kernel": "k_rollout2d<unicycle>", "bound": "alu", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "peak_kind": f"FP32 lanes x 2 x max SM clock ({pk_kind} clock)",
                     "flops_per_rollout_step": rollout_flops_per_step(n_obs)},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": 6 * args.steps,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        line["cpu_baseline"] = cpu_baseline(scenes, max_threads=N_EPISODES)
    if rank == 0:
        print(json.dumps(line), flush=True)
    for obj in [batch, e2e_batch] + planners + e2e_pl + plain_pl:
        obj.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
