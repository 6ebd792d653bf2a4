"""Benchmark of the CE-MPPI replan on B300.

Workload: 2-D unicycle closed loop with moving obstacles -- K=16384 rollouts,
horizon T=50, dt=0.05, 50 discs (radius U[0.2,0.6], speed U[0,1.5] m/s,
reflecting off the walls of a 20x20 m field), DBSCAN eps 0.25 / minPts 20,
obstacle-motion selection; 16 seeded episodes (seeds 0..15).  Synthetic scenes
from paper_2607_06499_b300.workloads; observation streams and robot states are
resident on the device and the loop is closed on the device (x_next = x0).

One step = one replan of each of the 16 episodes, one launch per stage for all
of them, replayed from a captured CUDA graph; an episode is 200 closed-loop
replans and restarts (untimed) after that.  value = rollout-steps/s
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
# Other workloads (--workload): the 6-DoF arm (K=4096, T=32, 20 moving spheres,
# 500-replan episodes) and the uneven batch (256 unicycle instances, K
# log-uniform in [512, 16384], T in [20, 60], 5-100 discs, 50 replans each).
WORKLOADS = {
    "unicycle": dict(scene="unicycle", n=N_EPISODES, episode=200, u_init=(1.0, 0.0),
                     config=WORKLOAD),
    "arm": dict(scene="arm", n=N_EPISODES, episode=500, u_init=None,
                config=dict(workload="ce-mppi replan, 6-DoF arm closed loop, moving spheres",
                            dyn="arm", K=4096, T=32, n_obs=20, episodes=N_EPISODES,
                            dbscan_eps=0.2, min_pts=16, lam=1.0, sigma=[0.3] * 6,
                            l2="flushed between timed steps (256 MB write)")),
    "arm12": dict(scene="arm12", n=N_EPISODES, episode=500, u_init=None,
                  config=dict(workload="ce-mppi replan, 12-D arm (joint accelerations) closed loop, "
                                       "moving spheres",
                              dyn="arm12", K=4096, T=32, n_obs=20, episodes=N_EPISODES,
                              dbscan_eps=0.2, min_pts=16, lam=1.0, sigma=[1.0] * 6,
                              l2="flushed between timed steps (256 MB write)")),
    "batch": dict(scene="batch_instance", n=256, episode=50, u_init=(1.0, 0.0),
                  config=dict(workload="ce-mppi replan, 256 uneven unicycle instances",
                              dyn="unicycle", K="log-uniform [512, 16384]", T="[20, 60]",
                              n_obs="[5, 100]", instances=256, static_fraction=0.5,
                              l2="flushed between timed steps (256 MB write)")),
}
METRIC = "CE-MPPI replan throughput (rollout-steps/s)"
UNIT = "rollout-steps/s"
STAGES = ("tracks", "rollout", "prune", "dbscan", "select", "update")
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one rollout
# launch over the workload's instances, from one ncu capture of the current
# kernel on this workload; issue-slot use of the same capture.


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


# Algorithmic FP32 operations of a unicycle rollout: 6 per circle test (2 sub,
# mul, fma counted 2, compare) over the obstacle tests the track builder keeps,
# plus 60 per step for the clip, the cost and the model step (Eq. 3-5, 21-23).


class ClockSampler:
    """SM clock, utilisation and throttle reasons sampled through NVML every
    10 ms (nvidia-smi every 50 ms where NVML is unavailable), from start() to
    stop() -- the whole benchmark run, so that a short timed region still has
    samples around it.  The clock reported is the median over the samples that
    saw the GPU busy."""

    REASONS = (("hw_slowdown", "nvmlClocksEventReasonHwSlowdown"),
               ("hw_thermal_slowdown", "nvmlClocksEventReasonHwThermalSlowdown"),
               ("sw_thermal_slowdown", "nvmlClocksEventReasonSwThermalSlowdown"),
               ("sw_power_cap", "nvmlClocksEventReasonSwPowerCap"))

    def __init__(self, index: int, bus_id: str = ""):
        import threading
        self.sm, self.util, self.reasons, self.max = [], [], set(), None
        self.stop_ev = threading.Event()
        self.p = None
        self.thread = None
        self.nvml_error = None
        try:
            import pynvml as nv
            nv.nvmlInit()
            try:
                h = nv.nvmlDeviceGetHandleByPciBusId(bus_id) if bus_id else None
            except nv.NVMLError:
                h = None
            if h is None:
                h = nv.nvmlDeviceGetHandleByIndex(index)
            self.max = float(nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM))
            masks = [(nm, getattr(nv, attr)) for nm, attr in self.REASONS]

            def loop():
                while not self.stop_ev.is_set():
                    try:
                        self.sm.append(float(nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM)))
                        self.util.append(float(nv.nvmlDeviceGetUtilizationRates(h).gpu))
                        r = nv.nvmlDeviceGetCurrentClocksEventReasons(h)
                        for nm, mk in masks:
                            if r & mk:
                                self.reasons.add(nm)
                    except nv.NVMLError:
                        pass
                    self.stop_ev.wait(0.01)

            self.thread = threading.Thread(target=loop, daemon=True)
            self.thread.start()
            self.source = "nvml, 10 ms, whole run"
            return
        except Exception as e:   # (no NVML in this container: nvidia-smi instead)
            self.nvml_error = repr(e)[:120]
        self.source = "nvidia-smi, 50 ms, whole run"
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("clocks.sm,clocks.max.sm,utilization.gpu,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def _summary(self, sm, util, mx):
        busy = [c for c, u in zip(sm, util) if u > 0]
        use = busy if busy else sm
        out = {"sm_mhz": float(np.median(use)) if use else None, "sm_max_mhz": mx,
               "reasons": sorted(self.reasons), "samples": len(sm),
               "samples_busy": len(busy), "source": self.source}
        if self.nvml_error:
            out["nvml"] = self.nvml_error
        return out

    def stop(self) -> dict:
        if self.thread is not None:
            self.stop_ev.set()
            self.thread.join()
            return self._summary(self.sm, self.util, self.max)
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock source"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, util, mx = [], [], None
        names = [nm for nm, _ in self.REASONS]
        for r in rows:
            try:
                c, m, u = float(r[0]), float(r[1]), float(r[2])
                sm.append(c)
                util.append(u)
                mx = m
                for nm, v in zip(names, r[3:7]):
                    if v.strip().lower() == "active":
                        self.reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return self._summary(sm, util, mx)


def cpu_baseline(scenes, u_init, max_threads: int, budget_s: float = 10.0) -> dict:
    """The FP64 oracle on the host cores: independent replans of the workload's
    instances (first replan, the bench's initial nominal), one per thread, with
    successive replan counters, repeated while within the time budget."""
    import oracle
    nthr = max(1, min(max_threads, os.cpu_count() or 1))
    done, secs, rnd, units = 0, 0.0, 0, 0
    t0 = time.perf_counter()
    while True:
        batch = [scenes[(done + i) % len(scenes)] for i in range(nthr)]
        Ps = [oracle.make_params(s["cfg"], counter=rnd) for s in batch]
        _, dt = oracle.replan_many(Ps, [s["x0"] for s in batch], [u_init(s) for s in batch],
                                   [W.history(s, 0) for s in batch], [s["radius"] for s in batch],
                                   n_threads=nthr)
        done += nthr
        units += sum(s["cfg"]["K"] * s["cfg"]["T"] for s in batch)
        secs += dt
        rnd += 1
        if time.perf_counter() - t0 > budget_s:
            break
    # the latency of one replan on one host thread (comparable with the GPU's
    # plain form): the median of two
    sc = scenes[0]
    lat = []
    for r in range(2):
        P = oracle.make_params(sc["cfg"], counter=rnd + r)
        _, dt = oracle.replan_many([P], [sc["x0"]], [u_init(sc)], [W.history(sc, 0)],
                                   [sc["radius"]], n_threads=1)
        lat.append(dt)
    return {"value": units / secs, "unit": UNIT, "cores": nthr,
            "kind": "oracle", "seconds": secs,
            "replan_ms_one_thread": 1e3 * float(np.median(lat)),
            "sample": f"{done} full replans (first replan of the episodes, warm nominal, "
                      f"successive counters), {nthr} host threads; FP64, O(|V|^2) DBSCAN; "
                      f"plus two replans of episode 0 on one thread for the latency"}


def bench_config(wl_name: str, world: int, noise_regen: int) -> dict:
    """The workload description both arms print (identical for the same run)."""
    return dict(WORKLOADS[wl_name]["config"],
                parallelism=f"replicas x{world}, instances sharded by rank",
                noise_regen=noise_regen, closed_loop=True,
                episode_replans=WORKLOADS[wl_name]["episode"])


def run_reference(args) -> None:
    """Reference arm: the FP64 oracle, as it stands, timed on the host cores on
    the same closed-loop episodes as the GPU arm (rank 0 only): each step is
    one replan of every episode -- the oracle's own replans, state and shifted
    nominal carried from step to step -- run as one host thread per episode
    (up to the core count).  A step is seconds long, so the run is bounded:
    after the warm-up, steps are timed until --steps are done or about two
    minutes of oracle time have passed (the sample is stated)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl_name = args.workload if args.workload in WORKLOADS else "unicycle"
    wl = WORKLOADS[wl_name]
    regen = args.noise_regen if args.noise_regen >= 0 else (0 if wl_name in ("arm", "arm12") else 1)
    n_inst = wl["n"] if wl_name != "batch" else 16
    nthr = max(1, min(os.cpu_count() or 1, n_inst))
    episode = wl["episode"]
    scenes = [W.make(wl["scene"], seed=s, n_replans=episode + 8, noise_regen=regen)
              for s in shard_seeds(0, n_inst)]
    m = W.DIMS[scenes[0]["cfg"]["dyn"]][1]

    def u0(sc):
        T_ = sc["cfg"]["T"]
        return np.zeros((T_, m)) if wl["u_init"] is None else np.tile(wl["u_init"], (T_, 1))

    xs = [np.asarray(sc["x0"], float) for sc in scenes]
    Us = [u0(sc) for sc in scenes]
    units = sum(sc["cfg"]["K"] * sc["cfg"]["T"] for sc in scenes)

    def step(r):
        Ps = [oracle.make_params(sc["cfg"], counter=r) for sc in scenes]
        U_new, dt = oracle.replan_many(Ps, xs, Us, [W.history(sc, r) for sc in scenes],
                                       [sc["radius"] for sc in scenes], n_threads=nthr)
        for i, (P, sc) in enumerate(zip(Ps, scenes)):   # (closed loop, untimed)
            xs[i] = oracle.step(P, xs[i], U_new[i][0])
            Us[i] = oracle.shift(P, U_new[i])
        return dt

    r = 0
    for _ in range(args.warmup):
        step(r % episode)
        r += 1
    t, budget = [], 120.0
    while len(t) < args.steps and (not t or sum(t) < budget):
        t.append(step(r % episode))
        r += 1
    done = len(t)
    tot = float(np.sum(t))
    value = units * done / tot
    sample = (f"{done} of {args.steps} steps (each: one closed-loop replan of each of the "
              f"{n_inst} episodes, replans {args.warmup}..{args.warmup + done - 1}), "
              f"{nthr} host threads, FP64, O(|V|^2) DBSCAN" +
              ("" if done == args.steps else f"; stopped after {budget:.0f} s of oracle time"))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / done, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(wl_name, args.gpus, regen),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthr, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serve(pkg, seconds: float, budget_gb: float, seed: int = 0, rate_hz: float = 200.0,
              max_batch: int = 1024, n_streams: int = 3, warmup_s: float = 20.0) -> dict:
    """The served request loop: controller sessions arrive as a Poisson process
    (rate_hz), 70 % unicycle (K in {1024, 4096, 16384}, T=50, 50 discs) and 30 %
    arm (K in {2048, 4096}, T=32, 20 spheres); each asks for a replan every 20 ms
    for a lifetime U[2, 20] s.  Sessions are admitted by the server's
    device-memory budget.  Requests are submitted in real time (1 ms ticks);
    a session's request that is still queued when its next one arrives is
    replaced by the newer one.  The first warmup_s seconds (the concurrency
    ramping up: lifetimes reach 20 s) are not measured; the statistics are
    reset then and cover the next `seconds`.  Returns served throughput,
    latency and the concurrency seen."""
    total = warmup_s + seconds
    arrivals = W.session_arrivals(rate_hz, total, seed=seed)
    n_rep = int(20.0 / 0.02) + 8
    tmpl = {"unicycle": [W.make("unicycle", seed=100 + i, n_replans=n_rep) for i in range(8)],
            "arm": [W.make("arm", seed=200 + i, n_replans=n_rep) for i in range(8)]}
    obs = {k: np.stack([t["obs"] for t in v]).astype(np.float32) for k, v in tmpl.items()}
    rad = {k: np.stack([t["radius"] for t in v]).astype(np.float32) for k, v in tmpl.items()}
    x0s = {k: np.stack([t["x0"] for t in v]).astype(np.float32) for k, v in tmpl.items()}
    H = 5
    srv = pkg.Server(mem_budget_bytes=int(budget_gb * (1 << 30)), max_sessions=4096,
                     max_batch=max_batch, n_streams=n_streams)
    active = {}   # sid -> [kind, template, t_start, t_end, next_due, K, T]
    rejected = opened = 0
    submitted = {"unicycle": 0, "arm": 0}
    steps_sub = 0.0
    conc = []
    nxt = 0
    measuring = warmup_s <= 0
    t0 = time.perf_counter()
    t_meas = t0
    while True:
        t = time.perf_counter() - t0
        if t >= total:
            break
        if not measuring and t >= warmup_s:
            srv.stats(reset=True)
            submitted = {"unicycle": 0, "arm": 0}
            steps_sub = 0.0
            rejected = opened = 0
            measuring = True
            t_meas = time.perf_counter()
        while nxt < len(arrivals) and arrivals[nxt]["t"] <= t:
            a = arrivals[nxt]
            nxt += 1
            tid = a["seed"] % 8
            cfg = dict(tmpl[a["kind"]][tid]["cfg"])
            cfg["K"] = a["K"]
            sid = srv.open(cfg, int(rad[a["kind"]].shape[1]))
            if sid is None:
                rejected += 1
                continue
            opened += 1
            active[sid] = [a["kind"], tid, t, t + a["lifetime"], t, cfg["K"], cfg["T"]]
        for sid in [s_ for s_, v in active.items() if v[3] <= t]:
            srv.close_session(sid)
            del active[sid]
        if measuring:
            conc.append(len(active))
        for kind in ("unicycle", "arm"):
            due = [s_ for s_, v in active.items() if v[0] == kind and v[4] <= t]
            if not due:
                continue
            tids = np.array([active[s_][1] for s_ in due])
            r = np.array([int((t - active[s_][2]) / 0.02) % (n_rep - 8) for s_ in due])
            win = obs[kind][tids[:, None], r[:, None] + np.arange(H)[None, :]]
            srv.submit_many(np.array(due, np.int32), x0s[kind][tids], win, rad[kind][tids],
                            np.full(len(due), rad[kind].shape[1], np.int32))
            submitted[kind] += len(due)
            for s_ in due:
                active[s_][4] += 0.02
                steps_sub += active[s_][5] * active[s_][6]
        time.sleep(max(0.0, 0.001 - ((time.perf_counter() - t0) - t)))
    st = srv.stats()
    elapsed = time.perf_counter() - t_meas
    for sid in list(active):
        srv.close_session(sid)
    srv.close()
    n_sub = sum(submitted.values())
    frac_served = st["replans"] / max(1, n_sub)
    return {"seconds": elapsed, "warmup_s": warmup_s, "sessions_opened": opened,
            "sessions_rejected": rejected, "sessions_concurrent_mean": float(np.mean(conc)) if conc else 0.0,
            "sessions_concurrent_peak": int(max(conc)) if conc else 0,
            "requests_submitted": n_sub, "replans_served": st["replans"],
            "superseded": st["superseded"], "replans_per_s": st["replans"] / elapsed,
            "rollout_steps_per_s": steps_sub * frac_served / elapsed,
            "p50_ms": 1e3 * st["p50_latency_s"], "p99_ms": 1e3 * st["p99_latency_s"],
            "mean_batch": st["mean_batch"], "budget_gb": budget_gb, "arrival_rate_hz": rate_hz,
            "max_batch": max_batch, "n_streams": n_streams}


STAMP_PHASES = ("cells and per-CTA counts", "occupied cells, offsets, cursors",
                "scatter into cell order, cell boxes", "core flags", "core boxes",
                "cell unions", "components, ids, core labels", "border points")
# the angle-bucket DBSCAN of 2-D features (stamp 15 = 1)
STAMP_PHASES_ANG = ("angle buckets, counts, radius range", "totals, scan, scatter",
                    "core flags", "runs, boundaries, components, ids", "labels")


def stage_stamps(planners, replay, restart, n_steps: int, episode: int) -> dict:
    """SM clock stamps that the fused clustering kernel leaves per instance
    (thread 0 of rank 0 of its cluster): kernel start, end of the prune stage,
    the DBSCAN phases, end of the DBSCAN stage.  Mean and max cycles over the
    replans of n_steps steps (each step synchronised and the stamps read back;
    a replan that clustered contributes its DBSCAN phases); the episodes are
    restarted every `episode` steps, as in the timed loop."""
    import torch
    prune, dbs, phases, sel, dense, upd, whole = [], [], [], [], [], [], []
    phases_ang, dbs_ang = [], []
    last = [None] * len(planners)
    for s in range(n_steps):
        if s and s % episode == 0:
            restart()
        replay()
        torch.cuda.synchronize()
        for i, pl in enumerate(planners):
            c = pl.peek("DBCYC")
            if last[i] is not None and c[9] == last[i][9]:
                continue   # this instance did not replan in the step
            last[i] = c.copy()
            prune.append(c[10] - c[9])
            if c[14] > c[13] >= c[12] > c[11]:   # the selection and update stamps of this replan
                sel.append(c[12] - c[11])
                dense.append(c[13] - c[12])
                upd.append(c[14] - c[13])
                whole.append(c[14] - c[9])
            if c[0] > c[10] and c[11] > c[8]:   # clustered in this replan
                if c[15] == 1:
                    phases_ang.append(np.diff(c[0:6]))
                    dbs_ang.append(c[11] - c[10])
                else:
                    phases.append(np.diff(c[0:9]))
                dbs.append(c[11] - c[10])
    def mm(v):
        return [int(np.mean(v)), int(np.max(v))] if v else None

    out = {"replans": len(prune), "clustered": len(dbs), "prune": mm(prune), "dbscan": mm(dbs),
           "select_weights": mm(sel), "dense_update_sums": mm(dense),
           "update_shift": mm(upd), "kernel": mm(whole)}
    if phases:
        ph = np.array(phases)
        out["dbscan_phases"] = {n: [int(ph[:, k].mean()), int(ph[:, k].max())]
                                for k, n in enumerate(STAMP_PHASES)}
    if phases_ang:
        ph = np.array(phases_ang)
        out["dbscan_angular"] = len(dbs_ang)
        out["dbscan_angular_phases"] = {n: [int(ph[:, k].mean()), int(ph[:, k].max())]
                                        for k, n in enumerate(STAMP_PHASES_ANG)}
    return out


def plain_mix_latency(pkg, n_each: int = 20) -> dict:
    """Plain form on the served mix: each replan alone through the blocking
    host-buffer call (launch chain + stream sync per replan)."""
    lat, steps = [], 0
    mix = [("unicycle", 1024, 0.7 / 3), ("unicycle", 4096, 0.7 / 3), ("unicycle", 16384, 0.7 / 3),
           ("arm", 2048, 0.15), ("arm", 4096, 0.15)]
    per_kind = {}
    for kind, K, w in mix:
        sc = W.make(kind, seed=300, K=K, n_replans=n_each + 2)
        pl = pkg.Planner(sc["cfg"], n_obs_max=sc["radius"].shape[0])
        ls = []
        for r in range(n_each + 2):
            t1 = time.perf_counter()
            pl.replan(sc["x0"], W.history(sc, r), sc["radius"])
            ls.append(time.perf_counter() - t1)
        pl.close()
        per_kind[(kind, K)] = (np.array(ls[2:]), w, K * sc["cfg"]["T"])
    # the mix-weighted latency distribution and capacity of one sequential loop
    samples = np.concatenate([np.repeat(v[0], int(round(v[1] * 100))) for v in per_kind.values()])
    mean_s = sum(v[1] * v[0].mean() for v in per_kind.values())
    steps = sum(v[1] * v[2] for v in per_kind.values())
    return {"p50_ms": 1e3 * float(np.percentile(samples, 50)),
            "p99_ms": 1e3 * float(np.percentile(samples, 99)),
            "replans_per_s": 1.0 / mean_s, "rollout_steps_per_s": steps / mean_s}


def shard_seeds(rank: int, n_per_rank: int) -> list:
    """Instances are independent: rank r replans its own n_per_rank seeded
    instances (weak scaling), with no exchange on the data path."""
    return [rank * n_per_rank + i for i in range(n_per_rank)]


def aggregate(tot_ms: float, units_per_rank: float, steps: int, world: int, dist=None):
    """Whole-job rate: the units of all ranks over the slowest rank's time
    (max-reduction of the timed region; the only collective)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([tot_ms], dtype=torch.float64)
        if dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    return world * units_per_rank * steps / (tot_ms / 1e3), tot_ms


# Algorithmic bytes per rollout of the clustering stages (the fused kernel,
# prune through the update): ~40 B read and written by pruning, DBSCAN and the
# selection (hit, S, p(x_T); the V / C_col lists, S in V order, z, g, cells,
# cell order, labels, weights), plus the update's least traffic when eps' is
# drawn again, (5 + 2p) 4 B per rollout (its records) -- 76 B for p = 2.
POST_BYTES_PER_ROLLOUT = {2: 40 + 36, 3: 40 + 44}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch from one
# ncu capture of the current build of the kernel, on the launch the line's
# timing covers: k_post over one pipelined half (8 instances), the rollout
# kernel over all 16 instances (the stage-by-stage profile launch).  None: not
# captured for the current build.
NCU_TRAFFIC = {("unicycle", "k_post"): 2398976, ("unicycle", "rollout"): 89600,
               ("arm", "k_post"): None, ("arm", "rollout"): 6018816,
               ("arm", "k_update"): 50703616}


def update_roofline(res: dict, m: int, hbm: float, pk_kind: str, wl_name: str):
    """The tiled update kernel against HBM where eps' is stored: |C*| T m 4 B
    read for the rows of nonzero weight + T m 8 B per instance, over the
    kernel's event time in the stage-by-stage replans (None with noise
    regeneration: the update then draws eps' again and reads no rows)."""
    if res["regen"]:
        return None
    TMs = res["Ts"] * m
    upd_bytes = float(np.sum(np.array(res["update_nnz"]) * TMs * 4 + TMs * 8))
    upd_ms = res["stage_ms"]["update"]
    upd_gbs = upd_bytes / (upd_ms * 1e-3) / 1e9
    return {"kernel": "k_update (tiled, eps' stored)", "bound": "hbm", "achieved": upd_gbs,
            "peak": hbm, "unit": "GB/s", "frac": upd_gbs / hbm,
            "traffic": NCU_TRAFFIC.get((wl_name, "k_update")),
            "peak_kind": f"copy bandwidth ({pk_kind})", "ms_per_launch": upd_ms,
            "algorithmic_bytes_per_launch": upd_bytes,
            "nonzero_weights_mean": float(np.mean(res["update_nnz"]))}


def early_tracks(args, wl_name: str) -> int:
    """The track kernels' place in the pipelined halves (see --early-tracks);
    by default both halves' early for the 2-D robots, the second half's for
    the arms (measured: arm 0.4451 / 0.4452 / 0.4564 ms per step for 0 / 1 /
    2)."""
    e = int(getattr(args, "early_tracks", -1))
    if e >= 0:
        return e
    return 1 if wl_name in ("arm", "arm12") else 2


def run_workload(pkg, torch, args, wl_name: str, dev, stream, rank: int, world: int, dist,
                 steps: int, warmup: int, flush, profile: bool):
    """Build the workload's device-resident closed-loop episodes, time `steps`
    pipelined steps (one replan of every episode each), and measure the
    stage times.  Returns the measurements and the objects to close."""
    wl = WORKLOADS[wl_name]
    regen = args.noise_regen if args.noise_regen >= 0 else (0 if wl_name in ("arm", "arm12") else 1)
    episode = args.episode_len if (args.episode_len > 0 and wl_name == args.workload) else wl["episode"]
    n_inst = wl["n"]
    seeds = shard_seeds(rank, n_inst)
    scenes = [W.make(wl["scene"], seed=s, n_replans=episode + 8, noise_regen=regen) for s in seeds]
    cfg0 = scenes[0]["cfg"]
    n_, m, p_dim = pkg.DIMS[cfg0["dyn"]]

    def u_init(sc):
        T_ = sc["cfg"]["T"]
        return np.zeros((T_, m)) if wl["u_init"] is None else np.tile(wl["u_init"], (T_, 1))

    units_per_step = sum(sc["cfg"]["K"] * sc["cfg"]["T"] for sc in scenes)
    planners, reqs = [], []
    for sc in scenes:
        pl = pkg.Planner(sc["cfg"], n_obs_max=sc["radius"].shape[0])
        n_obs = sc["radius"].shape[0]
        reqs.append(dict(
            x0=torch.tensor(sc["x0"], dtype=torch.float32, device=dev),
            hist=torch.tensor(sc["obs"], dtype=torch.float32, device=dev).contiguous(),
            radius=torch.tensor(sc["radius"], dtype=torch.float32, device=dev),
            u_out=torch.zeros((sc["cfg"]["T"], m), dtype=torch.float32, device=dev),
            diag=torch.zeros(128, dtype=torch.uint8, device=dev), obs_step=n_obs * p_dim))
        reqs[-1]["x_next"] = reqs[-1]["x0"]
        planners.append(pl)

    def reset_episodes():
        """Every episode back to its start: state, nominal, replan counter."""
        torch.cuda.synchronize()
        for sc, pl, rq in zip(scenes, planners, reqs):
            rq["x0"].copy_(torch.tensor(sc["x0"], dtype=torch.float32))
            pl.set_nominal(u_init(sc))
            pl.set_counter(0)
        torch.cuda.synchronize()

    reset_episodes()
    batch = pkg.Batch(planners, reqs, stream=stream, use_graph=True, n_branches=args.branches)
    # Software pipeline of two halves A, B of the episodes (independent
    # instances): one graph replay = [B clustering + update (replan s-1) |
    # A tracks + rollouts (s)], then [A clustering + update (s) | B tracks +
    # rollouts (s)] -- one replan of every episode per replay, each half's
    # latency-bound stages over the other half's rollouts.
    pipe = None
    if args.pipeline and n_inst >= 2:
        half = n_inst // 2
        bA = pkg.Batch(planners[:half], reqs[:half], stream=stream, use_graph=False)
        bB = pkg.Batch(planners[half:], reqs[half:], stream=stream, use_graph=False)
        bA.set_post_ctas(args.pipe_post_ctas)
        bB.set_post_ctas(args.pipe_post_ctas)
        side = torch.cuda.Stream()
        trk = torch.cuda.Stream()
        early = early_tracks(args, wl_name)
        graph = torch.cuda.CUDAGraph()
        # each half's rollouts wait for the other half's clustering kernel to
        # have begun on all its CTAs (launch-completion events), so that the
        # clustering CTAs, a whole SM each, are never left behind the rollouts
        started = [None, None]
        if getattr(args, "post_first", 1):
            started = [torch.cuda.Event(enable_timing=False) for _ in range(2)]
            for e in started:
                e.record(stream)   # (creates the event)
        torch.cuda.synchronize()
        with torch.cuda.graph(graph):
            main_s = torch.cuda.current_stream()
            side.wait_stream(main_s)
            if args.pipeline == 2:
                # the two halves as two chains joined only at the end: B's
                # clustering (s-1) then B's rollouts (s) on one stream, A's
                # rollouts (s) then A's clustering (s) on the other
                bB.run_part(1, main_s)
                bB.run_part(0, main_s)
                bA.run_part(0, side)
                bA.run_part(1, side)
            elif early:
                # B's track kernel of its next replan right after its
                # clustering + update, on a third stream, so that B's
                # rollouts do not start with it (early = 2: A's too, at the
                # end of each replay, its first in the prologue)
                bB.run_part(1, main_s, started=started[1])
                trk.wait_stream(main_s)
                bB.run_part(2, trk)                   # B's tracks (next replan)
                if started[1] is not None:
                    side.wait_event(started[1])
                bA.run_part(3 if early == 2 else 0, side)   # A's (tracks +) rollouts
                main_s.wait_stream(side)
                side.wait_stream(main_s)
                bA.run_part(1, main_s, started=started[0])
                if started[0] is not None:
                    side.wait_event(started[0])
                side.wait_stream(trk)                 # (B's tracks)
                if early == 2:
                    trk.wait_stream(main_s)
                    bA.run_part(2, trk)               # A's tracks (next replan)
                bB.run_part(3, side)                  # B's rollouts
                main_s.wait_stream(trk)
            else:
                bB.run_part(1, main_s, started=started[1])
                if started[1] is not None:
                    side.wait_event(started[1])
                bA.run_part(0, side)
                main_s.wait_stream(side)
                side.wait_stream(main_s)
                bA.run_part(1, main_s, started=started[0])
                if started[0] is not None:
                    side.wait_event(started[0])
                bB.run_part(0, side)
            main_s.wait_stream(side)
        torch.cuda.synchronize()
        pipe = (bA, bB, graph)

    def prologue():
        if pipe:
            pipe[1].run_part(0, stream)   # B's first tracks + rollouts, untimed
            if args.pipeline == 1 and early_tracks(args, wl_name) == 2:
                pipe[0].run_part(2, stream)   # A's first tracks

    def step():
        if pipe:
            pipe[2].replay()
        else:
            batch.run()

    reset_episodes()
    prologue()
    for _ in range(warmup):
        step()
    reset_episodes()
    prologue()
    if dist:
        dist.barrier()
    step_ms = []
    done = 0
    while done < steps:
        n = min(episode, steps - done)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n)]
        torch.cuda.synchronize()
        for i in range(n):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        step_ms += [x.elapsed_time(y) for x, y in ev]
        done += n
        if done < steps:
            reset_episodes()
            prologue()
    step_ms = np.array(step_ms)
    value, tot_ms = aggregate(float(step_ms.sum()), units_per_step, steps, world, dist)
    if dist:
        dist.barrier()
    modes = {}
    for r in reqs:
        d = np.frombuffer(r["diag"].cpu().numpy().tobytes()[:32], dtype=np.int32)
        modes[pkg.MODES.get(int(d[0]), int(d[0]))] = modes.get(pkg.MODES.get(int(d[0]), int(d[0])), 0) + 1
        assert d[7] == 0, f"device status {d[7]}"
    out = {"value": value, "tot_ms": tot_ms, "step_ms": step_ms,
           "replans_per_s": world * n_inst * steps / (tot_ms / 1e3),
           "units_per_step": units_per_step, "modes_last_step": modes, "regen": regen,
           "batch_config": pipe[0].config() if pipe else batch.config(),
           "n_inst": n_inst, "episode": episode, "pipelined": bool(pipe)}
    objs = [batch] + (list(pipe[:2]) if pipe else [])
    if not profile:
        return out, objs, planners, scenes, u_init, reset_episodes, step, prologue
    # per-stage device times: stage-by-stage replans over the start of the
    # episodes, L2 flushed before each; obstacle tests per rollout from diag
    reset_episodes()
    prof = {s_: [] for s_ in STAGES}
    tests = []
    for i in range(args.profile_steps):
        flush.fill_(float(i))
        for s_, ms in batch.profile().items():
            prof[s_].append(ms)
        for r in reqs:
            tests.append(int(np.frombuffer(r["diag"].cpu().numpy().tobytes()[72:76], np.int32)[0]))
    out["stage_ms"] = {s_: float(np.mean(v)) for s_, v in prof.items()}
    out["tests"] = np.array(tests, dtype=np.float64).reshape(args.profile_steps, len(reqs)).mean(0)
    # nonzero weights of each instance's last profiled replan: the rows of
    # eps' the update reads (the update kernel's algorithmic bytes)
    out["update_nnz"] = [int(np.count_nonzero(pl.peek("W"))) for pl in planners]
    # the fused clustering kernel as the pipeline launches it: one half's
    # instances, events around part 1 (prune + DBSCAN + selection + update)
    reset_episodes()
    bsrc = pipe[0] if pipe else batch
    post = []
    for i in range(args.profile_steps):
        flush.fill_(float(i))
        bsrc.run_part(0, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bsrc.run_part(1, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        post.append(e0.elapsed_time(e1))
    out["post_ms"] = float(np.mean(post))
    out["post_rollouts"] = sum(sc["cfg"]["K"] for sc in scenes[: (len(scenes) // 2 if pipe else len(scenes))])
    out["p_dim"] = p_dim
    out["Ks"] = np.array([sc["cfg"]["K"] for sc in scenes], dtype=np.float64)
    out["Ts"] = np.array([sc["cfg"]["T"] for sc in scenes], dtype=np.float64)
    return out, objs, planners, scenes, u_init, reset_episodes, step, prologue


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000,
                    help="timed steps (the 200-replan episodes restart every 200 steps)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the arm and uneven-batch workloads measured beside the main one")
    ap.add_argument("--plain-steps", type=int, default=10)
    ap.add_argument("--profile-steps", type=int, default=40)
    ap.add_argument("--extra-steps", type=int, default=100)
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--branches", type=int, default=0,
                    help="concurrent branches of the batch (0: autotuned)")
    ap.add_argument("--workload", default="unicycle", choices=sorted(WORKLOADS) + ["serve"])
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="measured length of the served run, after its warm-up (0: skip)")
    ap.add_argument("--serve-warmup", type=float, default=20.0,
                    help="unmeasured start of the served run (the concurrency ramps up)")
    ap.add_argument("--serve-budget-gb", type=float, default=16.0)
    ap.add_argument("--pipeline", type=int, default=1, choices=[0, 1, 2],
                    help="1: two halves of the episodes software-pipelined in one graph, "
                         "joined after each phase; 2: the same halves as two chains "
                         "joined once per step")
    ap.add_argument("--early-tracks", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="1: the second half's track kernel right after its clustering + "
                         "update, on a third stream, rather than at the head of its rollouts; "
                         "2: both halves' (the first's at the end of each replay; over whole "
                         "episodes 0.1341 against 0.1357 and 0.1386 ms per step, over their "
                         "first 20 replans 0.126 against 0.120); -1: 2 for the 2-D robots, "
                         "1 for the arms")
    ap.add_argument("--post-first", type=int, default=1, choices=[0, 1],
                    help="1: each half's tracks + rollouts wait on the other half's "
                         "clustering kernel having begun on all its CTAs")
    ap.add_argument("--pipe-post-ctas", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="clustering-kernel CTAs per instance in the pipelined halves "
                         "(0: from the occupancy, as if each half ran alone)")
    ap.add_argument("--stamps", type=int, default=0,
                    help="pipelined steps over which to read the clustering kernel's stage "
                         "clock stamps (0: off)")
    ap.add_argument("--episode-len", type=int, default=0,
                    help="closed-loop replans before the episodes restart (0: the workload's, "
                         "200 for the unicycle); longer episodes reach other states")
    ap.add_argument("--noise-regen", type=int, default=-1, choices=[-1, 0, 1],
                    help="1: perturbations not stored, drawn again by the update; "
                         "-1: 1 for 2-D robots (few nonzero weights), 0 for the arms")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import paper_2607_06499_b300 as pkg

    if args.workload == "serve":
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        served = run_serve(pkg, max(args.serve_seconds, 1.0), args.serve_budget_gb,
                           warmup_s=args.serve_warmup)
        plain = plain_mix_latency(pkg)
        line = {"metric": "CE-MPPI served replans (rollout-steps/s)",
                "value": served["rollout_steps_per_s"], "unit": UNIT, "n_gpus": 1,
                "steps": served["replans_served"], "warmup": 0, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "served request loop, Poisson sessions at 200/s, "
                                       "70 % unicycle / 30 % arm, replan every 20 ms"},
                "served": served, "plain": plain}
        print(json.dumps(line), flush=True)
        return

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
    bus = ""
    try:
        bus = "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except AttributeError:
        pass
    clocks = ClockSampler(local, bus)   # (the whole run)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    assert args.steps >= 1

    res, objs, planners, scenes, u_init, reset_episodes, step, prologue = run_workload(
        pkg, torch, args, args.workload, dev, stream, rank, world, dist, args.steps, args.warmup,
        flush, profile=True)
    value, tot_ms, step_ms = res["value"], res["tot_ms"], res["step_ms"]
    n_inst, episode, regen = res["n_inst"], res["episode"], res["regen"]
    cfg0 = scenes[0]["cfg"]
    n_dim, m, p_dim = pkg.DIMS[cfg0["dyn"]]
    stamps = None
    if args.stamps > 0:
        def restart():
            reset_episodes()
            prologue()

        restart()
        stamps = stage_stamps(planners, step, restart, args.stamps, episode)

    # ---- rooflines.  The fused clustering kernel (k_post) against HBM with
    # the algorithmic bytes above, and the rollout kernel against the FP32 ALU
    # peak; the kernel with the larger share of the step's device time heads
    # the line.
    pk, pk_kind = peaks()
    stage_ms = res["stage_ms"]
    post_ms = res["post_ms"]
    post_bytes = POST_BYTES_PER_ROLLOUT[p_dim] * res["post_rollouts"]
    post_gbs = post_bytes / (post_ms * 1e-3) / 1e9
    hbm = pk.get("hbm_gbs", 6400.0)
    tests = res["tests"]
    Ks, Ts = res["Ks"], res["Ts"]
    if cfg0["dyn"] in (pkg.DYN_ARM, pkg.DYN_ARM12):
        # per step: FK (6 DH transforms ~ 6*40) + 24 sphere centres (3*3*24)
        # + pose cost (~60); per sphere test 8 (3 sub, mul, 2 fma x2, compare)
        flops_roll = Ks * (Ts * (240 + 216 + 60) + 24 * 8 * tests)
    else:
        # 6 per circle test kept by the culling (2 sub, mul, fma counted 2,
        # compare) plus 60 per step for the clip, the cost and the model step
        flops_roll = Ks * (6.0 * tests + 60.0 * Ts)
    roll_ms = stage_ms["rollout"]
    achieved = float(flops_roll.sum()) / (roll_ms * 1e-3) / 1e12
    peak = alu_peak_tflops(props.multi_processor_count, pk.get("sm_max_mhz", 2032.0))
    launches_post = 2 if res["pipelined"] else 1
    post_share = launches_post * post_ms
    roll_share = roll_ms
    roof_post = {"kernel": "k_post (prune + DBSCAN + selection + update)", "bound": "hbm",
                 "achieved": post_gbs, "peak": hbm, "unit": "GB/s", "frac": post_gbs / hbm,
                 "traffic": NCU_TRAFFIC.get((args.workload, "k_post")),
                 "peak_kind": f"copy bandwidth ({pk_kind})",
                 "ms_per_launch": post_ms, "algorithmic_bytes_per_launch": post_bytes,
                 "bytes_per_rollout": POST_BYTES_PER_ROLLOUT[p_dim],
                 "note": "latency-bound: chains of dependent L2 accesses between cluster "
                         "barriers, far below the bandwidth bound; its DRAM traffic is below "
                         "the algorithmic bytes (the rollout epilogue's group records replace "
                         "per-rollout reads, and the working set stays in L2)"}
    roof_roll = {"kernel": "k_rollout_arm" if cfg0["dyn"] in (pkg.DYN_ARM, pkg.DYN_ARM12)
                 else "k_rollout2d<unicycle>", "bound": "alu", "achieved": achieved,
                 "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "traffic": NCU_TRAFFIC.get((args.workload, "rollout")),
                 "peak_kind": f"FP32 lanes x 2 x max SM clock ({pk_kind} clock)",
                 "ms_per_launch": roll_ms,
                 "flops_per_rollout": float(flops_roll.sum() / Ks.sum()),
                 "obstacle_tests_per_rollout": float(np.mean(tests))}
    dominant_post = post_share >= roll_share
    roof_upd = update_roofline(res, m, hbm, pk_kind, args.workload)

    # ---- end to end through the public API with host buffers: the batch
    # entry point that takes packed host arrays (ce_mppi_batch_run_host) --
    # per step the states and observation windows go in, the new nominals,
    # next states and diagnostics come back, one copy each way inside the
    # call; the loop is closed on the host (x0 <- x_next).
    e2e_pl = [pkg.Planner(sc["cfg"], n_obs_max=sc["radius"].shape[0]) for sc in scenes]
    for pl, sc in zip(e2e_pl, scenes):
        pl.set_nominal(u_init(sc))
    n_obs_l = [sc["radius"].shape[0] for sc in scenes]
    hb = pkg.HostBatch(e2e_pl, n_obs_l, stream=stream, use_graph=True, n_branches=args.branches)
    H = cfg0["hist_len"]
    n_e2e = max(1, min(args.e2e_steps, episode))
    windows = [np.concatenate([np.asarray(sc["obs"][r:r + H], np.float32).ravel()
                               for sc in scenes]) for r in range(n_e2e + 3)]
    radii = np.concatenate([sc["radius"] for sc in scenes]).astype(np.float32)
    x_host = np.concatenate([sc["x0"] for sc in scenes]).astype(np.float32)
    u_host = np.empty(hb.u_size, np.float32)
    xn_host = np.empty(hb.x_size, np.float32)

    def al16(v):
        return (v + 15) // 16 * 16

    h2d = sum(al16(4 * (n_dim + H * no * p_dim + no)) for no in n_obs_l)
    d2h = sum(al16(4 * (sc["cfg"]["T"] * m + n_dim)) + al16(80) for sc in scenes)
    for r in range(3):
        hb.run(x_host, windows[r], radii, u_host, xn_host)
        x_host, xn_host = xn_host, x_host
    t0 = time.perf_counter()
    for r in range(n_e2e):
        hb.run(x_host, windows[r + 3], radii, u_host, xn_host)
        x_host, xn_host = xn_host, x_host
    e2e_s = time.perf_counter() - t0
    e2e_value = world * res["units_per_step"] * n_e2e / e2e_s

    # ---- plain form: one instance per launch chain, blocking host-buffer call
    plain_pl = [pkg.Planner(sc["cfg"], n_obs_max=sc["radius"].shape[0]) for sc in scenes]
    for pl, sc in zip(plain_pl, scenes):
        pl.set_nominal(u_init(sc))
    lat = []
    t_plain = time.perf_counter()
    for r in range(args.plain_steps):
        for i, sc in enumerate(scenes):
            t1 = time.perf_counter()
            plain_pl[i].replan(sc["x0"], W.history(sc, r), sc["radius"])
            lat.append(time.perf_counter() - t1)
    t_plain = time.perf_counter() - t_plain
    lat = np.array(lat[n_inst:]) * 1e3  # first round is warm-up
    plain = {"replans_per_s": 1e3 / float(lat.mean()), "p50_ms": float(np.percentile(lat, 50)),
             "p99_ms": float(np.percentile(lat, 99)),
             "rollout_steps_per_s": res["units_per_step"] * args.plain_steps / t_plain}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(args.workload, world, regen),
        "run": {"pipeline": args.pipeline, "post_first": args.post_first,
                "early_tracks": early_tracks(args, args.workload),
                "pipe_post_ctas": args.pipe_post_ctas,
                "batch_config": res["batch_config"],
                "l2": "flushed between timed steps (256 MB write)"},
        "replans_per_s": res["replans_per_s"],
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99)),
                       "note": f"batched step: all {n_inst} replans complete"},
        "plain": plain,
        "stage_ms": stage_ms,
        "modes_last_step": res["modes_last_step"],
        "roofline": roof_post if dominant_post else roof_roll,
        ("roofline_rollout" if dominant_post else "roofline_post"):
            roof_roll if dominant_post else roof_post,
        "device_time_share_ms_per_step": {"k_post": post_share, "k_rollout": roll_share},
        **({"roofline_update": roof_upd} if roof_upd else {}),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "api": "ce_mppi_batch_run_host (packed host buffers, one copy each way, "
                       "graph replay, host-side closed loop)", "steps": n_e2e},
        # kernels per replan chain: tracks, rollouts, the fused clustering
        # kernel and the tiled update; per step two half chains (pipelined) or
        # one chain per branch (the L2 flush is torch's)
        "gpu_launches": 4 * (2 if res["pipelined"] else res["batch_config"]["n_branches"])
                        * args.steps,
    }
    if stamps is not None:
        line["post_stamps_cycles"] = stamps
    for obj in objs + [hb] + planners + e2e_pl + plain_pl:
        obj.close()
    # ---- the arm (config 3) and the uneven batch (config 4), measured
    # briefly beside the main workload (device-resident, graph, pipelined)
    if rank == 0 and not args.no_extra and args.workload == "unicycle":
        extra = {}
        for name in ("arm", "batch"):
            r2, objs2, pls2, _, _, _, _, _ = run_workload(
                pkg, torch, args, name, dev, stream, 0, 1, None, args.extra_steps, 3, flush,
                profile=(name == "arm"))
            extra[name] = {"config": bench_config(name, 1, r2["regen"]), "value": r2["value"],
                           "unit": UNIT, "replans_per_s": r2["replans_per_s"],
                           "ms_per_step": r2["tot_ms"] / args.extra_steps,
                           "steps": args.extra_steps,
                           "latency_ms": {"p50": float(np.percentile(r2["step_ms"], 50)),
                                          "p99": float(np.percentile(r2["step_ms"], 99))},
                           "modes_last_step": r2["modes_last_step"]}
            if name == "arm":
                ru = update_roofline(r2, pkg.DIMS[pkg.DYN_ARM][1], hbm, pk_kind, "arm")
                if ru:
                    extra[name]["roofline_update"] = ru
            for obj in objs2 + pls2:
                obj.close()
        line["extra_workloads"] = extra
    if rank == 0 and args.serve_seconds > 0 and args.workload == "unicycle":
        line["served"] = run_serve(pkg, args.serve_seconds, args.serve_budget_gb,
                                   warmup_s=args.serve_warmup)
        line["served"]["plain_mix"] = plain_mix_latency(pkg)
        # the plain form under the same offered load: the same server with one
        # instance per launch chain and one stream (a session's queued request
        # is still replaced by its newer one, which bounds the queue)
        line["served"]["plain_same_load"] = run_serve(pkg, min(args.serve_seconds, 5.0),
                                                      args.serve_budget_gb, max_batch=1,
                                                      n_streams=1, warmup_s=0.0)
    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        line["cpu_baseline"] = cpu_baseline(scenes, u_init, max_threads=16)
    line["clocks"] = clocks.stop()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
