"""Oracle parity at the benchmark's own configuration and launch shape.

The benchmark runs the unicycle workload (K=16384, T=50, 50 moving discs,
sigma 0.5, DBSCAN eps 0.25 / minPts 20) as 16 closed-loop episodes resident on
the device (observation streams replayed through obs_step, x_next aliasing
x0), with noise regeneration, in two software-pipelined halves of 8 episodes
whose half replans (tracks + rollouts; clustering + update) interleave on two
streams inside one captured CUDA graph.  This test builds exactly that, runs a
whole 200-replan episode, and checks replans 1, 50, 150 and 199 of episodes 0
and 1 stage by stage against the FP64 oracle fed the device's own state,
nominal and replan counter before that replan -- plus the first replan of the
episode without any colliding rollout (the standard-MPPI fallback).  The
episodes then run on without restarts until a no-collision replan with more
than 256 nonzero weights (the dense update, which draws every perturbation
again) is found and checked as well.
"""
import numpy as np
import pytest

import paper_2607_06499_b300 as pkg
from paper_2607_06499_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from parity_check import check_outputs, parity_report_fixture  # noqa: E402

_parity_report = parity_report_fixture()

N_EP, EPISODE, HALF = 16, 200, 8
CHECKS = (1, 50, 150, 199)
LONG = 2000          # replans run without restarts while looking for a dense fallback
PEEKS = ("S", "HIT", "HITJ", "PN", "IDXV", "IDXC", "Z", "G", "LABEL", "W")


def _diag(t):
    return pkg.Diag.from_buffer_copy(t.cpu().numpy().tobytes()[:C_DIAG]).as_dict()


C_DIAG = __import__("ctypes").sizeof(pkg.Diag)


def test_benchmark_configuration_against_the_oracle():
    dev = torch.device("cuda")
    scenes = [W.make("unicycle", seed=s, n_replans=LONG + 8, noise_regen=1) for s in range(N_EP)]
    cfg0 = scenes[0]["cfg"]
    assert (cfg0["K"], cfg0["T"], cfg0["sigma"], cfg0["noise_regen"]) == (16384, 50, [0.5, 0.5], 1)
    u_init = np.tile([1.0, 0.0], (cfg0["T"], 1))
    planners, reqs = [], []
    for sc in scenes:
        n_obs = sc["radius"].shape[0]
        planners.append(pkg.Planner(sc["cfg"], n_obs_max=n_obs))
        rq = dict(x0=torch.tensor(sc["x0"], dtype=torch.float32, device=dev),
                  hist=torch.tensor(sc["obs"], dtype=torch.float32, device=dev).contiguous(),
                  radius=torch.tensor(sc["radius"], dtype=torch.float32, device=dev),
                  u_out=torch.zeros((cfg0["T"], 2), dtype=torch.float32, device=dev),
                  diag=torch.zeros(128, dtype=torch.uint8, device=dev), obs_step=n_obs * 2)
        rq["x_next"] = rq["x0"]
        reqs.append(rq)
    for pl in planners:
        pl.set_nominal(u_init)
        pl.set_counter(0)
    torch.cuda.synchronize()
    # the benchmark's two pipelined halves in one captured graph
    bA = pkg.Batch(planners[:HALF], reqs[:HALF], use_graph=False)
    bB = pkg.Batch(planners[HALF:], reqs[HALF:], use_graph=False)
    side = torch.cuda.Stream()
    trk = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    # (as in the benchmark: each half's rollouts wait for the other half's
    # clustering kernel to have begun on all its CTAs; a half's track kernel
    # runs on a third stream right after its clustering + update)
    started = [torch.cuda.Event(enable_timing=False) for _ in range(2)]
    for e in started:
        e.record()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        main = torch.cuda.current_stream()
        side.wait_stream(main)
        bB.run_part(1, main, started=started[1])
        trk.wait_stream(main)
        bB.run_part(2, trk)
        side.wait_event(started[1])
        bA.run_part(3, side)
        main.wait_stream(side)
        side.wait_stream(main)
        bA.run_part(1, main, started=started[0])
        side.wait_event(started[0])
        side.wait_stream(trk)
        trk.wait_stream(main)
        bA.run_part(2, trk)
        bB.run_part(3, side)
        main.wait_stream(trk)
        main.wait_stream(side)
    torch.cuda.synchronize()
    bB.run_part(0, torch.cuda.current_stream())   # B's first tracks + rollouts
    bA.run_part(2, torch.cuda.current_stream())   # A's first tracks
    checked, nocol, dense = [], None, None
    modes = {}
    for r in range(LONG):
        # half A's replan r runs whole inside replay r: its inputs are the
        # device state now (x0 = the previous x_next, nominal, counter = r)
        torch.cuda.synchronize()
        pre = [(reqs[i]["x0"].cpu().numpy().astype(np.float64), planners[i].get_nominal(),
                planners[i].get_counter()) for i in range(HALF)]
        graph.replay()
        torch.cuda.synchronize()
        for i in range(HALF):
            d = _diag(reqs[i]["diag"])
            assert d["status"] == 0 and d["counter"] == r == pre[i][2]
            modes[d["mode"]] = modes.get(d["mode"], 0) + 1
            want = (r < EPISODE and i < 2 and r in CHECKS)
            is_nocol = d["mode"] == 0
            if is_nocol and nocol is None and r < EPISODE:
                want = True
            nnz = None
            if is_nocol and dense is None:
                nnz = int(np.count_nonzero(planners[i].peek("W")))
                want = want or nnz > 256
            if not want:
                continue
            sc, pl = scenes[i], planners[i]
            out = {k: pl.peek(k) for k in PEEKS}
            out["nominal_after"] = pl.get_nominal()
            out["counter_after"] = pl.get_counter()
            u = reqs[i]["u_out"].cpu().numpy()
            hist = W.history(sc, r)
            case = f"bench-config episode {i} replan {r}"
            check_outputs(sc["cfg"], pre[i][0], pre[i][1], hist, sc["radius"], r, u, d, out,
                          case=case)
            checked.append((i, r, pkg.MODES[d["mode"]]))
            if is_nocol and nocol is None and r < EPISODE:
                nocol = (i, r)
            if is_nocol and nnz is not None and nnz > 256:
                dense = (i, r, nnz)
        if r + 1 >= EPISODE and nocol is not None and dense is not None:
            break
    print("BENCH-CONFIG checked", checked, "modes", modes, "nocol", nocol, "dense", dense)
    for obj in [bA, bB] + planners:
        obj.close()
    assert len([c for c in checked if c[1] in CHECKS and c[0] < 2]) == 2 * len(CHECKS)
    assert nocol is not None, "no replan without collisions in the 200-replan episode"
    assert dense is not None, f"no dense no-collision replan within {LONG} replans"
