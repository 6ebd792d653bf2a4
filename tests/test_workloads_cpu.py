"""The seeded input generators follow the stated recipe: a seed names the same
scene every time, different seeds give different scenes, and the sizes, value
ranges and motion are those the workloads are described with (unicycle: 50
discs of radius 0.2-0.6 m in a 20 x 20 m field at up to 1.5 m/s, clear of the
start and goal; the uneven batch: K log-uniform in [512, 16384], T in [20, 60],
5-100 discs; the served mix: Poisson arrivals, 70 % unicycle)."""
import math

import numpy as np
import pytest

from paper_2607_06499_b300 import workloads as W

NAMES = ("di_static", "di_blocked", "unicycle", "unicycle_blocked", "unicycle_paper",
         "batch_instance", "arm", "arm_blocked", "arm_paper", "arm12", "arm12_blocked")


@pytest.mark.parametrize("name", NAMES)
def test_a_seed_names_one_scene(name):
    a = W.make(name, seed=3, n_replans=4)
    b = W.make(name, seed=3, n_replans=4)
    assert a["cfg"] == b["cfg"]
    for key in ("x0", "U0", "radius", "obs"):
        assert np.array_equal(a[key], b[key]), key
    n, m, p = W.DIMS[a["cfg"]["dyn"]]
    H = a["cfg"]["hist_len"]
    assert a["x0"].shape == (n,) and a["U0"].shape == (a["cfg"]["T"], m)
    assert a["obs"].shape == (4 + H - 1, a["radius"].shape[0], p)
    assert W.history(a, 3).shape == (H, a["radius"].shape[0], p)


@pytest.mark.parametrize("name", ("di_static", "unicycle", "batch_instance", "arm"))
def test_different_seeds_differ(name):
    a, b = W.make(name, seed=1), W.make(name, seed=2)
    assert a["radius"].shape != b["radius"].shape or not np.allclose(a["obs"], b["obs"])


def test_unicycle_recipe():
    sc = W.make("unicycle", seed=5, n_replans=200)
    cfg = sc["cfg"]
    assert (cfg["K"], cfg["T"], cfg["dyn"]) == (16384, 50, W.DYN_UNICYCLE)
    r, obs = sc["radius"], sc["obs"]
    assert r.shape == (50,) and np.all((r >= 0.2) & (r <= 0.6))
    # inside the field (centre at least a radius from each wall)
    assert np.all(obs >= r[None, :, None] - 1e-9) and np.all(obs <= 20 - r[None, :, None] + 1e-9)
    # clear of the start and the goal at the first observation
    for q in ((1.0, 1.0), (19.0, 19.0)):
        assert np.all(np.linalg.norm(obs[0] - np.array(q), axis=1) >= 1.0 + r - 1e-9)
    # speed at most 1.5 m/s (a wall reflection only shortens a step)
    step = np.linalg.norm(np.diff(obs, axis=0), axis=2)
    assert step.max() <= 1.5 * cfg["obs_dt"] + 1e-9 and step.max() > 0


def test_batch_instance_ranges():
    Ks, Ts, ns, static = [], [], [], 0
    for s in range(64):
        sc = W.make("batch_instance", seed=s, n_replans=3)
        Ks.append(sc["cfg"]["K"])
        Ts.append(sc["cfg"]["T"])
        ns.append(sc["radius"].shape[0])
        static += int(np.array_equal(sc["obs"][0], sc["obs"][-1]))
    assert min(Ks) >= 512 and max(Ks) <= 16384 and len(set(Ks)) > 32
    assert min(Ts) >= 20 and max(Ts) <= 60
    assert min(ns) >= 5 and max(ns) <= 100
    assert 16 <= static <= 48   # static with probability 1/2


def test_session_arrivals_are_poisson_with_the_stated_mix():
    arr = W.session_arrivals(200.0, 60.0, seed=0)
    t = np.array([a["t"] for a in arr])
    assert np.all(np.diff(t) > 0) and t[-1] < 60.0
    assert abs(len(arr) - 12000) < 5 * math.sqrt(12000)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 200) < 0.05 / 200
    uni = [a for a in arr if a["kind"] == "unicycle"]
    assert abs(len(uni) / len(arr) - 0.7) < 0.02
    assert {a["K"] for a in uni} == {1024, 4096, 16384}
    assert {a["K"] for a in arr if a["kind"] == "arm"} == {2048, 4096}
    life = np.array([a["lifetime"] for a in arr])
    assert life.min() >= 2.0 and life.max() <= 20.0
