"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
published known-answer vectors, closed forms, hand-worked kinematics, library
routines (scipy, scikit-learn) and invariants the paper states.  Each test names
the paper passage (section / equation number in display order) it pins.
"""
import math
import os

import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_2607_06499_b300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _cfg(name="di_static", **over):
    sc = W.make(name, seed=0, **over)
    return sc


def _params(cfg, **kw):
    P = oracle.make_params(cfg)
    for k, v in kw.items():
        if k in ("sigma", "u_min", "u_max", "goal", "w"):
            arr = getattr(P, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(P, k, v)
    return P


# --------------------------------------------------------------------------- Philox
def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_normals_are_standard_gaussian():
    # Sec. II-A: eps ~ N(0, Sigma).  Kolmogorov-Smirnov against N(0,1) over many
    # rollouts, plus near-zero lag correlation inside a rollout.
    z = np.concatenate([oracle.normals(7, 3, k, 64) for k in range(800)])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1.0) < 0.03
    a = z.reshape(800, 64)
    lag = np.mean(a[:, :-1] * a[:, 1:])
    assert abs(lag) < 0.02


def test_normals_depend_on_rollout_counter_and_seed():
    base = oracle.normals(1, 0, 5, 12)
    assert not np.allclose(base, oracle.normals(1, 0, 6, 12))
    assert not np.allclose(base, oracle.normals(1, 1, 5, 12))
    assert not np.allclose(base, oracle.normals(2, 0, 5, 12))
    # a prefix request gives the prefix of a longer one (counter = normal index / 4)
    assert np.array_equal(oracle.normals(1, 0, 5, 7), base[:7])


def test_normals_lie_on_the_23_bit_uniform_grid():
    """Each pair (z0, z1) is (r cos 2 pi u2, r sin 2 pi u2), r^2 = -2 ln u1,
    with u1, u2 on the grid (f + 1/2) 2^-23 of 23-bit fields: exp(-r^2/2) 2^23
    - 1/2 and the angle's fraction of a turn times 2^23 - 1/2 are integers.
    Normals 4b .. 4b+3 come from Philox block b (words pinned by the published
    test vectors): pair p's u1 and u2 are the top 23 bits of words 2p and
    2p + 1."""
    z = np.concatenate([oracle.normals(11, 5, k, 60) for k in range(200)]).reshape(-1, 2)
    r2 = (z ** 2).sum(1)
    f1 = np.exp(-r2 / 2) * 2.0 ** 23 - 0.5
    ang = np.mod(np.arctan2(z[:, 1], z[:, 0]) / (2 * np.pi), 1.0)
    f2 = ang * 2.0 ** 23 - 0.5
    assert np.abs(f1 - np.round(f1)).max() < 1e-2
    # (the angle's fraction of a turn is u2 or u2 - 1, both on the grid mod 1)
    d2 = np.abs(f2 - np.round(f2))
    assert np.minimum(d2, 1 - d2).max() < 1e-2
    seed, counter, k, b = 0x299F31D0A4093822, (7 << 32) + 12345, 3, 2
    zk = oracle.normals(seed, counter, k, 4 * (b + 1))[4 * b:]
    w = oracle.philox4x32_10([k, b, counter & 0xFFFFFFFF, counter >> 32],
                             [seed & 0xFFFFFFFF, seed >> 32])
    for p in range(2):
        r2p = zk[2 * p] ** 2 + zk[2 * p + 1] ** 2
        assert abs(np.exp(-r2p / 2) * 2.0 ** 23 - 0.5 - (int(w[2 * p]) >> 9)) < 1e-2
        a = np.mod(np.arctan2(zk[2 * p + 1], zk[2 * p]) / (2 * np.pi), 1.0) * 2.0 ** 23 - 0.5
        assert abs(a - (int(w[2 * p + 1]) >> 9)) < 1e-2


# --------------------------------------------------------------------------- Eq. 17
def test_obstacle_velocity_telescopes():
    sc = _cfg("unicycle", K=64)
    P = oracle.make_params(sc["cfg"])
    hist = np.random.default_rng(0).normal(size=(5, 7, 2))
    v = oracle.obstacle_velocity(P, hist)
    closed = (hist[-1] - hist[0]) / ((5 - 1) * P.obs_dt)
    np.testing.assert_allclose(v, closed, rtol=1e-12, atol=1e-12)
    P1 = _params(sc["cfg"], hist_len=1)
    assert np.all(oracle.obstacle_velocity(P1, hist[:1]) == 0)


def test_tracks_constant_velocity_from_newest():
    sc = _cfg("unicycle", K=64, T=9)
    P = oracle.make_params(sc["cfg"])
    hist = np.random.default_rng(1).normal(size=(5, 4, 2))
    tr = oracle.tracks(P, hist)
    assert tr.shape == (10, 4, 2)
    np.testing.assert_array_equal(tr[0], hist[-1])
    d = np.diff(tr, axis=0)
    np.testing.assert_allclose(d, np.broadcast_to(d[0], d.shape), atol=1e-12)
    v = (hist[-1] - hist[0]) / (4 * P.obs_dt)
    np.testing.assert_allclose(d[0], v * P.dt, atol=1e-12)


# --------------------------------------------------------------------------- Eq. 4-5
def test_double_integrator_closed_form_and_cost():
    sc = _cfg("di_static", K=16, T=11)
    cfg = sc["cfg"]
    P = oracle.make_params(cfg)
    x0 = np.array([0.3, -0.2, 0.7, 0.1])
    U = np.random.default_rng(2).uniform(-1, 1, size=(11, 2))
    far = np.array([[100.0, 100.0]])
    trk = np.repeat(far[None], 12, axis=0)
    r = oracle.rollouts(P, x0, U, trk, np.array([0.1]), want_traj=True)
    dt, N = P.dt, P.T
    a = U[None] + r["eps"]                               # applied accelerations
    jw = (N - 1 - np.arange(N))[None, :, None]
    pN = x0[None, :2] + N * dt * x0[None, 2:] + dt * dt * np.sum(jw * a, axis=1)
    vN = x0[None, 2:] + dt * np.sum(a, axis=1)
    np.testing.assert_allclose(r["traj"][:, -1, :2], pN, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["traj"][:, -1, 2:], vN, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["pN"], pN, rtol=1e-12, atol=1e-12)
    # positions p_j from the closed form at every j; Eq. 5 with the DI cost
    g = np.array(cfg["goal"][:2])
    S = np.zeros(16)
    for j in range(N + 1):
        jwj = np.clip(j - 1 - np.arange(N), 0, None)[None, :, None]
        pj = x0[None, :2] + j * dt * x0[None, 2:] + dt * dt * np.sum(jwj * a, axis=1)
        if j < N:
            S += np.sum((pj - g) ** 2, axis=1) + 0.01 * np.sum(a[:, j] ** 2, axis=1)
        else:
            S += np.sum((pj - g) ** 2, axis=1)
    np.testing.assert_allclose(r["S"], S, rtol=1e-12)
    # Eq. 3 with clipping: applied controls inside the box, eps' = u - nominal
    assert np.all(a <= 2.0 + 1e-15) and np.all(a >= -2.0 - 1e-15)


def test_perturbation_is_sigma_times_normals_when_unclipped():
    sc = _cfg("di_static", K=8, T=6)
    P = _params(sc["cfg"], u_min=[-1e9, -1e9], u_max=[1e9, 1e9], sigma=[0.3, 0.7])
    trk = np.full((7, 1, 2), 100.0)
    r = oracle.rollouts(P, np.zeros(4), np.zeros((6, 2)), trk, np.array([0.1]))
    for k in range(8):
        z = oracle.normals(P.seed, P.counter, k, 12).reshape(6, 2)
        np.testing.assert_allclose(r["eps"][k], z * np.array([0.3, 0.7]), rtol=1e-14)


def test_unicycle_straight_line_and_arc():
    sc = _cfg("unicycle", K=4, T=20)
    cfg = sc["cfg"]
    P = _params(cfg, sigma=[0.0, 0.0])
    trk = np.full((21, 1, 2), 1e3)
    x0 = np.array([1.0, 2.0, 0.3])
    U = np.tile([1.5, 0.0], (20, 1))
    r = oracle.rollouts(P, x0, U, trk, np.array([0.1]), want_traj=True)
    tr = r["traj"][0]
    dist = 1.5 * P.dt * 20
    np.testing.assert_allclose(tr[-1, :2], x0[:2] + dist * np.array([math.cos(0.3), math.sin(0.3)]),
                               rtol=1e-12)
    # constant omega: Euler polygon, sum of cos(theta0 + j phi) in closed form
    w, v, N, dt = 0.8, 1.2, 20, P.dt
    U = np.tile([v, w], (20, 1))
    tr = oracle.rollouts(P, x0, U, trk, np.array([0.1]), want_traj=True)["traj"][0]
    phi = w * dt
    ratio = math.sin(N * phi / 2) / math.sin(phi / 2)
    xN = x0[0] + v * dt * ratio * math.cos(0.3 + (N - 1) * phi / 2)
    yN = x0[1] + v * dt * ratio * math.sin(0.3 + (N - 1) * phi / 2)
    np.testing.assert_allclose(tr[-1], [xN, yN, 0.3 + N * phi], rtol=1e-12)


def test_unicycle_cost_at_rest_closed_form():
    # Eq. 22-23: robot held still (v = 0): S = T * l(x0) + phi(x0)
    sc = _cfg("unicycle", K=2, T=7)
    P = _params(sc["cfg"], sigma=[0.0, 0.0])
    x0 = np.array([3.0, 4.0, 1.0])
    r = oracle.rollouts(P, x0, np.zeros((7, 2)), np.full((8, 1, 2), 1e3), np.array([0.1]))
    e = x0 - np.array([19.0, 19.0, math.pi / 4])
    expect = 7 * (10 * e[0] ** 2 + 10 * e[1] ** 2) + 50 * np.sum(e ** 2)
    np.testing.assert_allclose(r["S"], expect, rtol=1e-13)


# --------------------------------------------------------------------------- arm
def test_arm_fk_zero_pose_hand_worked():
    rows = [l.split() for l in open(os.path.join(GOLD, "ur5e_zero_pose.txt"))
            if l.strip() and not l.startswith("#")]
    O, R = oracle.arm_fk(np.zeros(6))
    for r in rows:
        if r[0] == "R":
            np.testing.assert_allclose(R.ravel(), [float(x) for x in r[1:]], atol=1e-12)
        else:
            np.testing.assert_allclose(O[int(r[0])], [float(x) for x in r[1:]], atol=1e-12)


def test_arm_fk_invariants():
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = rng.uniform(-math.pi, math.pi, 6)
        O, R = oracle.arm_fk(q)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - 1) < 1e-12
        # joint 1 turns the whole arm about the base z axis
        dq = 0.7
        O2, R2 = oracle.arm_fk(q + np.array([dq, 0, 0, 0, 0, 0]))
        Rz = np.array([[math.cos(dq), -math.sin(dq), 0], [math.sin(dq), math.cos(dq), 0], [0, 0, 1]])
        np.testing.assert_allclose(O2, O @ Rz.T, atol=1e-12)
        np.testing.assert_allclose(R2, Rz @ R, atol=1e-12)
        # link lengths are fixed by the DH table whatever the joint angles
        np.testing.assert_allclose(np.linalg.norm(O[1] - O[0]), 0.1625, atol=1e-12)
        np.testing.assert_allclose(np.linalg.norm(O[2] - O[1]), 0.425, atol=1e-12)
        np.testing.assert_allclose(np.linalg.norm(O[3] - O[2]), 0.3922, atol=1e-12)
        np.testing.assert_allclose(np.linalg.norm(O[6] - O[5]), 0.0996, atol=1e-12)


def test_arm_spheres_on_link_segments():
    sc = _cfg("arm", K=4)
    P = oracle.make_params(sc["cfg"])
    q = np.random.default_rng(4).uniform(-2, 2, 6)
    pts = oracle.robot_points(P, q)
    O, _ = oracle.arm_fk(q)
    assert pts.shape == (24, 3)
    for link in range(6):
        for f in range(4):
            np.testing.assert_allclose(pts[link * 4 + f],
                                       O[link] + f / 3 * (O[link + 1] - O[link]), atol=1e-12)


def test_arm_pose_cost_closed_form():
    # Eq. 24: goal displaced by d and rotated by alpha about an axis ->
    # l = w_p |d| + w_R alpha (no collision); with the arm held still
    # S = (T + 1) * l since phi(x_N) = l(x_N).
    sc = _cfg("arm", K=2, T=3)
    q0 = np.array(W.ARM_Q0)
    O, R = oracle.arm_fk(q0)
    d = np.array([0.03, -0.04, 0.12])
    alpha = 0.37
    ax = np.array([1.0, 2.0, -0.5])
    ax /= np.linalg.norm(ax)
    Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rot = np.eye(3) + math.sin(alpha) * Kx + (1 - math.cos(alpha)) * Kx @ Kx
    goal = list(O[6] + d) + list((R @ Rot).ravel())
    P = _params(sc["cfg"], sigma=[0.0] * 6, goal=goal)
    trk = np.full((4, 1, 3), 50.0)
    r = oracle.rollouts(P, q0, np.zeros((3, 6)), trk, np.array([0.1]))
    expect = 4 * (10 * np.linalg.norm(d) + 3 * alpha)
    np.testing.assert_allclose(r["S"], expect, rtol=1e-12)
    # an obstacle touching the end effector at every step adds w_c per state
    trk2 = np.repeat(O[6][None, None, :], 4, axis=0)
    r2 = oracle.rollouts(P, q0, np.zeros((3, 6)), trk2, np.array([0.1]))
    np.testing.assert_allclose(r2["S"], expect + 4 * 1000, rtol=1e-12)
    assert np.all(r2["col"] == 1) and np.all(r2["hit_j"] == 1)


# --------------------------------------------------------------------------- Eq. 8-10
def test_collision_first_hit_and_pruning():
    # DI at constant velocity (no noise): p_j = (0.1 j, 0) with dt=0.05, v=2
    sc = _cfg("di_static", K=3, T=12)
    P = _params(sc["cfg"], sigma=[0.0, 0.0])
    x0 = np.array([0.0, 0.0, 2.0, 0.0])
    cent = np.array([[0.85, 0.0], [0.5, 0.2], [0.3, 5.0], [0.5, -0.02]])
    rad = np.array([0.06, 0.21, 0.1, 0.03])
    trk = np.repeat(cent[None], 13, axis=0)
    r = oracle.rollouts(P, x0, np.zeros((12, 2)), trk, rad)
    # j = 5 (x = 0.5) is the first time inside obstacles 1 and 3; obstacle 0 from j = 8
    assert list(r["hit"]) == [1, 1, 1] and list(r["hit_j"]) == [5, 5, 5]
    pos = np.stack([0.1 * np.arange(1, 13), np.zeros(12)], 1)
    clear = np.linalg.norm(pos[:, None] - cent[None], axis=2) - rad[None]
    np.testing.assert_allclose(r["min_abs_clear"], np.abs(clear).min(), rtol=1e-12)
    # the current state is not tested unless check_j0
    trk0 = trk.copy()
    trk0[0] = [[0.0, 0.0], [9, 9], [9, 9], [9, 9]]
    trk0[1:] = 9.0
    assert oracle.rollouts(P, x0, np.zeros((12, 2)), trk0, rad)["col"].sum() == 0
    P.check_j0 = 1
    rj = oracle.rollouts(P, x0, np.zeros((12, 2)), trk0, rad)
    assert list(rj["hit_j"]) == [0, 0, 0]
    col = np.array([0, 1, 1, 0, 1, 0, 0], np.int32)
    V, Cc = oracle.prune(col)
    assert list(V) == list(np.flatnonzero(col == 0)) and list(Cc) == list(np.flatnonzero(col))


# --------------------------------------------------------------------------- Eq. 11-15
def test_reference_point_closest_obstacle_and_features():
    sc = _cfg("di_static", K=6, T=5)
    P = oracle.make_params(sc["cfg"])
    x0 = np.array([0.0, 0.0, 0.0, 0.0])
    trk = np.zeros((6, 3, 2))
    trk[:] = np.array([[2.0, 0.0], [1.0, 0.0], [5.0, 0.0]])
    rad = np.array([0.5, 0.2, 0.1])
    pN = np.array([[1, 1], [2, 2], [3, 0], [4, 4], [9, 9], [5, 1]], float)
    hit = np.array([-1, 0, 1, 1, -1, 2], np.int32)
    idxC = np.array([1, 2, 3, 5], np.int32)
    o, pbar = oracle.reference_point(P, x0, trk, rad, idxC, hit, pN)
    # clearances 1.5, 0.8, 4.9 -> obstacle 1; mean of rollouts 2 and 3
    assert o == 1
    np.testing.assert_allclose(pbar, [3.5, 2.0])
    P.ref_mode = 1
    _, pbar1 = oracle.reference_point(P, x0, trk, rad, idxC, hit, pN)
    np.testing.assert_allclose(pbar1, pN[idxC].mean(axis=0))
    # single colliding rollout -> pbar is its terminal position
    P.ref_mode = 0
    _, pb = oracle.reference_point(P, x0, trk, rad, np.array([5], np.int32), hit, pN)
    np.testing.assert_allclose(pb, pN[5])
    z, g = oracle.features(P, x0, pbar, np.array([0, 4], np.int32), pN)
    for i, k in enumerate([0, 4]):
        d = pN[k] - pbar
        assert np.linalg.norm(z[i]) < 1.0
        np.testing.assert_allclose(z[i] * (np.linalg.norm(d) + 1e-6), d, rtol=1e-13)
        e = pN[k] - x0[:2]
        np.testing.assert_allclose(g[i] * (np.linalg.norm(e) + 1e-6), e, rtol=1e-13)


# --------------------------------------------------------------------------- DBSCAN
def _well_separated_points(rng, n, p, eps):
    """Random points on arcs of the unit circle/sphere whose pairwise distances
    all stay at least 1e-4 away from eps (FP32 and FP64 predicates agree)."""
    while True:
        if p == 2:
            centres = rng.uniform(0, 2 * math.pi, size=3)
            ang = centres[rng.integers(0, 3, n)] + rng.normal(scale=0.15, size=n)
            z = np.stack([np.cos(ang), np.sin(ang)], 1) * 0.999
            z[rng.integers(0, n, n // 20)] = rng.uniform(-1, 1, (n // 20, 2)) * 0.7
        else:
            z = rng.normal(size=(n, 3))
            z /= np.linalg.norm(z, axis=1, keepdims=True)
            z[: n // 2] = z[0] + 0.15 * rng.normal(size=(n // 2, 3))
        z = z.astype(np.float32).astype(np.float64)
        D = np.sqrt(((z[:, None, :] - z[None, :, :]) ** 2).sum(-1))
        if np.min(np.abs(D - eps)) > 1e-4:
            return z


@pytest.mark.parametrize("p,n,eps,mp", [(2, 300, 0.25, 20), (2, 200, 0.3, 10), (3, 250, 0.2, 16)])
def test_dbscan_matches_scikit_learn(p, n, eps, mp):
    from sklearn.cluster import DBSCAN
    rng = np.random.default_rng(10 + p + n)
    z = _well_separated_points(rng, n, p, eps)
    labels, M = oracle.dbscan(z, eps, mp)
    sk = DBSCAN(eps=eps, min_samples=mp).fit(z)
    core = np.zeros(n, bool)
    core[sk.core_sample_indices_] = True
    D = np.sqrt(((z[:, None, :] - z[None, :, :]) ** 2).sum(-1))
    # same noise set
    assert np.array_equal(labels < 0, sk.labels_ < 0)
    # same partition of the core points (one-to-one label correspondence)
    pairs = set(zip(labels[core], sk.labels_[core]))
    assert len(pairs) == len(set(labels[core])) == len(set(sk.labels_[core])) == M
    # canonical ids: cluster c's smallest core member precedes cluster c+1's
    firsts = [np.flatnonzero(core & (labels == c)).min() for c in range(M)]
    assert firsts == sorted(firsts)
    # border points: label of the lowest-index core point within eps
    for a in np.flatnonzero(~core & (labels >= 0)):
        nbrs = np.flatnonzero(core & (D[a] <= eps))
        assert labels[a] == labels[nbrs.min()]


def test_dbscan_permutation_invariant_and_brute_force_tiny():
    rng = np.random.default_rng(5)
    z = _well_separated_points(rng, 120, 2, 0.3)
    lab, M = oracle.dbscan(z, 0.3, 6)
    perm = rng.permutation(120)
    lab2, M2 = oracle.dbscan(z[perm], 0.3, 6)
    assert M == M2
    # same co-membership of core points under the permutation
    D = np.sqrt(((z[:, None] - z[None]) ** 2).sum(-1))
    core = (D <= 0.3).sum(1) >= 6
    same = (lab[:, None] == lab[None, :]) & (lab[:, None] >= 0)
    inv = np.argsort(perm)
    same2 = (lab2[inv][:, None] == lab2[inv][None, :]) & (lab2[inv][:, None] >= 0)
    assert np.array_equal(same[np.ix_(core, core)], same2[np.ix_(core, core)])
    # brute force on 6 points: two pairs and a chain, minPts 2
    pts = np.array([[0, 0], [0.1, 0], [1, 1], [1.05, 1], [0.5, 0.5], [3, 3]], float)
    lab, M = oracle.dbscan(pts, 0.2, 2)
    assert list(lab) == [0, 0, 1, 1, -1, -1] and M == 2


def test_dbscan_predicate_is_fp32_inclusive():
    # distance exactly eps (in FP32) counts as a neighbour (<=)
    z = np.array([[0.0, 0.0], [0.25, 0.0]], np.float32)
    lab, M = oracle.dbscan(z, 0.25, 2)
    assert M == 1 and list(lab) == [0, 0]
    above = np.nextafter(np.float32(0.25), np.float32(1.0))
    z = np.array([[0.0, 0.0], [above, 0.0]], np.float32)
    lab, M = oracle.dbscan(z, 0.25, 2)
    assert M == 0


# --------------------------------------------------------------------------- Eq. 14-18
def test_selection_static_and_dynamic():
    sc = _cfg("di_static", K=6)
    P = oracle.make_params(sc["cfg"])
    idxV = np.arange(6, dtype=np.int32)
    labels = np.array([0, 0, 1, 1, -1, 1], np.int32)
    S = np.array([5.0, 7.0, 1.0, 2.0, -100.0, 3.0])
    g = np.array([[1, 0], [1, 0], [-1, 0], [-1, 0.1], [0, 1], [-1, -0.1]], float)
    r = oracle.select(P, labels, idxV, S, g, 2, np.zeros(2))
    assert r["dynamic"] == 0 and r["sel"] == 1                # means 6 vs 2; noise ignored
    np.testing.assert_allclose(r["Sbar"], [6.0, 2.0])
    np.testing.assert_allclose(r["vhat"][0], [1 / (1 + 1e-6), 0])
    # obstacle moving toward -x: the cluster moving toward +x is "most opposite"
    r = oracle.select(P, labels, idxV, S, g, 2, np.array([-0.5, 0.0]))
    assert r["dynamic"] == 1 and r["sel"] == 0
    r = oracle.select(P, labels, idxV, S, g, 2, np.array([0.5, 0.0]))
    assert r["sel"] == 1
    # below the static threshold the cost criterion applies
    r = oracle.select(P, labels, idxV, S, g, 2, np.array([0.03, 0.0]))
    assert r["dynamic"] == 0 and r["sel"] == 1
    # ties go to the lowest id
    S2 = np.array([1.0, 1.0, 1.0, 1.0, 0.0, 1.0])
    assert oracle.select(P, labels, idxV, S2, g, 2, np.zeros(2))["sel"] == 0


# --------------------------------------------------------------------------- Eq. 6-7, 19-20
def test_update_matches_softmax_and_limits():
    sc = _cfg("di_static", K=50, T=4)
    P = oracle.make_params(sc["cfg"])
    rng = np.random.default_rng(6)
    U = rng.uniform(-1, 1, (4, 2))
    S = rng.uniform(0, 5, 50)
    eps = rng.normal(size=(50, 4, 2))
    allk = np.arange(50, dtype=np.int32)
    U_new, w, smin = oracle.update(P, U, S, eps, allk)
    ws = special.softmax(-S / P.lam)
    np.testing.assert_allclose(w, ws, rtol=1e-12)
    np.testing.assert_allclose(U_new, U + np.einsum("k,kjd->jd", ws, eps), rtol=1e-12)
    assert abs(w.sum() - 1) < 1e-12 and smin == S.min()
    # member subset: zero weight outside, renormalised inside (Eq. 19)
    mem = np.array([3, 9, 20], np.int32)
    U2, w2, _ = oracle.update(P, U, S, eps, mem)
    assert np.all(w2[np.setdiff1d(allk, mem)] == 0)
    np.testing.assert_allclose(w2[mem], special.softmax(-S[mem] / P.lam), rtol=1e-12)
    # lambda -> infinity: plain mean; lambda -> 0: the arg-min rollout
    P.lam = 1e12
    U3, _, _ = oracle.update(P, U, S, eps, allk)
    np.testing.assert_allclose(U3, U + eps.mean(0), rtol=1e-9, atol=1e-12)
    P.lam = 1e-6
    U4, _, _ = oracle.update(P, U, S, eps, allk)
    np.testing.assert_allclose(U4, U + eps[np.argmin(S)], atol=1e-12)
    # equal costs: uniform weights; huge costs do not underflow
    P.lam = 1.0
    _, w5, _ = oracle.update(P, U, np.full(50, 4e5), eps, allk)
    np.testing.assert_allclose(w5, 1 / 50, rtol=1e-12)


def test_shift_warm_start():
    sc = _cfg("di_static", K=2, T=4)
    P = oracle.make_params(sc["cfg"])
    U = np.arange(8.0).reshape(4, 2)
    np.testing.assert_array_equal(oracle.shift(P, U), [[2, 3], [4, 5], [6, 7], [6, 7]])


# --------------------------------------------------------------------------- Algorithm 1
def test_replan_without_collision_is_standard_mppi():
    sc = W.make("di_static", seed=0, K=256)
    P = oracle.make_params(sc["cfg"])
    r = oracle.replan(P, sc["x0"], sc["U0"], W.history(sc, 0), sc["radius"])
    assert r["diag"]["mode"] == oracle.MODE_NOCOL and r["col"].sum() == 0
    ws = special.softmax(-r["S"] / P.lam)
    np.testing.assert_allclose(r["U_new"], sc["U0"] + np.einsum("k,kjd->jd", ws, r["eps"]),
                               rtol=1e-10, atol=1e-14)


def test_replan_all_colliding_is_standard_mppi_over_all_rollouts():
    """Every rollout collides (the robot starts inside a disc, so its step-1
    position, which equals x_0 for a double integrator at rest, is inside for
    every k): V is empty, and the update is Eq. 6-7 over all K -- the reading
    taken where Algorithm 1 leaves this case undefined.  Weighting over V
    (empty) or over C_col minus some rollouts would fail here."""
    sc = W.make("di_static", seed=0, K=300, T=12)
    sc["radius"] = np.append(sc["radius"], 1.0)
    start = np.array(sc["x0"][:2])
    sc["obs"] = np.concatenate(
        [sc["obs"], np.broadcast_to(start, (sc["obs"].shape[0], 1, 2))], axis=1)
    P = oracle.make_params(sc["cfg"])
    r = oracle.replan(P, sc["x0"], sc["U0"], W.history(sc, 0), sc["radius"])
    d = r["diag"]
    assert d["mode"] == oracle.MODE_ALLCOL and d["n_valid"] == 0 and d["n_col"] == 300
    assert d["n_clusters"] == 0 and d["sel_label"] == -1 and np.all(r["col"] == 1)
    ws = special.softmax(-r["S"] / P.lam)
    np.testing.assert_allclose(r["w"], ws, rtol=1e-12, atol=1e-300)
    assert np.count_nonzero(r["w"]) == np.count_nonzero(ws) and r["w"][np.argmin(r["S"])] > 0
    np.testing.assert_allclose(r["U_new"], sc["U0"] + np.einsum("k,kjd->jd", ws, r["eps"]),
                               rtol=1e-12, atol=1e-14)
    assert d["S_min"] == r["S"].min()


def test_replan_all_noise_is_standard_mppi_over_the_valid_rollouts():
    """DBSCAN finds no cluster (minPts above |V|, so no point is core): the
    update is Eq. 6-7 over V alone -- colliding rollouts keep zero weight
    (the reading taken where Algorithm 1 leaves this case undefined)."""
    sc = W.make("di_blocked", seed=0, K=400)
    P = oracle.make_params(sc["cfg"])
    P.min_pts = 401
    r = oracle.replan(P, sc["x0"], sc["U0"], W.history(sc, 0), sc["radius"])
    d = r["diag"]
    assert d["n_col"] > 0 and d["n_valid"] > 0
    assert d["mode"] == oracle.MODE_ALLNOISE and d["n_clusters"] == 0 and d["sel_label"] == -1
    assert np.all(r["labels"] == -1)
    V = np.flatnonzero(r["col"] == 0)
    C_col = np.flatnonzero(r["col"] == 1)
    ws = special.softmax(-r["S"][V] / P.lam)
    np.testing.assert_allclose(r["w"][V], ws, rtol=1e-12, atol=1e-300)
    assert np.all(r["w"][C_col] == 0)
    np.testing.assert_allclose(r["U_new"],
                               sc["U0"] + np.einsum("k,kjd->jd", ws, r["eps"][V]),
                               rtol=1e-12, atol=1e-14)
    # the least cost is taken over V, not over all K
    assert d["S_min"] == r["S"][V].min()


@pytest.mark.parametrize("name", ["di_blocked", "unicycle_paper", "arm_paper", "unicycle_blocked"])
def test_replan_invariants(name):
    # the first seed whose first replan clusters (with the paper's K = 50 for
    # the arm, a collision is a matter of the draw)
    kw = dict(K=1024) if name == "unicycle_blocked" else {}
    for seed in range(10):
        sc = W.make(name, seed=seed, **kw)
        cfg = sc["cfg"]
        P = oracle.make_params(cfg)
        r = oracle.replan(P, sc["x0"], sc["U0"], W.history(sc, 0), sc["radius"])
        d = r["diag"]
        if d["n_col"] > 0 and d["n_valid"] > 0 and d["n_clusters"] >= 1:
            break
    assert d["n_col"] > 0 and d["n_valid"] > 0 and d["n_clusters"] >= 1
    w = r["w"]
    assert abs(w.sum() - 1) < 1e-12
    assert np.all(w[r["col"] == 1] == 0)                 # pruned rollouts never weigh in
    V = np.flatnonzero(r["col"] == 0)
    sel = V[r["labels"] == d["sel_label"]]
    assert np.all(w[np.setdiff1d(np.arange(cfg["K"]), sel)] == 0)
    assert np.all(w[sel] >= 0) and np.argmax(w) == sel[np.argmin(r["S"][sel])]
    # the update is a convex combination of feasible controls
    lo, hi = np.array(cfg["u_min"]), np.array(cfg["u_max"])
    assert np.all(r["U_new"] >= lo - 1e-12) and np.all(r["U_new"] <= hi + 1e-12)


# ----------------------------------------------------------------- 12-D arm
def test_arm12_double_integrator_closed_form():
    # explicit Euler with acceleration input: q_N = q_0 + N dt qdot_0 +
    # dt^2 sum_j (N-1-j) a_j, qdot_N = qdot_0 + dt sum_j a_j, per joint
    sc = _cfg("arm12", K=8, T=9)
    P = oracle.make_params(sc["cfg"])
    rng = np.random.default_rng(12)
    x0 = np.concatenate([rng.uniform(-1, 1, 6), rng.uniform(-0.5, 0.5, 6)])
    U = rng.uniform(-1, 1, size=(9, 6))
    far = np.full((10, 1, 3), 50.0)
    r = oracle.rollouts(P, x0, U, far, np.array([0.1]), want_traj=True)
    dt, N = P.dt, P.T
    a = U[None] + r["eps"]
    jw = (N - 1 - np.arange(N))[None, :, None]
    qN = x0[None, :6] + N * dt * x0[None, 6:] + dt * dt * np.sum(jw * a, axis=1)
    vN = x0[None, 6:] + dt * np.sum(a, axis=1)
    np.testing.assert_allclose(r["traj"][:, -1, :6], qN, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["traj"][:, -1, 6:], vN, rtol=1e-12, atol=1e-12)
    # the terminal task position is the end effector of q_N
    for k in range(8):
        O, _ = oracle.arm_fk(qN[k])
        np.testing.assert_allclose(r["pN"][k], O[6], atol=1e-12)


def test_arm12_at_rest_matches_the_velocity_arm():
    # zero velocity, zero input, no noise: both arm models hold q_0, so the
    # costs (Eq. 24 on q) are equal, (T+1) l(q_0)
    sc6, sc12 = _cfg("arm", K=2, T=6), _cfg("arm12", K=2, T=6)
    P6 = _params(sc6["cfg"], sigma=[0.0] * 6)
    P12 = _params(sc12["cfg"], sigma=[0.0] * 6)
    P12.goal[:] = P6.goal[:]
    q0 = np.random.default_rng(6).uniform(-2, 2, 6)
    far = np.full((7, 1, 3), 50.0)
    r6 = oracle.rollouts(P6, q0, np.zeros((6, 6)), far, np.array([0.1]))
    r12 = oracle.rollouts(P12, np.concatenate([q0, np.zeros(6)]), np.zeros((6, 6)), far,
                          np.array([0.1]))
    np.testing.assert_allclose(r12["S"], r6["S"], rtol=1e-14)
    np.testing.assert_allclose(r12["pN"], r6["pN"], atol=1e-14)



# ------------------------------------------------------- standard MPPI baseline
def test_collision_penalty_added_once_to_colliding_rollouts():
    sc = _cfg("di_blocked", K=64, T=30)
    P0 = oracle.make_params(sc["cfg"])
    P1 = oracle.make_params(sc["cfg"])
    P1.w[7] = 123.5
    hist = W.history(sc, 0)
    trk = oracle.tracks(P0, hist)
    r0 = oracle.rollouts(P0, sc["x0"], sc["U0"], trk, sc["radius"])
    r1 = oracle.rollouts(P1, sc["x0"], sc["U0"], trk, sc["radius"])
    assert r0["col"].sum() > 0 and (1 - r0["col"]).sum() > 0
    np.testing.assert_array_equal(r1["col"], r0["col"])
    np.testing.assert_allclose(r1["S"] - r0["S"], 123.5 * r0["col"], rtol=0, atol=1e-9)


def test_standard_mppi_replan_is_the_softmin_over_all_rollouts():
    sc = _cfg("di_blocked", K=96, T=30, mppi_only=1)
    P = oracle.make_params(sc["cfg"])
    out = oracle.replan(P, sc["x0"], sc["U0"], W.history(sc, 0), sc["radius"])
    assert out["diag"]["mode"] == 5 and out["diag"]["n_col"] > 0
    # Eq. 6-7 written out: weights softmin(S / lambda) over all K
    w = np.exp(-(out["S"] - out["S"].min()) / P.lam)
    w /= w.sum()
    np.testing.assert_allclose(out["w"], w, rtol=1e-12, atol=1e-15)
    U_ref = sc["U0"] + np.einsum("k,kjd->jd", w, out["eps"])
    np.testing.assert_allclose(out["U_new"], U_ref, rtol=1e-12, atol=1e-13)


# --------------------------------------------------------- task-level scenes
def test_scenario_scenes_and_evaluation():
    from paper_2607_06499_b300 import scenarios as SC
    s = SC.scene("static", 0, 60)
    assert s["obs"].shape == (65, 1, 2) and np.allclose(s["obs"][0], s["obs"][-1])
    c = SC.scene("crossing", 1, 50)
    v = (c["obs"][1:, 0] - c["obs"][:-1, 0]) / c["dt"]
    assert np.allclose(v[:, 0], 0.0) and np.all(v[:, 1] > 0.4)
    # a straight path through the wall collides; a detour above it reaches
    steps = 60
    xs = np.linspace(0.0, 4.0, steps + 1)
    straight = np.stack([xs, np.zeros_like(xs), np.zeros_like(xs)], 1)[:, None, :]
    r = SC.evaluate([s], straight)
    assert r["collided"] == 1 and r["reached"] == 0
    detour = straight.copy()
    detour[:, 0, 1] = 1.5 * np.sin(np.pi * xs / 4.0)
    r = SC.evaluate([s], detour)
    assert r["collided"] == 0 and r["reached"] == 1 and r["time_to_goal_median_s"] > 0


def test_averaging_failure_on_the_symmetric_blocking_scene():
    """Sec. I (Fig. 1) and Sec. III-B, Scenario 1: with the robot driving
    straight at a disc on its line to the goal, the free rollouts pass on both
    sides.  Standard MPPI (softmin over all K with the collision penalty,
    Eq. 6-7) averages the two sides into a nominal that still runs into the
    disc; CE-MPPI clusters the free rollouts (two clusters) and updates within
    one, so its nominal passes on one side.  Same seeds, so both methods see
    the same perturbations."""
    from paper_2607_06499_b300 import scenarios as SC
    sc = SC.scene("blocking", 0, 8)
    c, rad = sc["obs"][0, 0], sc["radius"]
    x0 = np.array([1.1, 0.0, 0.0])
    meets = {False: 0, True: 0}
    two = 0
    for seed in range(24):
        for mppi in (False, True):
            cfg = SC.planner_cfg(sc["goal"], mppi, seed, lam=5.0)
            P = oracle.make_params(cfg)
            U = np.tile([0.8, 0.0], (cfg["T"], 1))
            r = oracle.replan(P, x0, U, sc["obs"][:sc["H"]], rad)
            path = SC.nominal_path(x0, r["U_new"], sc["dt"])
            meets[mppi] += int((np.linalg.norm(path[:, :2] - c[None], axis=1) - (rad[0] + 0.1)).min() < 0)
            if not mppi:
                two += int(r["diag"]["n_clusters"] >= 2)
    assert two >= 20                       # the free rollouts split into two sides
    assert meets[False] == 0               # CE-MPPI's nominal commits to one side
    assert meets[True] >= 8                # MPPI's average runs into the disc
