"""ctypes binding of the FP64 CE-MPPI oracle (``ce_mppi_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the oracle checks the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It shares no code with ``paper_2607_06499_b300``; the one module
both sides read is the seeded input generator ``paper_2607_06499_b300.workloads``,
which holds no arithmetic of the method.

Each wrapper takes and returns numpy arrays in the layouts documented in
``ce_mppi_oracle.h`` and names the paper passage it restates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ce_mppi_oracle.cpp")
_HDR = os.path.join(_HERE, "ce_mppi_oracle.h")
_LIB = os.path.join(_HERE, "libce_mppi_oracle.so")

MODE_NOCOL, MODE_ALLCOL, MODE_ALLNOISE, MODE_STATIC, MODE_DYNAMIC = range(5)
DIMS = {0: (4, 2, 2), 1: (3, 2, 2), 2: (6, 6, 3), 3: (12, 6, 3)}  # dyn -> (n, m, p)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP contraction off, see the .cpp header)."""
    stale = not os.path.exists(_LIB) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if force or stale:
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-pthread", _SRC, "-o", _LIB]
        subprocess.run(cmd, check=True)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("dyn", C.c_int), ("K", C.c_int), ("T", C.c_int),
        ("dt", C.c_double), ("obs_dt", C.c_double), ("lam", C.c_double),
        ("dbscan_eps", C.c_double), ("min_pts", C.c_int),
        ("sigma", C.c_double * 6), ("u_min", C.c_double * 6), ("u_max", C.c_double * 6),
        ("goal", C.c_double * 16), ("w", C.c_double * 8),
        ("hist_len", C.c_int), ("robot_radius", C.c_double), ("norm_eps", C.c_double),
        ("v_static_thresh", C.c_double), ("seed", C.c_uint64), ("counter", C.c_uint64),
        ("ref_mode", C.c_int), ("check_j0", C.c_int), ("mppi_only", C.c_int),
    ]


class Diag(C.Structure):
    _fields_ = [
        ("mode", C.c_int), ("n_col", C.c_int), ("n_valid", C.c_int),
        ("n_clusters", C.c_int), ("sel_label", C.c_int), ("o_star", C.c_int),
        ("dynamic", C.c_int), ("pbar", C.c_double * 3), ("v_obs", C.c_double * 3),
        ("S_min", C.c_double),
    ]


def make_params(cfg: dict, counter: int = 0) -> Params:
    """Fill the oracle's own parameter struct from a workload config dict."""
    P = Params()
    P.dyn = cfg["dyn"]
    P.K, P.T = cfg["K"], cfg["T"]
    P.dt = cfg["dt"]
    P.obs_dt = cfg.get("obs_dt", cfg["dt"])
    P.lam = cfg["lambda"]
    P.dbscan_eps = cfg["dbscan_eps"]
    P.min_pts = cfg["min_pts"]
    for name in ("sigma", "u_min", "u_max", "goal", "w"):
        arr = getattr(P, name)
        for i, v in enumerate(cfg[name]):
            arr[i] = v
    if "goal_q" in cfg:  # arm goal given in joint space: pose from the oracle's FK
        O, R = arm_fk(np.asarray(cfg["goal_q"], float))
        for i, v in enumerate(list(O[6]) + list(R.ravel())):
            P.goal[i] = v
    P.hist_len = cfg["hist_len"]
    P.robot_radius = cfg["robot_radius"]
    P.norm_eps = cfg["norm_eps"]
    P.v_static_thresh = cfg["v_static_thresh"]
    P.seed = cfg["seed"]
    P.counter = counter
    P.ref_mode = cfg.get("ref_mode", 0)
    P.check_j0 = cfg.get("check_j0", 0)
    P.mppi_only = cfg.get("mppi_only", 0)
    return P


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, u32, u64 = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_uint32), C.c_uint64
        P = C.POINTER(Params)
        _lib.orc_philox4x32_10.argtypes = [u32, u32, u32]
        _lib.orc_normals.argtypes = [u64, u64, C.c_int, C.c_int, d]
        _lib.orc_obstacle_velocity.argtypes = [P, d, C.c_int, d]
        _lib.orc_tracks.argtypes = [P, d, C.c_int, d]
        _lib.orc_step.argtypes = [P, d, d, d]
        _lib.orc_task_pos.argtypes = [P, d, d]
        _lib.orc_arm_fk.argtypes = [d, d, d]
        _lib.orc_robot_points.argtypes = [P, d, d]
        _lib.orc_rollouts.argtypes = [P, d, d, d, d, C.c_int, d, i, i, i, d, d, d, d]
        _lib.orc_prune.argtypes = [i, C.c_int, i, i, i, i]
        _lib.orc_reference_point.argtypes = [P, d, d, d, C.c_int, i, C.c_int, i, d, d]
        _lib.orc_features.argtypes = [P, d, d, i, C.c_int, d, d, d]
        _lib.orc_dbscan.argtypes = [C.POINTER(C.c_float), C.c_int, C.c_int, C.c_float,
                                    C.c_int, i]
        _lib.orc_select.argtypes = [P, i, C.c_int, i, d, d, C.c_int, d, i, i, d, d]
        _lib.orc_update.argtypes = [P, d, d, d, i, C.c_int, d, d]
        _lib.orc_update.restype = C.c_double
        _lib.orc_shift.argtypes = [P, d, d]
        _lib.orc_replan.argtypes = [P, d, d, d, d, C.c_int, d, C.POINTER(Diag),
                                    d, i, i, d, d, d, i, d]
        pd = C.POINTER(d)
        _lib.orc_replan_many.argtypes = [P, pd, pd, pd, pd, i, C.c_int, C.c_int, pd]
        _lib.orc_replan_many.restype = C.c_double
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block function (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    p = C.POINTER(C.c_uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(p), k.ctypes.data_as(p), out.ctypes.data_as(p))
    return out


def normals(seed: int, counter: int, k: int, n: int) -> np.ndarray:
    """Standard normals of rollout k (Sec. II-A, eps ~ N(0, Sigma))."""
    out = np.zeros(n)
    lib().orc_normals(seed, counter, k, n, _d(out))
    return out


def obstacle_velocity(P: Params, hist) -> np.ndarray:
    """Eq. 17 obstacle velocity estimate, literal sum of differences."""
    hist = _f64(hist)
    n_obs, p = hist.shape[1], hist.shape[2]
    v = np.zeros((n_obs, p))
    lib().orc_obstacle_velocity(C.byref(P), _d(hist), n_obs, _d(v))
    return v


def tracks(P: Params, hist) -> np.ndarray:
    hist = _f64(hist)
    n_obs, p = hist.shape[1], hist.shape[2]
    out = np.zeros((P.T + 1, n_obs, p))
    lib().orc_tracks(C.byref(P), _d(hist), n_obs, _d(out))
    return out


def step(P: Params, x, u) -> np.ndarray:
    x, u = _f64(x), _f64(u)
    out = np.zeros_like(x)
    lib().orc_step(C.byref(P), _d(x), _d(u), _d(out))
    return out


def task_pos(P: Params, x) -> np.ndarray:
    x = _f64(x)
    out = np.zeros(3)
    lib().orc_task_pos(C.byref(P), _d(x), _d(out))
    return out[: DIMS[P.dyn][2]]


def arm_fk(q):
    """Standard DH chain; returns frame origins O[7][3] and EE rotation R[3][3]."""
    q = _f64(q)
    O = np.zeros((7, 3))
    R = np.zeros((3, 3))
    lib().orc_arm_fk(_d(q), _d(O), _d(R))
    return O, R


def robot_points(P: Params, x) -> np.ndarray:
    x = _f64(x)
    out = np.zeros((24, 3))
    n = lib().orc_robot_points(C.byref(P), _d(x), _d(out))
    return out[:n]


def rollouts(P: Params, x0, U, trk, radius, want_traj: bool = False) -> dict:
    """Algorithm 1 [Rollouts] (Eq. 3-5, Eq. 8)."""
    n, m, p = DIMS[P.dyn]
    K, T = P.K, P.T
    x0, U, trk, radius = _f64(x0), _f64(U), _f64(trk), _f64(radius)
    n_obs = radius.shape[0]
    r = dict(S=np.zeros(K), col=np.zeros(K, np.int32), hit=np.zeros(K, np.int32),
             hit_j=np.zeros(K, np.int32), pN=np.zeros((K, p)), eps=np.zeros((K, T, m)),
             min_abs_clear=np.zeros(K))
    traj = np.zeros((K, T + 1, n)) if want_traj else None
    lib().orc_rollouts(C.byref(P), _d(x0), _d(U), _d(trk), _d(radius), n_obs,
                       _d(r["S"]), _i(r["col"]), _i(r["hit"]), _i(r["hit_j"]), _d(r["pN"]),
                       _d(r["eps"]), _d(r["min_abs_clear"]),
                       _d(traj) if traj is not None else None)
    if traj is not None:
        r["traj"] = traj
    return r


def prune(col):
    """Eq. 9-10: V and C_col in ascending k."""
    col = _i32(col)
    K = col.shape[0]
    idxV = np.zeros(K, np.int32)
    idxC = np.zeros(K, np.int32)
    nV = C.c_int()
    nC = C.c_int()
    lib().orc_prune(_i(col), K, _i(idxV), C.byref(nV), _i(idxC), C.byref(nC))
    return idxV[: nV.value], idxC[: nC.value]


def reference_point(P: Params, x0, trk, radius, idxC, hit, pN):
    """Eq. 11 over the colliding rollouts near the closest obstacle."""
    p = DIMS[P.dyn][2]
    x0, trk, radius, pN = _f64(x0), _f64(trk), _f64(radius), _f64(pN)
    idxC, hit = _i32(idxC), _i32(hit)
    pbar = np.zeros(3)
    o = lib().orc_reference_point(C.byref(P), _d(x0), _d(trk), _d(radius), radius.shape[0],
                                  _i(idxC), idxC.shape[0], _i(hit), _d(pN), _d(pbar))
    return o, pbar[:p]


def features(P: Params, x0, pbar, idxV, pN):
    """Eq. 12-13 (z) and Eq. 15 (g) for k in V."""
    p = DIMS[P.dyn][2]
    x0, pN, idxV = _f64(x0), _f64(pN), _i32(idxV)
    pb = np.zeros(3)
    pb[:p] = pbar
    nV = idxV.shape[0]
    z = np.zeros((nV, p))
    g = np.zeros((nV, p))
    lib().orc_features(C.byref(P), _d(x0), _d(pb), _i(idxV), nV, _d(pN), _d(z), _d(g))
    return z, g


def dbscan(z, eps: float, min_pts: int):
    """DBSCAN with the FP32 neighbour predicate; returns (labels, M)."""
    zf = np.ascontiguousarray(z, dtype=np.float32)
    n, p = zf.shape
    eps2 = np.float32(eps) * np.float32(eps)  # FP32 product of the FP32 radius
    labels = np.zeros(n, np.int32)
    M = lib().orc_dbscan(zf.ctypes.data_as(C.POINTER(C.c_float)), n, p, C.c_float(eps2),
                         min_pts, _i(labels))
    return labels, M


def select(P: Params, labels, idxV, S, g, M, v_obs):
    """Cluster statistics and selection (Eq. 14, 16, 18)."""
    p = DIMS[P.dyn][2]
    labels, idxV, S, g = _i32(labels), _i32(idxV), _f64(S), _f64(g)
    v = np.zeros(3)
    v[:p] = v_obs
    dyn = C.c_int()
    cnt = np.zeros(max(M, 1), np.int32)
    Sbar = np.zeros(max(M, 1))
    vhat = np.zeros((max(M, 1), p))
    cs = lib().orc_select(C.byref(P), _i(labels), labels.shape[0], _i(idxV), _d(S), _d(g), M,
                          _d(v), C.byref(dyn), _i(cnt), _d(Sbar), _d(vhat))
    return dict(sel=cs, dynamic=dyn.value, cnt=cnt[:M], Sbar=Sbar[:M], vhat=vhat[:M])


def update(P: Params, U, S, eps, members):
    """Eq. 6-7 / Eq. 19-20 softmin-weighted update over a member list."""
    U, S, eps, members = _f64(U), _f64(S), _f64(eps), _i32(members)
    w = np.zeros(P.K)
    U_new = np.zeros_like(U)
    smin = lib().orc_update(C.byref(P), _d(U), _d(S), _d(eps), _i(members), members.shape[0],
                            _d(w), _d(U_new))
    return U_new, w, smin


def shift(P: Params, U_new):
    U_new = _f64(U_new)
    out = np.zeros_like(U_new)
    lib().orc_shift(C.byref(P), _d(U_new), _d(out))
    return out


def replan(P: Params, x0, U, hist, radius) -> dict:
    """One CE-MPPI iteration (Algorithm 1) with every intermediate result."""
    n, m, p = DIMS[P.dyn]
    K, T = P.K, P.T
    x0, U, hist, radius = _f64(x0), _f64(U), _f64(hist), _f64(radius)
    n_obs = radius.shape[0]
    r = dict(U_new=np.zeros((T, m)), S=np.zeros(K), col=np.zeros(K, np.int32),
             hit=np.zeros(K, np.int32), pN=np.zeros((K, p)), eps=np.zeros((K, T, m)),
             min_abs_clear=np.zeros(K), labels=np.zeros(K, np.int32), w=np.zeros(K))
    dg = Diag()
    lib().orc_replan(C.byref(P), _d(x0), _d(U), _d(hist), _d(radius), n_obs, _d(r["U_new"]),
                     C.byref(dg), _d(r["S"]), _i(r["col"]), _i(r["hit"]), _d(r["pN"]),
                     _d(r["eps"]), _d(r["min_abs_clear"]), _i(r["labels"]), _d(r["w"]))
    r["diag"] = dict(mode=dg.mode, n_col=dg.n_col, n_valid=dg.n_valid,
                     n_clusters=dg.n_clusters, sel_label=dg.sel_label, o_star=dg.o_star,
                     dynamic=dg.dynamic, pbar=np.array(dg.pbar[:p]),
                     v_obs=np.array(dg.v_obs[:p]), S_min=dg.S_min)
    r["labels"] = r["labels"][: dg.n_valid]
    return r


def replan_many(Ps, x0s, Us, hists, radii, n_threads: int):
    """Independent replans on n_threads host threads; returns (U_news, seconds)."""
    n = len(Ps)
    Parr = (Params * n)(*Ps)
    keep = [[_f64(a) for a in arrs] for arrs in (x0s, Us, hists, radii)]
    outs = [np.zeros_like(u) for u in keep[1]]
    pd = C.POINTER(C.c_double)

    def ptrs(arrs):
        return (pd * n)(*[_d(a) for a in arrs])

    nob = np.array([r.shape[0] for r in keep[3]], np.int32)
    secs = lib().orc_replan_many(Parr, ptrs(keep[0]), ptrs(keep[1]), ptrs(keep[2]),
                                 ptrs(keep[3]), _i(nob), n, n_threads, ptrs(outs))
    return outs, secs
