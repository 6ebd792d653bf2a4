"""Python binding of the B300 CE-MPPI replanning library (``libcemppi.so``).

Argument marshalling only: every step of a replan runs in the library's CUDA
kernels; PyTorch supplies device memory and streams.  The C ABI is declared in
``include/ce_mppi.h``.  Importing this package does not need a GPU; creating a
planner does, and fails loudly when the CUDA library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads  # noqa: F401  (seeded input generators)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcemppi.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "ce_mppi.h")

DYN_DI, DYN_UNICYCLE, DYN_ARM, DYN_ARM12 = 0, 1, 2, 3
DIMS = {DYN_DI: (4, 2, 2), DYN_UNICYCLE: (3, 2, 2), DYN_ARM: (6, 6, 3),
        DYN_ARM12: (12, 6, 3)}  # (n, m, p)
MODES = {0: "nocol", 1: "allcol", 2: "allnoise", 3: "static", 4: "dynamic", 5: "mppi"}
BUF = dict(S=0, HIT=1, PN=2, EPS=3, IDXV=4, IDXC=5, Z=6, G=7, LABEL=8, W=9, HITJ=10, DBCYC=11)
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NO_MEMORY", 3: "CUDA", 4: "TIMEOUT", 5: "BUSY"}


class CeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ce_mppi {STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [
        ("dyn", C.c_int), ("K", C.c_int), ("T", C.c_int), ("dt", C.c_float),
        ("obs_dt", C.c_float), ("lam", C.c_float), ("dbscan_eps", C.c_float),
        ("min_pts", C.c_int), ("sigma", C.c_float * 6), ("u_min", C.c_float * 6),
        ("u_max", C.c_float * 6), ("goal", C.c_float * 16), ("w", C.c_float * 8),
        ("n_obs_max", C.c_int), ("hist_len", C.c_int), ("robot_radius", C.c_float),
        ("norm_eps", C.c_float), ("v_static_thresh", C.c_float), ("seed", C.c_ulonglong),
        ("ref_mode", C.c_int), ("check_j0", C.c_int), ("mppi_only", C.c_int),
        ("noise_regen", C.c_int), ("uf_limit", C.c_int),
    ]


class Diag(C.Structure):
    _fields_ = [
        ("mode", C.c_int), ("n_col", C.c_int), ("n_valid", C.c_int), ("n_clusters", C.c_int),
        ("sel_label", C.c_int), ("o_star", C.c_int), ("dynamic", C.c_int), ("status", C.c_int),
        ("S_min", C.c_float), ("pbar", C.c_float * 3), ("v_obs", C.c_float * 3),
        ("counter", C.c_ulonglong), ("col_tests", C.c_int),
    ]

    def as_dict(self) -> dict:
        return dict(mode=self.mode, n_col=self.n_col, n_valid=self.n_valid,
                    n_clusters=self.n_clusters, sel_label=self.sel_label, o_star=self.o_star,
                    dynamic=self.dynamic, status=self.status, S_min=self.S_min,
                    pbar=list(self.pbar), v_obs=list(self.v_obs), counter=self.counter,
                    col_tests=self.col_tests)


class Request(C.Structure):
    _fields_ = [
        ("x0", C.c_void_p), ("obs_hist", C.c_void_p), ("obs_radius", C.c_void_p),
        ("n_obs", C.c_int), ("obs_step", C.c_longlong), ("u_out", C.c_void_p),
        ("x_next", C.c_void_p), ("diag", C.c_void_p),
    ]


EXPORTS = (
    "ce_mppi_create", "ce_mppi_destroy", "ce_mppi_set_nominal", "ce_mppi_get_nominal",
    "ce_mppi_set_counter", "ce_mppi_get_counter", "ce_mppi_replan", "ce_mppi_check_inputs",
    "ce_mppi_replan_dev",
    "ce_mppi_batch_create", "ce_mppi_batch_run", "ce_mppi_batch_run_part", "ce_mppi_batch_run_part_ev", "ce_mppi_batch_config",
    "ce_mppi_batch_create_host", "ce_mppi_batch_run_host",
    "ce_mppi_batch_set_post_ctas", "ce_mppi_batch_profile",
    "ce_mppi_batch_destroy", "ce_mppi_peek",
    "ce_mppi_philox_dev", "ce_mppi_normals_dev", "ce_mppi_neg2ln_dev", "ce_mppi_dbscan_workspace_bytes",
    "ce_mppi_dbscan_dev", "ce_mppi_dbscan_noalloc_dev", "ce_mppi_arm_fk", "ce_mppi_last_error",
    "ce_mppi_server_create", "ce_mppi_server_destroy", "ce_mppi_server_open",
    "ce_mppi_server_close", "ce_mppi_server_submit", "ce_mppi_server_submit_many",
    "ce_mppi_server_poll",
    "ce_mppi_server_stats",
)

_lib = None


def lib() -> C.CDLL:
    """Load the CUDA library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i, f, u64 = C.c_void_p, C.c_int, C.c_float, C.c_ulonglong
        L.ce_mppi_create.argtypes = [C.POINTER(Params), vp, C.POINTER(vp)]
        L.ce_mppi_destroy.argtypes = [vp]
        L.ce_mppi_set_nominal.argtypes = [vp, vp]
        L.ce_mppi_get_nominal.argtypes = [vp, vp]
        L.ce_mppi_set_counter.argtypes = [vp, u64]
        L.ce_mppi_get_counter.argtypes = [vp, C.POINTER(u64)]
        L.ce_mppi_replan.argtypes = [vp, vp, vp, vp, i, vp, C.POINTER(Diag)]
        L.ce_mppi_check_inputs.argtypes = [C.POINTER(Params), vp, vp, vp, i]
        L.ce_mppi_replan_dev.argtypes = [vp, C.POINTER(Request)]
        L.ce_mppi_batch_create.argtypes = [C.POINTER(vp), C.POINTER(Request), i, vp, i, i,
                                           C.POINTER(vp)]
        L.ce_mppi_batch_run.argtypes = [vp]
        L.ce_mppi_batch_create_host.argtypes = [C.POINTER(vp), vp, i, vp, i, i, C.POINTER(vp)]
        L.ce_mppi_batch_run_host.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.ce_mppi_batch_run_part.argtypes = [vp, i, vp]
        L.ce_mppi_batch_run_part_ev.argtypes = [vp, i, vp, vp]
        L.ce_mppi_batch_config.argtypes = [vp, C.POINTER(i), C.POINTER(i)]
        L.ce_mppi_batch_set_post_ctas.argtypes = [vp, i]
        L.ce_mppi_batch_profile.argtypes = [vp, C.POINTER(C.c_float)]
        L.ce_mppi_batch_destroy.argtypes = [vp]
        L.ce_mppi_peek.argtypes = [vp, i, vp, C.c_size_t]
        L.ce_mppi_philox_dev.argtypes = [u64, u64, i, i, vp, vp]
        L.ce_mppi_normals_dev.argtypes = [u64, u64, i, i, vp, vp]
        L.ce_mppi_neg2ln_dev.argtypes = [vp, vp]
        L.ce_mppi_dbscan_workspace_bytes.argtypes = [i]
        L.ce_mppi_dbscan_workspace_bytes.restype = C.c_size_t
        L.ce_mppi_dbscan_dev.argtypes = [vp, i, i, i, f, i, vp, vp, vp, C.c_size_t, vp]
        L.ce_mppi_dbscan_noalloc_dev.argtypes = [vp, i, i, i, f, i, vp, vp, vp]
        L.ce_mppi_arm_fk.argtypes = [C.POINTER(C.c_double)] * 3
        L.ce_mppi_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("ce_mppi_last_error", "ce_mppi_dbscan_workspace_bytes"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise CeError(status, lib().ce_mppi_last_error().decode())


def arm_fk(q):
    """Frame origins O[7][3] and end-effector rotation R[3][3] (library helper)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    O = np.zeros((7, 3))
    R = np.zeros((3, 3))
    dp = C.POINTER(C.c_double)
    _check(lib().ce_mppi_arm_fk(q.ctypes.data_as(dp), O.ctypes.data_as(dp), R.ctypes.data_as(dp)))
    return O, R


def make_params(cfg: dict, n_obs_max: int) -> Params:
    """Fill ce_mppi_params from a workload config dict."""
    P = Params()
    P.dyn, P.K, P.T = cfg["dyn"], cfg["K"], cfg["T"]
    P.dt, P.obs_dt, P.lam = cfg["dt"], cfg.get("obs_dt", cfg["dt"]), cfg["lambda"]
    P.dbscan_eps, P.min_pts = cfg["dbscan_eps"], cfg["min_pts"]
    for name in ("sigma", "u_min", "u_max", "goal", "w"):
        arr = getattr(P, name)
        for k, v in enumerate(cfg[name]):
            arr[k] = v
    if "goal_q" in cfg:  # joint-space goal -> pose goal through the library's FK
        O, R = arm_fk(cfg["goal_q"])
        for k, v in enumerate(list(O[6]) + list(R.ravel())):
            P.goal[k] = v
    P.n_obs_max = n_obs_max
    P.hist_len = cfg["hist_len"]
    P.robot_radius, P.norm_eps = cfg["robot_radius"], cfg["norm_eps"]
    P.v_static_thresh, P.seed = cfg["v_static_thresh"], cfg["seed"]
    P.ref_mode, P.check_j0 = cfg.get("ref_mode", 0), cfg.get("check_j0", 0)
    P.mppi_only = cfg.get("mppi_only", 0)
    P.noise_regen = cfg.get("noise_regen", 0)
    P.uf_limit = cfg.get("uf_limit", 0)
    return P


def check_inputs(cfg: dict, x0, hist, radius, n_obs_max: int | None = None):
    """Host-side check of one replan's inputs (no GPU needed); raises CeError."""
    x0 = np.ascontiguousarray(x0, dtype=np.float32)
    hist = np.ascontiguousarray(hist, dtype=np.float32)
    radius = np.ascontiguousarray(radius, dtype=np.float32)
    n_obs = int(radius.shape[0])
    P = make_params(cfg, n_obs if n_obs_max is None else n_obs_max)
    _check(lib().ce_mppi_check_inputs(C.byref(P), x0.ctypes.data, hist.ctypes.data,
                                      radius.ctypes.data, n_obs))


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _ptr(t) -> int:
    return 0 if t is None else t.data_ptr()


class Planner:
    """One CE-MPPI controller instance (owns its device state)."""

    def __init__(self, cfg: dict, n_obs_max: int, stream=None):
        self.cfg = cfg
        self.n, self.m, self.p = DIMS[cfg["dyn"]]
        self.K, self.T = cfg["K"], cfg["T"]
        self.params = make_params(cfg, n_obs_max)
        self.stream = _stream_ptr(stream)
        h = C.c_void_p()
        _check(lib().ce_mppi_create(C.byref(self.params), C.c_void_p(self.stream), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().ce_mppi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_nominal(self, U):
        U = np.ascontiguousarray(U, dtype=np.float32)
        assert U.shape == (self.T, self.m)
        _check(lib().ce_mppi_set_nominal(self.h, U.ctypes.data))

    def get_nominal(self) -> np.ndarray:
        U = np.zeros((self.T, self.m), np.float32)
        _check(lib().ce_mppi_get_nominal(self.h, U.ctypes.data))
        return U

    def set_counter(self, c: int):
        _check(lib().ce_mppi_set_counter(self.h, c))

    def get_counter(self) -> int:
        c = C.c_ulonglong()
        _check(lib().ce_mppi_get_counter(self.h, C.byref(c)))
        return c.value

    def replan(self, x0, hist, radius):
        """Host-buffer replan (blocking): returns (u_out [T][m], diag dict)."""
        x0 = np.ascontiguousarray(x0, dtype=np.float32)
        hist = np.ascontiguousarray(hist, dtype=np.float32)
        radius = np.ascontiguousarray(radius, dtype=np.float32)
        n_obs = int(radius.shape[0])
        # the library reads exactly these many floats from each buffer
        if x0.size != self.n or hist.size != self.cfg["hist_len"] * n_obs * self.p:
            raise ValueError(f"x0 must hold {self.n} floats and hist "
                             f"{self.cfg['hist_len']} x {n_obs} x {self.p}")
        u = np.zeros((self.T, self.m), np.float32)
        dg = Diag()
        _check(lib().ce_mppi_replan(self.h, x0.ctypes.data, hist.ctypes.data, radius.ctypes.data,
                                    int(radius.shape[0]), u.ctypes.data, C.byref(dg)))
        return u, dg.as_dict()

    def replan_dev(self, x0, hist, radius, u_out=None, x_next=None, diag=None, obs_step=0):
        """Device-buffer replan queued on the planner's stream (torch tensors)."""
        q = Request(_ptr(x0), _ptr(hist), _ptr(radius), int(radius.shape[0]), obs_step,
                    _ptr(u_out), _ptr(x_next), _ptr(diag))
        _check(lib().ce_mppi_replan_dev(self.h, C.byref(q)))

    def peek(self, name: str) -> np.ndarray:
        K, p, TM = self.K, self.p, self.T * self.m
        shapes = dict(S=(K,), HIT=(K,), PN=(p, K), EPS=(K, self.T, self.m), IDXV=(K,),
                      IDXC=(K,), Z=(p, K), G=(p, K), LABEL=(K,), W=(K,), HITJ=(K,), DBCYC=(16,))
        ints = ("HIT", "IDXV", "IDXC", "LABEL", "HITJ")
        dt = np.int64 if name == "DBCYC" else (np.int32 if name in ints else np.float32)
        out = np.zeros(shapes[name], dt)
        _check(lib().ce_mppi_peek(self.h, BUF[name], out.ctypes.data, out.nbytes))
        return out


class Batch:
    """Several planners replanned together, one launch per stage (optionally a
    captured CUDA graph).  requests: list of dicts of torch device tensors with
    keys x0, hist, radius and optional u_out, x_next, diag, obs_step."""

    def __init__(self, planners, requests, stream=None, use_graph=True, n_branches=1):
        n = len(planners)
        self.planners = planners
        self.requests = requests  # keep tensors alive
        self.stream = _stream_ptr(stream)
        hs = (C.c_void_p * n)(*[pl.h.value for pl in planners])
        rq = (Request * n)()
        for i, r in enumerate(requests):
            rq[i] = Request(_ptr(r["x0"]), _ptr(r.get("hist")), _ptr(r.get("radius")),
                            int(r["radius"].shape[0]) if r.get("radius") is not None else 0,
                            int(r.get("obs_step", 0)), _ptr(r.get("u_out")),
                            _ptr(r.get("x_next")), _ptr(r.get("diag")))
        b = C.c_void_p()
        _check(lib().ce_mppi_batch_create(hs, rq, n, C.c_void_p(self.stream), int(use_graph),
                                          int(n_branches), C.byref(b)))
        self.b = b

    def run(self):
        _check(lib().ce_mppi_batch_run(self.b))

    def config(self) -> dict:
        """Branch count and clustering-kernel CTAs per instance (autotuned with
        n_branches=0; 0 CTAs: chosen per launch from the device occupancy)."""
        nb, pc = C.c_int(), C.c_int()
        _check(lib().ce_mppi_batch_config(self.b, C.byref(nb), C.byref(pc)))
        return dict(n_branches=nb.value, post_ctas=pc.value)

    def set_post_ctas(self, n: int):
        """Clustering-kernel CTAs per instance of later launches without a
        graph (0: from the device occupancy, as if the batch ran alone)."""
        _check(lib().ce_mppi_batch_set_post_ctas(self.b, int(n)))

    def run_part(self, part: int, stream=None, started=None):
        """Half a replan (0: tracks + rollouts, 1: clustering + update; 2: the
        tracks alone, 3: the rollouts alone) on stream.
        started (part 1): a torch.cuda.Event(enable_timing=False) that fires once
        every CTA of the clustering kernel has begun execution (the event must
        exist: recorded once before)."""
        s = 0 if stream is None else _stream_ptr(stream)
        ev = 0
        if started is not None:
            ev = started.cuda_event
            if not ev:
                raise ValueError("started: the event has not been created (record it once)")
        _check(lib().ce_mppi_batch_run_part_ev(self.b, int(part), C.c_void_p(s), C.c_void_p(ev)))

    STAGES = ("tracks", "rollout", "prune", "dbscan", "select", "update")

    def profile(self) -> dict:
        """One stage-by-stage replan with device times (ms) per stage."""
        ms = (C.c_float * 6)()
        _check(lib().ce_mppi_batch_profile(self.b, ms))
        return dict(zip(self.STAGES, list(ms)))

    def close(self):
        if getattr(self, "b", None):
            lib().ce_mppi_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostBatch:
    """Planners replanned together from host buffers (one packed copy each way
    per replan, inside the library): run(x0s, hists, radii) with packed numpy
    float32 arrays returns (u_outs, x_nexts) packed the same way."""

    def __init__(self, planners, n_obs, stream=None, use_graph=True, n_branches=1):
        n = len(planners)
        self.planners = planners
        self.stream = _stream_ptr(stream)
        hs = (C.c_void_p * n)(*[pl.h.value for pl in planners])
        self.n_obs = np.ascontiguousarray(n_obs, dtype=np.int32)
        b = C.c_void_p()
        _check(lib().ce_mppi_batch_create_host(hs, self.n_obs.ctypes.data, n,
                                               C.c_void_p(self.stream), int(use_graph),
                                               int(n_branches), C.byref(b)))
        self.b = b
        self.u_size = sum(pl.T * pl.m for pl in planners)
        self.x_size = sum(pl.n for pl in planners)
        self.diags = (Diag * n)()

    def run(self, x0s, hists, radii, u_out=None, x_next=None):
        x0s = np.ascontiguousarray(x0s, dtype=np.float32)
        hists = np.ascontiguousarray(hists, dtype=np.float32)
        radii = np.ascontiguousarray(radii, dtype=np.float32)
        u = np.empty(self.u_size, np.float32) if u_out is None else u_out
        x = np.empty(self.x_size, np.float32) if x_next is None else x_next
        _check(lib().ce_mppi_batch_run_host(self.b, x0s.ctypes.data, hists.ctypes.data,
                                            radii.ctypes.data, u.ctypes.data, x.ctypes.data,
                                            C.cast(self.diags, C.c_void_p)))
        return u, x

    def diag(self, i: int) -> dict:
        return self.diags[i].as_dict()

    def close(self):
        if getattr(self, "b", None):
            lib().ce_mppi_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def philox_dev(seed: int, counter: int, K: int, nblk: int, out, stream=None):
    _check(lib().ce_mppi_philox_dev(seed, counter, K, nblk, out.data_ptr(),
                                    C.c_void_p(_stream_ptr(stream))))


def normals_dev(seed: int, counter: int, K: int, n: int, out, stream=None):
    _check(lib().ce_mppi_normals_dev(seed, counter, K, n, out.data_ptr(),
                                     C.c_void_p(_stream_ptr(stream))))


def neg2ln_dev(out, stream=None):
    """-2 ln u for every uniform u = (m + 1/2) 2^-23 (out: 2^23 float32, device)."""
    _check(lib().ce_mppi_neg2ln_dev(out.data_ptr(), C.c_void_p(_stream_ptr(stream))))


def dbscan_dev(z, eps: float, min_pts: int, stream=None):
    """DBSCAN of device points z [p][n] (torch float32); returns (labels, M)."""
    import torch
    p, n = z.shape
    labels = torch.empty(max(n, 1), dtype=torch.int32, device=z.device)
    M = torch.zeros(1, dtype=torch.int32, device=z.device)
    nbytes = lib().ce_mppi_dbscan_workspace_bytes(n)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=z.device)
    _check(lib().ce_mppi_dbscan_dev(z.data_ptr(), n, z.stride(0), p, eps, min_pts,
                                    labels.data_ptr(), M.data_ptr(), ws.data_ptr(), nbytes,
                                    C.c_void_p(_stream_ptr(stream))))
    return labels[:n], M


def dbscan_noalloc_dev(z, eps: float, min_pts: int, stream=None):
    """DBSCAN of device points z [p][n] through the allocation-free entry point
    (fixed scratch inside the library, n <= 16384); returns (labels, M)."""
    import torch
    p, n = z.shape
    labels = torch.empty(max(n, 1), dtype=torch.int32, device=z.device)
    M = torch.zeros(1, dtype=torch.int32, device=z.device)
    _check(lib().ce_mppi_dbscan_noalloc_dev(z.data_ptr(), n, z.stride(0) if n else 0, p, eps,
                                            min_pts, labels.data_ptr(), M.data_ptr(),
                                            C.c_void_p(_stream_ptr(stream))))
    return labels[:n], M


class ServerParams(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_size_t), ("max_sessions", C.c_int),
                ("max_batch", C.c_int), ("n_streams", C.c_int), ("device", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("replans", C.c_ulonglong), ("batches", C.c_ulonglong),
                ("sessions_opened", C.c_ulonglong), ("sessions_rejected", C.c_ulonglong),
                ("superseded", C.c_ulonglong), ("mem_in_use", C.c_size_t),
                ("sessions_open", C.c_int), ("mean_batch", C.c_double),
                ("p50_latency_s", C.c_double), ("p99_latency_s", C.c_double),
                ("mean_latency_s", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_SERVER_BOUND = False


def _bind_server():
    global _SERVER_BOUND
    if _SERVER_BOUND:
        return
    L = lib()
    vp, i = C.c_void_p, C.c_int
    L.ce_mppi_server_create.argtypes = [C.POINTER(ServerParams), C.POINTER(vp)]
    L.ce_mppi_server_destroy.argtypes = [vp]
    L.ce_mppi_server_open.argtypes = [vp, C.POINTER(Params), C.POINTER(i)]
    L.ce_mppi_server_close.argtypes = [vp, i]
    L.ce_mppi_server_submit.argtypes = [vp, i, vp, vp, vp, i, C.POINTER(C.c_ulonglong)]
    L.ce_mppi_server_submit_many.argtypes = [vp, i, vp, vp, vp, vp, vp]
    L.ce_mppi_server_poll.argtypes = [vp, C.c_ulonglong, vp, C.POINTER(Diag),
                                      C.POINTER(C.c_double)]
    L.ce_mppi_server_stats.argtypes = [vp, C.POINTER(ServerStats), i]
    for n in ("create", "destroy", "open", "close", "submit", "submit_many", "poll", "stats"):
        getattr(L, "ce_mppi_server_" + n).restype = C.c_int
    _SERVER_BOUND = True


class Server:
    """Continuous-batching replan server (sessions resident on the device)."""

    def __init__(self, mem_budget_bytes: int, max_sessions: int = 4096, max_batch: int = 512,
                 n_streams: int = 3, device: int = 0):
        _bind_server()
        self.P = ServerParams(mem_budget_bytes, max_sessions, max_batch, n_streams, device)
        s = C.c_void_p()
        _check(lib().ce_mppi_server_create(C.byref(self.P), C.byref(s)))
        self.s = s
        self.shapes = {}

    def open(self, cfg: dict, n_obs_max: int):
        """Admit a session; returns its id, or None when the budget is exhausted."""
        P = make_params(cfg, n_obs_max)
        sid = C.c_int(-1)
        st = lib().ce_mppi_server_open(self.s, C.byref(P), C.byref(sid))
        if st == 2:
            return None
        _check(st)
        n, m, p = DIMS[cfg["dyn"]]
        self.shapes[sid.value] = (cfg["T"], m)
        return sid.value

    def close_session(self, sid: int):
        _check(lib().ce_mppi_server_close(self.s, sid))

    def submit(self, sid: int, x0, hist, radius, want_result: bool = True):
        x0 = np.ascontiguousarray(x0, dtype=np.float32)
        hist = np.ascontiguousarray(hist, dtype=np.float32)
        radius = np.ascontiguousarray(radius, dtype=np.float32)
        tk = C.c_ulonglong(0)
        _check(lib().ce_mppi_server_submit(self.s, sid, x0.ctypes.data, hist.ctypes.data,
                                           radius.ctypes.data, int(radius.shape[0]),
                                           C.byref(tk) if want_result else None))
        return tk.value if want_result else None

    def submit_many(self, sids, x0s, hists, radii, n_obs):
        """Bulk submit without tickets; packed float32 arrays, inputs in order."""
        sids = np.ascontiguousarray(sids, dtype=np.int32)
        x0s = np.ascontiguousarray(x0s, dtype=np.float32)
        hists = np.ascontiguousarray(hists, dtype=np.float32)
        radii = np.ascontiguousarray(radii, dtype=np.float32)
        n_obs = np.ascontiguousarray(n_obs, dtype=np.int32)
        _check(lib().ce_mppi_server_submit_many(self.s, int(sids.shape[0]), sids.ctypes.data,
                                                x0s.ctypes.data, hists.ctypes.data,
                                                radii.ctypes.data, n_obs.ctypes.data))

    def poll(self, ticket: int, sid: int):
        """(u_out, diag, latency_s) when done, else None."""
        T, m = self.shapes[sid]
        u = np.zeros((T, m), np.float32)
        dg = Diag()
        lat = C.c_double()
        st = lib().ce_mppi_server_poll(self.s, ticket, u.ctypes.data, C.byref(dg), C.byref(lat))
        if st == 5:
            return None
        _check(st)
        return u, dg.as_dict(), lat.value

    def stats(self, reset: bool = False) -> dict:
        out = ServerStats()
        _check(lib().ce_mppi_server_stats(self.s, C.byref(out), int(reset)))
        return out.as_dict()

    def close(self):
        if getattr(self, "s", None):
            lib().ce_mppi_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
