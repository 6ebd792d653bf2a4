"""Stage-by-stage parity of one GPU replan against the FP64 oracle, shared by
the GPU test modules, and the report of every FP32-vs-FP64 error they measure.

Pass criteria:
  * Philox words, pruning lists, DBSCAN partitions: bit-exact;
  * collision flags, first hit: exact wherever the oracle's smallest
    |clearance| of the rollout exceeds the band BAND (1e-5 m);
  * costs, terminal positions, perturbations, reference point, features and the
    updated nominal: relative error <= 1e-4 against the denominators stated
    at each check.

Each comparison is also recorded under max(|ref|, 1e-3 scale) (scale = sigma
for controls, 1 otherwise), and written as one JSON line per replan to the
file named by $PARITY_REPORT when it is set.
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2607_06499_b300 as pkg

BAND = 1e-5
RTOL = 1e-4

# Every stage comparison of the GPU test modules, written as JSON to $PARITY_REPORT
# (when set) at the end of the module: the FP32-vs-FP64 error of each result.
REPORT = []


def _current_case():
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]


def parity_report_fixture():
    """A module-scoped autouse fixture that appends the module's records to
    $PARITY_REPORT when the module's tests are done."""
    @pytest.fixture(scope="module", autouse=True)
    def _fixture():
        yield
        path = os.environ.get("PARITY_REPORT")
        if path and REPORT:
            with open(path, "a") as f:
                for r in REPORT:
                    f.write(json.dumps(r) + "\n")
        REPORT.clear()
    return _fixture


def _rel(a, ref, floor):
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - ref) / np.maximum(np.abs(ref), floor)))


def check_outputs(cfg, x0, U0, hist, radius, counter, u, diag, out, report=None, case=None):
    """Stage-by-stage parity of one GPU replan (its inputs x0, U0, hist,
    radius, counter; its outputs u, diag and the peeked buffers `out`) against
    the oracle.  Without out["EPS"] (noise regeneration: the GPU stores no
    perturbations) the oracle's own eps' enters the update check, which then
    covers the regenerated perturbations too.  Records every error under the
    tolerance's own denominator and under max(|ref|, 1e-3 scale) (scale =
    sigma for controls, 1 otherwise) in REPORT."""
    n, m, p = pkg.DIMS[cfg["dyn"]]
    K = cfg["K"]
    x0 = np.asarray(x0, np.float64)
    U0 = np.asarray(U0, np.float64)
    assert diag["status"] == 0
    P = oracle.make_params(cfg, counter=counter)
    trk = oracle.tracks(P, hist)
    ref = oracle.rollouts(P, x0, U0, trk, radius)
    sig = np.array(cfg["sigma"])
    # ---- rollouts: flags outside the band, first hit, costs, positions, perturbations
    col_g = out["HIT"] >= 0
    col_o = ref["col"] == 1
    clear = ref["min_abs_clear"] > BAND
    assert not np.any((col_g != col_o) & clear), "collision flag differs outside the band"
    assert np.array_equal(out["HIT"][clear], ref["hit"][clear])
    assert np.array_equal(out["HITJ"][clear], ref["hit_j"][clear])
    errS = _rel(out["S"][clear], ref["S"][clear], 1.0)
    errP = _rel(out["PN"].T[clear], ref["pN"][clear], 1.0)
    errs = dict(S=errS, pN=errP)
    e8 = dict(S=_rel(out["S"][clear], ref["S"][clear], 1e-3),
              pN=_rel(out["PN"].T[clear], ref["pN"][clear], 1e-3))
    band = int(np.count_nonzero(~clear))
    if "EPS" in out:
        # eps' = u - U with u = U + eps' held in FP32: its rounding scales with
        # |U| + |eps'| (the magnitude of the applied control); the normal
        # behind it carries an absolute error up to 4.6e-6 (the Box-Muller
        # angle's sine and cosine from the special-function unit, 2^-21.41 +
        # pi 2^-24, times the radius <= 5.77, plus a few ulp of the radius),
        # i.e. sigma * 4.6e-6, so the scale is floored at 0.05 sigma
        sg = sig[None, None, :]
        scaleE = np.maximum(np.abs(U0)[None] + np.abs(ref["eps"]), 0.05 * sg)
        errs["eps"] = float(np.max(np.abs(out["EPS"] - ref["eps"]) / scaleE))
        e8["eps"] = float(np.max(np.abs(out["EPS"] - ref["eps"]) /
                                 np.maximum(np.abs(ref["eps"]), 1e-3 * sg)))
        assert errs["eps"] < RTOL, errs
        eps_u = out["EPS"].astype(np.float64)
    else:
        eps_u = ref["eps"]
    assert errS < RTOL and errP < RTOL, errs
    # ---- pruning (bit-exact on the GPU's flags)
    idxV, idxC = oracle.prune(col_g.astype(np.int32))
    nV, nC = diag["n_valid"], diag["n_col"]
    assert (nV, nC) == (len(idxV), len(idxC))
    assert np.array_equal(out["IDXV"][:nV], idxV) and np.array_equal(out["IDXC"][:nC], idxC)
    S_g = out["S"].astype(np.float64)
    pN_g = out["PN"].T.astype(np.float64)
    near_tie = False
    if cfg.get("mppi_only", 0):
        assert diag["mode"] == 5          # standard MPPI over all K
        members = np.arange(K, dtype=np.int32)
    elif nC == 0 or nV == 0:
        assert diag["mode"] == (0 if nC == 0 else 1)
        members = np.arange(K, dtype=np.int32)
    else:
        # ---- reference point and features (GPU flags and positions handed in)
        o_star, pbar = oracle.reference_point(P, x0, trk, radius, idxC, out["HIT"], pN_g)
        assert o_star == diag["o_star"]
        errs["pbar"] = _rel(np.array(diag["pbar"][:p]), pbar, 1.0)
        e8["pbar"] = _rel(np.array(diag["pbar"][:p]), pbar, 1e-3)
        assert errs["pbar"] < RTOL
        z_ref, g_ref = oracle.features(P, x0, pbar, idxV, pN_g)
        dnorm = np.linalg.norm(pN_g[idxV] - pbar[None, :], axis=1)
        tol_z = RTOL + 4e-6 / np.maximum(dnorm, 1e-9)
        z_g = out["Z"][:, :nV].T.astype(np.float64)
        g_g = out["G"][:, :nV].T.astype(np.float64)
        assert np.all(np.abs(z_g - z_ref).max(axis=1) <= tol_z)
        enorm = np.linalg.norm(pN_g[idxV] - oracle.task_pos(P, x0)[None, :], axis=1)
        tol_g = RTOL + 4e-6 / np.maximum(enorm, 1e-9)
        assert np.all(np.abs(g_g - g_ref).max(axis=1) <= tol_g)
        if nV:
            errs["z"] = float(np.max(np.abs(z_g - z_ref)))   # (unit vectors: absolute)
            errs["g"] = float(np.max(np.abs(g_g - g_ref)))
            e8["z"] = _rel(z_g, z_ref, 1e-3)
            e8["g"] = _rel(g_g, g_ref, 1e-3)
        # ---- DBSCAN on the GPU's own features: bit-exact
        lab_o, M_o = oracle.dbscan(out["Z"][:, :nV].T, cfg["dbscan_eps"], cfg["min_pts"])
        assert M_o == diag["n_clusters"]
        assert np.array_equal(lab_o, out["LABEL"][:nV])
        if M_o == 0:
            assert diag["mode"] == 2
            members = idxV
        else:
            v_obs = oracle.obstacle_velocity(P, hist)[o_star]
            sel = oracle.select(P, lab_o, idxV, S_g, g_g, M_o, v_obs)
            assert diag["dynamic"] == sel["dynamic"]
            assert diag["mode"] == (4 if sel["dynamic"] else 3)
            crit = sel["Sbar"] if not sel["dynamic"] else sel["vhat"] @ (v_obs / (np.linalg.norm(v_obs) + 1e-6))
            srt = np.sort(crit)
            near_tie = len(srt) > 1 and (srt[1] - srt[0]) <= 1e-5 * max(1.0, abs(srt[0]))
            if not near_tie:
                assert diag["sel_label"] == sel["sel"]
            members = idxV[lab_o == diag["sel_label"]]
    # ---- update (GPU costs and selection handed in)
    U_ref, w_ref, smin = oracle.update(P, U0, S_g, eps_u, members)
    # relative to the magnitude of the terms of U + sum_k w_k eps'_k (the
    # condition of the weighted sum), floored at 1e-3 sigma
    sig2 = sig[None, :]
    scaleU = np.maximum(np.abs(U0) + np.einsum("k,kjd->jd", w_ref, np.abs(eps_u)), 1e-3 * sig2)
    scaleU = np.maximum(scaleU, np.abs(U_ref))
    errs["U"] = float(np.max(np.abs(u - U_ref) / scaleU))
    e8["U"] = float(np.max(np.abs(u - U_ref) / np.maximum(np.abs(U_ref), 1e-3 * sig2)))
    errs["w"] = float(np.max(np.abs(out["W"] - w_ref)))
    e8["w"] = errs["w"]
    assert errs["U"] < RTOL, errs
    assert errs["w"] < 1e-5 + 1e-4 * w_ref.max()
    assert abs(out["W"].sum() - 1.0) < 1e-5
    # ---- receding-horizon shift and counter
    np.testing.assert_array_equal(out["nominal_after"], np.vstack([u[1:], u[-1:]]))
    assert out["counter_after"] == counter + 1 and diag["counter"] == counter
    if report is not None:
        report.update(errs)
    REPORT.append(dict(case=case or _current_case(), mode=pkg.MODES.get(diag["mode"], diag["mode"]),
                       K=K, T=cfg["T"], n_col=int(nC), n_clusters=int(diag["n_clusters"]),
                       nnz_w=int(np.count_nonzero(out["W"])), band=band, near_tie=bool(near_tie),
                       err=errs, err_8c=e8))
    return diag, errs


