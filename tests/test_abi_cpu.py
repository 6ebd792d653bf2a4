"""CPU checks of the C ABI: the library loads without a GPU, exports every
entry point the header declares, rejects bad parameters before any launch, and
its host FK helper agrees with the oracle's."""
import ctypes as C
import math
import re

import numpy as np
import pytest

import oracle
import paper_2607_06499_b300 as pkg
from paper_2607_06499_b300 import workloads as W


def _declared():
    src = open(pkg.HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ce_mppi_\w+)\s*\(", src)))


def test_header_declares_every_binding_export():
    assert set(_declared()) == set(pkg.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = pkg.lib()
    for name in _declared():
        assert hasattr(L, name), name


def _params(**kw):
    sc = W.make("unicycle", seed=0, K=256)
    P = pkg.make_params(sc["cfg"], 50)
    for k, v in kw.items():
        if k in ("sigma", "u_min", "u_max"):
            arr = getattr(P, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(P, k, v)
    return P


@pytest.mark.parametrize("kw,msg", [
    (dict(dyn=5), "dyn"), (dict(K=0), "K must"), (dict(T=0), "T must"), (dict(T=1000), "T must"),
    (dict(dt=0.0), "dt"), (dict(dt=float("nan")), "dt"), (dict(lam=0.0), "lambda"),
    (dict(dbscan_eps=0.0), "dbscan_eps"), (dict(min_pts=0), "min_pts"),
    (dict(sigma=[-1.0, 0.5]), "sigma"), (dict(u_min=[3.0, -2.0]), "u_min"),
    (dict(n_obs_max=100000), "n_obs_max"), (dict(hist_len=0), "hist_len"),
    (dict(norm_eps=0.0), "norm_eps"), (dict(ref_mode=3), "ref_mode"),
    (dict(n_obs_max=4000, T=100), "shared memory"), (dict(noise_regen=2), "noise_regen"),
    (dict(check_j0=-1), "check_j0"), (dict(dyn=4), "dyn"),
])
def test_invalid_parameters_rejected_before_launch(kw, msg):
    P = _params(**kw)
    h = C.c_void_p()
    st = pkg.lib().ce_mppi_create(C.byref(P), None, C.byref(h))
    assert st == 1 and not h.value
    assert msg in pkg.lib().ce_mppi_last_error().decode()


def test_dbscan_grid_limit_for_3d_features():
    sc = W.make("arm", seed=0, K=64)
    P = pkg.make_params(sc["cfg"], 20)
    P.dbscan_eps = 0.1
    h = C.c_void_p()
    assert pkg.lib().ce_mppi_create(C.byref(P), None, C.byref(h)) == 1
    assert "grid" in pkg.lib().ce_mppi_last_error().decode()


def test_arm_fk_helper_matches_oracle():
    rng = np.random.default_rng(0)
    for _ in range(10):
        q = rng.uniform(-math.pi, math.pi, 6)
        O1, R1 = pkg.arm_fk(q)
        O2, R2 = oracle.arm_fk(q)
        np.testing.assert_allclose(O1, O2, atol=1e-12)
        np.testing.assert_allclose(R1, R2, atol=1e-12)


def test_null_arguments_rejected():
    L = pkg.lib()
    assert L.ce_mppi_create(None, None, None) == 1
    assert L.ce_mppi_replan(None, None, None, None, 0, None, None) == 1
    assert L.ce_mppi_batch_create(None, None, 0, None, 0, 1, None) == 1
    assert L.ce_mppi_dbscan_dev(None, 4, 4, 5, 0.3, 3, None, None, None, 0, None) == 1


def test_binding_structs_match_the_header(tmp_path):
    """sizeof / offsetof of the ABI structs as compiled by gcc from
    include/ce_mppi.h equal the ctypes mirrors of the binding."""
    import subprocess
    src = tmp_path / "sizes.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "ce_mppi.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(ce_mppi_params),"
        " sizeof(ce_mppi_diag), sizeof(ce_mppi_request), offsetof(ce_mppi_params, seed),"
        " offsetof(ce_mppi_diag, counter), offsetof(ce_mppi_diag, col_tests),"
        " offsetof(ce_mppi_request, obs_step));return 0;}\n")
    exe = tmp_path / "sizes"
    inc = pkg.HEADER.rsplit("/", 1)[0]
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [C.sizeof(pkg.Params), C.sizeof(pkg.Diag), C.sizeof(pkg.Request),
            pkg.Params.seed.offset, pkg.Diag.counter.offset, pkg.Diag.col_tests.offset,
            pkg.Request.obs_step.offset]
    assert got == want


def test_batch_run_part_rejects_bad_arguments():
    L = pkg.lib()
    assert L.ce_mppi_batch_run_part(None, 0, None) == 1
    assert "NULL" in L.ce_mppi_last_error().decode()
    assert L.ce_mppi_batch_set_post_ctas(None, 4) == 1
    assert "NULL" in L.ce_mppi_last_error().decode()
    assert L.ce_mppi_batch_run_part_ev(None, 1, None, None) == 1
    assert "NULL" in L.ce_mppi_last_error().decode()


def test_neg2ln_stage_rejects_null_output():
    L = pkg.lib()
    assert L.ce_mppi_neg2ln_dev(None, None) == 1
    assert "NULL" in L.ce_mppi_last_error().decode()


def test_twelve_d_arm_dims_and_parameters_accepted_by_validation():
    # dyn 3 passes the host-side checks up to the device allocation (no GPU
    # here: creation then fails with a CUDA or memory status, not INVALID_ARG)
    sc = W.make("arm12", seed=0, K=64)
    assert pkg.DIMS[sc["cfg"]["dyn"]] == (12, 6, 3)
    P = pkg.make_params(sc["cfg"], 20)
    h = C.c_void_p()
    st = pkg.lib().ce_mppi_create(C.byref(P), None, C.byref(h))
    assert st != 1, pkg.lib().ce_mppi_last_error().decode()


def test_host_inputs_checked_without_a_gpu():
    """ce_mppi_check_inputs (the check ce_mppi_replan and the server's submit
    calls run before copying anything) refuses NaN and infinite inputs."""
    sc = W.make("unicycle", seed=0, K=256)
    cfg, hist, rad = sc["cfg"], W.history(sc, 0), sc["radius"]
    pkg.check_inputs(cfg, sc["x0"], hist, rad)          # valid inputs pass
    bad_cases = []
    x = sc["x0"].copy(); x[2] = np.nan; bad_cases.append((x, hist, rad, "x0"))
    x = sc["x0"].copy(); x[0] = np.inf; bad_cases.append((x, hist, rad, "x0"))
    h = hist.copy(); h[4, 17, 1] = np.nan; bad_cases.append((sc["x0"], h, rad, "obs_hist"))
    h = hist.copy(); h[0, 0, 0] = -np.inf; bad_cases.append((sc["x0"], h, rad, "obs_hist"))
    r = rad.copy(); r[3] = np.nan; bad_cases.append((sc["x0"], hist, r, "obs_radius"))
    r = rad.copy(); r[3] = -0.1; bad_cases.append((sc["x0"], hist, r, "obs_radius"))
    for x, h, r, what in bad_cases:
        with pytest.raises(pkg.CeError) as e:
            pkg.check_inputs(cfg, x, h, r)
        assert e.value.status == 1 and what in str(e.value)
    with pytest.raises(pkg.CeError) as e:                 # more obstacles than the planner holds
        pkg.check_inputs(cfg, sc["x0"], hist, rad, n_obs_max=10)
    assert "n_obs" in str(e.value)
    P = pkg.make_params(cfg, 50)
    P.lam = float("nan")                                   # the parameters are checked too
    st = pkg.lib().ce_mppi_check_inputs(C.byref(P), sc["x0"].astype(np.float32).ctypes.data,
                                         None, None, 0)
    assert st == 1 and "lambda" in pkg.lib().ce_mppi_last_error().decode()
