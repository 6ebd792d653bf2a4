"""The allocation-free DBSCAN entry point (ce_mppi_dbscan_noalloc_dev) against
the workspace entry point (ce_mppi_dbscan_dev): callers that may not allocate
device memory get the same labels from the library's fixed scratch.  Two calls
in a row, with different inputs, must each match bit for bit (the labels are
integers); sizes beyond the fixed scratch are refused.  Collected last so that
a run stopping at the first failure has run every other test first."""
import ctypes as C

import numpy as np
import pytest

import paper_2607_06499_b300 as pkg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _points(seed, n, p):
    rng = np.random.default_rng(seed)
    if p == 2:
        c = rng.uniform(0, 2 * np.pi, size=3)
        ang = c[rng.integers(0, 3, n)] + rng.normal(scale=0.15, size=n)
        z = np.stack([np.cos(ang), np.sin(ang)], 1) * rng.uniform(0.9, 0.999, (n, 1))
    else:
        z = rng.normal(size=(n, 3))
        z /= np.linalg.norm(z, axis=1, keepdims=True)
        z[: n // 2] = np.clip(z[0] + 0.1 * rng.normal(size=(n // 2, 3)), -1, 1)
    return torch.from_numpy(np.ascontiguousarray(z.T.astype(np.float32))).cuda()


@pytest.mark.parametrize("p,eps,mp", [(2, 0.25, 20), (3, 0.2, 16)])
def test_noalloc_matches_workspace_entry_point_twice(p, eps, mp):
    # calls in a row, largest first: each later call finds the previous,
    # larger call's data in the shared scratch and must not depend on it
    for call, (seed, n) in enumerate([(11, 16384), (12, 5000), (13, 700)]):
        z = _points(seed + p, n, p)
        lab_ref, M_ref = pkg.dbscan_dev(z, eps, mp)
        lab, M = pkg.dbscan_noalloc_dev(z, eps, mp)
        torch.cuda.synchronize()
        assert int(M.item()) == int(M_ref.item()) > 0, call
        assert torch.equal(lab, lab_ref), call


def test_noalloc_rejects_more_points_than_the_scratch():
    z = torch.zeros((2, 16385), dtype=torch.float32, device="cuda")
    labels = torch.empty(16385, dtype=torch.int32, device="cuda")
    M = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = pkg.lib().ce_mppi_dbscan_noalloc_dev(z.data_ptr(), 16385, 16385, 2, 0.25, 20,
                                              labels.data_ptr(), M.data_ptr(), C.c_void_p(0))
    assert st == 1
    assert "16384" in pkg.lib().ce_mppi_last_error().decode()
