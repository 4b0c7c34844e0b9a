"""Host logic of the bench's memory plan: the box depth it estimates from the vertices
covers the active box the anchors give (oracle stencil anchors), and the z transform length
it assumes is the one the library picks for that box."""
import numpy as np
import pytest

import bench
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import make_workload


@pytest.mark.parametrize("name", ["sphere480", "sphere7680", "ellipsoid20k", "plate1160", "array_sub3_n384"])
def test_box_depth_estimate(name):
    w = make_workload(name)
    rwg = build_rwg(*w.mesh)
    az = np.clip(np.floor((rwg.midpoint()[:, 2] - w.origin[2]) / w.h).astype(int) - 1, 0, w.grid_n - 4)
    nz = int(az.max() + 3 - az.min() + 1)                      # the box's z-planes
    lz = next(n for n in bench.Z_LENGTHS if 2 * nz <= n <= 2 * w.grid_n)
    nz_est, lz_est = bench.box_depth(w)
    assert nz_est >= nz and lz_est == lz, (nz_est, nz, lz_est, lz)
