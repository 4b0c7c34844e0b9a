"""The launch-plan autotuner (aim_opts.autotune).

Every launch shape a plan may choose (tile widths of the z and y passes, rows per block
of the x passes) runs the same arithmetic per grid line, so the operator product must
be bitwise identical under the tuned and the default plan.  Checked for power-of-two
and factor-3 padded lengths in both precisions, together with the plan cache: a first
setup measures and records the plan, a second setup with the same GPU, length,
precision and batch reads it back, and autotune = 2 measures again.
"""
import json

import numpy as np
import pytest

from paper_1408_7060_gb300.inputs import make_workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,precision", [("sphere480", "c64"), ("sphere_sub3_n32", "c128"),
                                            ("sphere_sub3_n96", "c64")])
def test_tuned_plan_gives_identical_products(name, precision, tmp_path, monkeypatch):
    from paper_1408_7060_gb300 import AimContext, abi

    cache = tmp_path / "plans.jsonl"
    monkeypatch.setenv("AIM_GB300_PLAN_CACHE", str(cache))
    w = make_workload(name)
    rng = np.random.default_rng(41)
    with AimContext.from_workload(w, precision=precision, batch_max=2) as c0:
        x = rng.standard_normal((2, c0.ns)) + 1j * rng.standard_normal((2, c0.ns))
        assert c0.info["plan_source"] == abi.AIM_PLAN_DEFAULT
        ref = [c0.matvec(m, x) for m in (0, 1)]
    with AimContext.from_workload(w, precision=precision, batch_max=2, autotune=1) as c1:
        assert c1.info["plan_source"] == abi.AIM_PLAN_MEASURED
        plan = {k: c1.info["plan_" + k] for k in ("zw", "cw", "rp", "ypb")}
        for m, r in zip((0, 1), ref):
            assert np.array_equal(c1.matvec(m, x), r), (m, plan)
    lines = [json.loads(l) for l in cache.read_text().splitlines()]
    assert len(lines) == 1 and {k: lines[0][k] for k in plan} == plan
    assert f"L={2 * w.grid_n}" in lines[0]["key"] and f"prec={precision}" in lines[0]["key"]
    with AimContext.from_workload(w, precision=precision, batch_max=2, autotune=1) as c2:
        assert c2.info["plan_source"] == abi.AIM_PLAN_CACHED
        assert {k: c2.info["plan_" + k] for k in plan} == plan
        assert np.array_equal(c2.matvec(0, x), ref[0])
    with AimContext.from_workload(w, precision=precision, batch_max=2, autotune=2) as c3:
        assert c3.info["plan_source"] == abi.AIM_PLAN_MEASURED
    assert len(cache.read_text().splitlines()) == 2


def test_tuned_plan_march_matches_default(monkeypatch, tmp_path):
    """A march under a tuned plan equals the march under the default plan (bitwise)."""
    from paper_1408_7060_gb300 import AimContext

    monkeypatch.setenv("AIM_GB300_PLAN_CACHE", str(tmp_path / "plans.jsonl"))
    w = make_workload("sphere_sub3_n32")
    with AimContext.from_workload(w, precision="c64") as c0:
        a, _, _ = c0.march(w.khat, w.phat, w.sigma, w.t_d, 15, 1e-6)
    with AimContext.from_workload(w, precision="c64", autotune=2) as c1:
        b, _, _ = c1.march(w.khat, w.phat, w.sigma, w.t_d, 15, 1e-6)
    assert np.array_equal(a, b)
