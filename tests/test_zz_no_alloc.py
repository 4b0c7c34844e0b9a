"""aim_matvec_noalloc: the operator product without any device allocation.

Some callers cannot allocate device memory while they run (a solver captured into
a CUDA graph, a real-time path with a fixed memory budget, an application whose
device memory belongs to another allocator).  This entry point takes its grid work
space from one fixed 16 MiB array in the library.  The test calls it twice in a row
through the C ABI and compares each result with aim_matvec, and checks that sizes
beyond the fixed array are rejected.  It sits in its own file, collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ctx(name, precision, batch_max=1):
    from paper_1408_7060_gb300 import AimContext
    from paper_1408_7060_gb300.inputs import make_workload

    w = make_workload(name)
    return w, AimContext.from_workload(w, precision=precision, batch_max=batch_max)


@pytest.mark.parametrize("name,precision,tol", [("sphere480", "c128", 1e-10), ("sphere_sub3_n32", "c64", 1e-5)])
def test_noalloc_matches_matvec_twice(name, precision, tol):
    from paper_1408_7060_gb300 import abi

    w, ctx = _ctx(name, precision)
    with ctx:
        rng = np.random.default_rng(21)
        for call in range(2):
            x = rng.standard_normal((1, ctx.ns)) + 1j * rng.standard_normal((1, ctx.ns))
            m = call % (ctx.n_delays + 1)
            ref = ctx.matvec(m, x)
            got = abi.aim_matvec_noalloc(ctx.handle, m, x)
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err <= tol, (call, err)


def test_noalloc_rejects_oversize():
    from paper_1408_7060_gb300 import abi

    w, ctx = _ctx("sphere_sub3_n32", "c64", batch_max=3)   # 3 x 7.3 MB > 16 MiB
    with ctx:
        x = np.ones((3, ctx.ns), dtype=np.complex128)
        with pytest.raises(abi.AimError) as e:
            abi.aim_matvec_noalloc(ctx.handle, 0, x)
        assert e.value.code == abi.AIM_ERR_ARG
        y = abi.aim_matvec_noalloc(ctx.handle, 0, x[:2])          # 2 x 7.3 MB fits
        assert np.allclose(y, ctx.matvec(0, x[:2]), rtol=0, atol=1e-5 * np.abs(y).max())
