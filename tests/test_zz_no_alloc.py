"""aim_matvec_noalloc: the operator product without any device allocation.

Some callers cannot allocate device memory while they run: a real-time path whose
memory budget is fixed at start-up, an application whose device memory belongs to
another allocator, a process under a hard device-memory quota.  This entry point takes
its grid work space from one fixed 16 MiB array in the library.  The tests call it
twice in a row through the C ABI and compare each result with aim_matvec (host arrays,
device arrays written in place, and two right-hand sides in complex128), and check that
sizes beyond the fixed array are rejected.  The file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ctx(name, precision, batch_max=1):
    from paper_1408_7060_gb300 import AimContext
    from paper_1408_7060_gb300.inputs import make_workload

    w = make_workload(name)
    return w, AimContext.from_workload(w, precision=precision, batch_max=batch_max)


@pytest.mark.parametrize("name,precision,tol,nb,device", [
    ("sphere480", "c128", 1e-10, 1, False),
    ("sphere_sub3_n32", "c64", 1e-5, 1, False),
    ("sphere_sub3_n32", "c64", 1e-5, 1, True),
    ("sphere480", "c128", 1e-10, 2, True),
])
def test_noalloc_matches_matvec_twice(name, precision, tol, nb, device):
    import torch

    from paper_1408_7060_gb300 import abi

    w, ctx = _ctx(name, precision, batch_max=nb)
    with ctx:
        rng = np.random.default_rng(21)
        for call in range(2):
            x = rng.standard_normal((nb, ctx.ns)) + 1j * rng.standard_normal((nb, ctx.ns))
            m = call % (ctx.n_delays + 1)
            ref = ctx.matvec(m, x)
            if device:
                xd = torch.tensor(x, device="cuda")
                yd = torch.full_like(xd, float("nan"))
                abi.aim_matvec_noalloc(ctx.handle, m, xd, out=yd)
                got = yd.cpu().numpy()
            else:
                got = abi.aim_matvec_noalloc(ctx.handle, m, x)
            for b in range(nb):
                err = np.linalg.norm(got[b] - ref[b]) / np.linalg.norm(ref[b])
                assert err <= tol, (call, b, err)


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
