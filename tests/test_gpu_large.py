"""The largest grid (384^3 nodes, 768-point FFT lines) and the 491k-RWG sphere array.

* 16 spheres of 1920 RWG on the 384^3 grid: sampled output rows against the
  oracle's direct grid sums and near-zone entries.
* The full 4x4 array of icosphere-5 spheres (491 520 RWG): set up, one product in
  complex64 and in complex128 (they agree to the complex64 tolerance), and a few
  march steps (every GMRES solve converges).
* The 19 998-RWG ellipsoid on the 96^3 grid: the adjoint march and the autograd
  gradient at that size.
"""
import numpy as np
import pytest

from oracle import aim as oaim
from oracle import efie
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import make_workload

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def test_array_384_sampled_rows():
    """complex128 path: sampled rows against the oracle (1e-10).  complex64 path: the
    same rows within 1e-5 times the cancellation ratio |grid part| / |product| of
    those rows.  These 1920-RWG spheres are coarse for the 384^3 grid (edges of ~5 grid
    spacings), so the grid part is much larger than the product it sums to with the
    near-zone correction, and FP32 rounding in the grid part is amplified by that
    ratio; the resolved 491k-RWG array is held to 1e-5 below."""
    import torch

    from paper_1408_7060_gb300 import AimContext

    w = make_workload("array_sub3_n384")
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    rng = np.random.default_rng(12)
    x = rng.standard_normal((1, rwg.ns)) + 1j * rng.standard_normal((1, rwg.ns))
    rows = np.sort(rng.choice(rwg.ns, 3, replace=False))
    xd = torch.tensor(x, device="cuda")
    with AimContext.from_workload(w, precision="c128") as c:
        assert c.n_delays == A.n_delays
        y128 = c.matvec(0, xd).cpu().numpy()[0]
    with AimContext.from_workload(w, precision="c64") as c:
        y64 = c.matvec(0, xd).cpu().numpy()[0]
    grid = A.fft_part_rows(0, x[0], rows)
    ref = grid.copy()
    sel = np.isin(A.pairs[:, 0], rows)
    pr = A.pairs[sel]
    Zn = efie.fill_pairs(rwg, p, pr, 0)[0] - A.fft_pairs(0, pr)
    for (k, kp), z in zip(pr, Zn):
        ref[np.searchsorted(rows, k)] += z * x[0, kp]
    assert rel(y128[rows], ref) < 1e-10
    ratio = np.linalg.norm(grid) / np.linalg.norm(ref)
    e64 = rel(y64[rows], ref)
    print(f"384^3 sampled rows: complex64 error {e64:.3e}, cancellation ratio {ratio:.1f}, "
          f"complex64 vs complex128 over the whole product {rel(y64, y128):.3e}")
    assert e64 < 1e-5 * max(1.0, ratio)


def test_array491k_full_size():
    import torch

    from paper_1408_7060_gb300 import AimContext

    w = make_workload("array491k")
    assert w.grid_n == 384
    rng = np.random.default_rng(13)
    with AimContext.from_workload(w, batch_max=1) as c64:
        assert c64.ns == 491520
        x = torch.tensor(rng.standard_normal((1, c64.ns)) + 1j * rng.standard_normal((1, c64.ns)), device="cuda")
        y64 = c64.matvec(0, x).cpu().numpy()
        cur, st, rc = c64.march(w.khat[:1], w.phat[:1], w.sigma, w.t_d, 3, w.tol,
                                out=torch.empty((3, 1, c64.ns), dtype=torch.complex128, device="cuda"))
        assert st["last_step"] == 3 and st["max_rel_res"] <= w.tol
    with AimContext.from_workload(w, batch_max=1, precision="c128") as c128:
        y128 = c128.matvec(0, x).cpu().numpy()
    print(f"491k-RWG array: complex64 vs complex128 relative L2 {rel(y64, y128):.3e}")
    assert rel(y64, y128) < 1e-5


def test_ellipsoid_adjoint_at_scale():
    """Ellipsoid (19 998 RWG, 96^3 grid, complex64 grid path, near-zone SAI
    preconditioner with near sets of up to 83 RWGs), 40-step march.

    The march solves each step only to the GMRES tolerance, so the map from incident
    samples a to far field F(a) is linear only up to solver error, and the adjoint
    consistency <y, F d> = <F^H y, d> holds to an error that shrinks with the
    tolerance.  Checked: that error at tol 1e-6 is below 2e-3 and at least 3x smaller
    than at 1e-5; and the autograd gradient of J = sum |F|^2 agrees with central
    differences along band-limited directions to 3 % at tol 1e-6 (a wrong factor 2 or
    a missing conjugation would be off by 50 % or more).  The exact algebra of the
    adjoint is pinned against the oracle in complex128 on the 480-RWG sphere."""
    import torch

    from paper_1408_7060_gb300 import AimContext, abi
    from paper_1408_7060_gb300.autograd import far_field_objective
    from paper_1408_7060_gb300.inputs import random_plane_waves

    w = make_workload("ellipsoid20k")
    nt, i0, n_samp, n0, n_out = 40, -3, 46, -6, 54
    r, _ = random_plane_waves(8, 2)
    e1 = np.cross(r, np.where(np.abs(r[:, 2:3]) < 0.9, [[0, 0, 1.0]], [[1.0, 0, 0]]))
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(r, e1)
    t = (np.arange(n_samp) + i0) * w.dt
    # samples of the modulated Gaussian's envelope g(t - t_d) e^{-j w t_d} on the grid
    a0 = np.exp(-((t - w.t_d) ** 2) / (2 * w.sigma ** 2)) * np.exp(-2j * np.pi * w.f_c * w.t_d)
    k, p = w.khat[0], w.phat[0]
    rng = np.random.Generator(np.random.PCG64(1))
    f = np.fft.fftfreq(n_samp, d=w.dt)

    def band():  # random envelope with the incident pulse's spectrum
        z = rng.standard_normal(n_samp) + 1j * rng.standard_normal(n_samp)
        d = np.fft.ifft(np.fft.fft(z) * np.exp(-0.5 * (2 * np.pi * f * w.sigma) ** 2))
        return d / np.linalg.norm(d)

    with AimContext.from_workload(w, precision="c64", max_iter=2000, restart=63, precond="sai") as c:
        h = c.handle

        def F(a, tol):
            V = abi.aim_excitation_samples(h, k, p, i0, torch.tensor(a, device="cuda"), nt)
            I, _, rc = abi.aim_march_source(h, V.reshape(nt, 1, -1), tol)
            assert rc == 0
            return abi.aim_farfield(h, r, e1, e2, I.reshape(nt, -1), n0, n_out).cpu().numpy()

        def FH(y, tol):
            G = abi.aim_farfield_adjoint(h, r, e1, e2, nt, n0, torch.tensor(y, device="cuda"))
            src = torch.flip(G, dims=[0]).conj().resolve_conj().contiguous().reshape(nt, 1, -1)
            u, _, rc = abi.aim_march_source(h, src, tol, transpose=True)
            assert rc == 0
            lam = torch.flip(u, dims=[0]).conj().resolve_conj().contiguous().reshape(nt, -1)
            return abi.aim_excitation_samples_adjoint(h, k, p, i0, n_samp, lam).cpu().numpy()

        dirs = [band() for _ in range(2)]
        err = {}
        for tol in (1e-5, 1e-6):
            e = []
            for d in dirs:
                Fd = F(d, tol)
                y = rng.standard_normal(Fd.shape) + 1j * rng.standard_normal(Fd.shape)
                e.append(abs(np.vdot(y, Fd) - np.vdot(FH(y, tol), d)) / abs(np.vdot(y, Fd)))
            err[tol] = max(e)
        assert err[1e-6] < 2e-3, err
        assert err[1e-6] < err[1e-5] / 3, err

        tol = 1e-6
        a = torch.tensor(a0, device="cuda", requires_grad=True)
        J = far_field_objective(a, c, (k, p), (r, e1, e2), nt, tol, i0, n0, n_out)
        J.backward()
        g = a.grad.detach().cpu().numpy()
        eps = 0.5 * np.linalg.norm(a0)
        with torch.no_grad():
            for _ in range(2):
                dd = torch.tensor(band(), device="cuda")
                jp = far_field_objective(a + eps * dd, c, (k, p), (r, e1, e2), nt, tol, i0, n0, n_out).item()
                jm = far_field_objective(a - eps * dd, c, (k, p), (r, e1, e2), nt, tol, i0, n0, n_out).item()
                fd = (jp - jm) / (2 * eps)
                an = float(np.real(np.vdot(g, dd.cpu().numpy())))
                assert abs(fd - an) <= 3e-2 * abs(an), (fd, an)
