"""The adjoint path on the GPU: excitation from envelope samples, far-field
envelopes, their adjoints, the transposed march, and the autograd gradient of the
far-field objective -- against the oracle, dot-product identities and central
finite differences."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import aim as oaim
from oracle import efie, march
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import make_workload, random_plane_waves

pytestmark = pytest.mark.gpu

NT = 40            # march steps
I0, NSAMP = -3, 46  # envelope samples a_i, i = I0 .. I0 + NSAMP - 1
N0, NOUT = -5, 52   # far-field times


@pytest.fixture(scope="module")
def case():
    w = make_workload("sphere480")
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    ZA = np.stack([A.dense(m) for m in range(A.n_delays + 1)])
    return w, rwg, p, A, ZA


@pytest.fixture(scope="module")
def ctx(case):
    from paper_1408_7060_gb300 import AimContext

    c = AimContext.from_workload(case[0], precision="c128")
    yield c
    c.close()


def dirs(n=8, seed=2):
    r, _ = random_plane_waves(n, seed)
    e1 = np.cross(r, np.where(np.abs(r[:, 2:3]) < 0.9, [[0, 0, 1.0]], [[1.0, 0, 0]]))
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(r, e1)
    return r, e1, e2


WAVE = (np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0]))


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_excitation_samples(case, ctx):
    w, rwg, p, A, ZA = case
    from paper_1408_7060_gb300 import abi

    rng = np.random.default_rng(0)
    a = crandn(rng, NSAMP)
    got = abi.aim_excitation_samples(ctx.handle, *WAVE, I0, a, NT)
    s = list(range(-12, 12))
    B = oadj.incident_taps(rwg, p, *WAVE, s)
    ref = oadj.excitation_from_samples(B, s, a, I0, NT)
    assert rel(got, ref) < 1e-12
    lam = crandn(rng, NT, rwg.ns)
    g = abi.aim_excitation_samples_adjoint(ctx.handle, *WAVE, I0, NSAMP, lam)
    assert abs(np.vdot(got, lam) - np.vdot(a, g)) < 1e-12 * abs(np.vdot(got, lam))


def test_farfield(case, ctx):
    w, rwg, p, A, ZA = case
    from paper_1408_7060_gb300 import abi

    r, e1, e2 = dirs()
    rng = np.random.default_rng(1)
    I = crandn(rng, NT, rwg.ns)
    got = abi.aim_farfield(ctx.handle, r, e1, e2, I, N0, NOUT)
    s = list(range(-12, 12))
    At = oadj.farfield_taps(rwg, p, r, e1, e2, s)
    ref = oadj.farfield(At, s, I, list(range(N0, N0 + NOUT)))
    assert rel(got, ref) < 1e-12
    Fr = crandn(rng, NOUT, len(r), 2)
    G = abi.aim_farfield_adjoint(ctx.handle, r, e1, e2, NT, N0, Fr)
    assert abs(np.vdot(got, Fr) - np.vdot(I, G)) < 1e-12 * abs(np.vdot(got, Fr))


@pytest.mark.parametrize("transpose", [False, True])
def test_march_source(case, ctx, transpose):
    w, rwg, p, A, ZA = case
    from paper_1408_7060_gb300 import abi

    rng = np.random.default_rng(3)
    S = crandn(rng, 20, 1, rwg.ns)
    Z = np.transpose(ZA, (0, 2, 1)) if transpose else ZA
    ref = march.march_dense(Z, S)
    got, st, _ = abi.aim_march_source(ctx.handle, S, 1e-12, transpose=transpose)
    assert rel(got, ref) < 1e-9


def test_gradient_vs_oracle_and_fd(case, ctx):
    import torch

    from paper_1408_7060_gb300.autograd import far_field_objective

    w, rwg, p, A, ZA = case
    r, e1, e2 = dirs()
    rng = np.random.default_rng(4)
    a0 = crandn(rng, NSAMP)
    a = torch.tensor(a0, device="cuda", requires_grad=True)
    J = far_field_objective(a, ctx, WAVE, (r, e1, e2), NT, 1e-12, I0, N0, NOUT)
    J.backward()
    g = a.grad.detach().cpu().numpy()
    # oracle: dense march, dense adjoint
    s = list(range(-12, 12))
    B = oadj.incident_taps(rwg, p, *WAVE, s)
    At = oadj.farfield_taps(rwg, p, r, e1, e2, s)
    Jr, gr = oadj.gradient(ZA, B, s, At, s, a0, I0, NT, list(range(N0, N0 + NOUT)))
    assert abs(J.item() - Jr) < 1e-8 * Jr
    assert rel(g, 2 * gr) < 1e-6
    # central differences along 32 random directions (J is quadratic: exact up to rounding)
    with torch.no_grad():
        for _ in range(32):
            d = torch.tensor(crandn(rng, NSAMP), device="cuda")
            eps = 1e-3 * (np.linalg.norm(a0) / np.sqrt(NSAMP))
            jp = far_field_objective(a + eps * d, ctx, WAVE, (r, e1, e2), NT, 1e-12, I0, N0, NOUT).item()
            jm = far_field_objective(a - eps * d, ctx, WAVE, (r, e1, e2), NT, 1e-12, I0, N0, NOUT).item()
            fd = (jp - jm) / (2 * eps)
            an = float(np.real(np.vdot(g, d.cpu().numpy())))
            assert abs(fd - an) <= 1e-4 * abs(an) + 1e-9 * J.item(), (fd, an)


def test_march_adjoint_vs_dense(case, ctx):
    """aim_march_adjoint solves M^H lam = G: backward substitution with Z_m^H."""
    w, rwg, p, A, ZA = case
    from paper_1408_7060_gb300 import abi

    rng = np.random.default_rng(5)
    nt = 20
    G = crandn(rng, nt, 1, rwg.ns)
    ZH = np.conj(np.transpose(ZA, (0, 2, 1)))
    ref = np.zeros_like(G)
    for l in range(nt, 0, -1):
        r = G[l - 1, 0].copy()
        for m in range(1, len(ZA)):
            if l + m <= nt:
                r -= ZH[m] @ ref[l + m - 1, 0]
        ref[l - 1, 0] = np.linalg.solve(ZH[0], r)
    lam, st, rc = abi.aim_march_adjoint(ctx.handle, G, 1e-12)
    assert st["last_step"] == nt
    assert rel(lam, ref) < 1e-9


def test_fused_farfield_passes_match_composed_calls(case, ctx):
    """aim_march_farfield (far field added step by step, no current history) equals the
    far field of the stored march; aim_march_adjoint_farfield (sources and gradient formed
    step by step in reversed time) equals B^H of the adjoint march of A^H F."""
    import torch

    w, rwg, p, A, ZA = case
    from paper_1408_7060_gb300 import abi

    r, e1, e2 = dirs()
    rng = np.random.default_rng(6)
    a = torch.tensor(crandn(rng, NSAMP), device="cuda")
    F, st, _ = abi.aim_march_farfield(ctx.handle, *WAVE, I0, a, NT, 1e-12, r, e1, e2, N0, NOUT)
    V = abi.aim_excitation_samples(ctx.handle, *WAVE, I0, a, NT)
    I, _, _ = abi.aim_march_source(ctx.handle, V.reshape(NT, 1, -1), 1e-12)
    F2 = abi.aim_farfield(ctx.handle, r, e1, e2, I.reshape(NT, -1), N0, NOUT)
    assert rel(F.cpu().numpy(), F2.cpu().numpy()) < 1e-12
    Fy = torch.tensor(crandn(rng, NOUT, len(r), 2), device="cuda")
    g, _, _ = abi.aim_march_adjoint_farfield(ctx.handle, *WAVE, I0, NSAMP, NT, 1e-12, r, e1, e2, N0, Fy)
    G = abi.aim_farfield_adjoint(ctx.handle, r, e1, e2, NT, N0, Fy)
    lam, _, _ = abi.aim_march_adjoint(ctx.handle, G.reshape(NT, 1, -1), 1e-12)
    g2 = abi.aim_excitation_samples_adjoint(ctx.handle, *WAVE, I0, NSAMP, lam.reshape(NT, -1))
    assert rel(g.cpu().numpy(), g2.cpu().numpy()) < 1e-10
    # the adjoint identity of the whole map a -> F
    lhs = np.vdot(Fy.cpu().numpy(), F.cpu().numpy())
    assert abs(lhs - np.vdot(g.cpu().numpy(), a.cpu().numpy())) < 1e-9 * abs(lhs)
