"""The complex64 march (FP64 solve) of the 7680-RWG sphere workloads against the oracle.

Expected values: ``tests/golden/sphere7680_march_rows.txt``, written by the committed
script ``tests/golden/make_sphere7680_marches.py`` from the oracle alone (its ET-AIM
operator with FFT grid sums pinned to direct sums, GMRES to a true residual of 1e-10),
on 48 sampled rows over steps 1..24, which cover the incident pulse (peak near step 15).

* sphere7680 (600 MHz +-30 %, chi = 4.33, N_g = 7): one wave, the benchmark's solver
  settings (near-zone SAI on 2.5 near radii, tol 1e-6);
* sphere7680_b64 (600 MHz +-10 %, chi = 11, N_g = 3): the first four of the 64 seeded
  waves marched as one batch (per-RHS GMRES inside one graph); waves 0 and 1 against
  the oracle, and every wave of the batch against its own single-wave march.

Tolerance: 1e-4 relative L2 over the sampled rows and steps (the marched-current bound);
batch vs single-wave marches 1e-10 (the same arithmetic per right-hand side).
"""
import os

import numpy as np
import pytest

from paper_1408_7060_gb300.inputs import make_workload

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "sphere7680_march_rows.txt")


def golden():
    out = {}
    for line in open(GOLD):
        if line.startswith("#"):
            continue
        name, wv, l, r, re, im = line.split()
        out.setdefault((name, int(wv)), {}).setdefault(int(l), []).append((int(r), float(re) + 1j * float(im)))
    res = {}
    for key, steps in out.items():
        ls = sorted(steps)
        rows = np.array([r for r, _ in steps[ls[0]]])
        res[key] = (rows, np.array([[v for _, v in steps[l]] for l in ls]))
    return res


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def _ctx(w, **over):
    from paper_1408_7060_gb300 import AimContext

    kw = dict(precond="sai", precond_radius=2.5 * w.near_radius)
    kw.update(over)
    return AimContext.from_workload(w, **kw)


def test_march_sphere7680_vs_oracle():
    import torch

    g = golden()
    rows, ref = g[("sphere7680", 0)]
    w = make_workload("sphere7680")
    nt = ref.shape[0]
    with _ctx(w) as c:
        out = torch.empty((nt, 1, c.ns), dtype=torch.complex128, device="cuda")
        _, st, rc = c.march(w.khat, w.phat, w.sigma, w.t_d, nt, w.tol, out=out)
        cur = out.cpu().numpy()
    err = rel(cur[:, 0, rows], ref)
    print(f"sphere7680 complex64 march vs oracle, {nt} steps x {len(rows)} rows: {err:.3e}")
    assert err < 1e-4, err


def test_batched_march_sphere7680_b64_vs_oracle():
    import torch

    g = golden()
    w = make_workload("sphere7680_b64")
    nb, nt = 4, g[("sphere7680_b64", 0)][1].shape[0]
    k, p = w.khat[:nb], w.phat[:nb]
    with _ctx(w, batch_max=nb) as c:
        out = torch.empty((nt, nb, c.ns), dtype=torch.complex128, device="cuda")
        _, st, rc = c.march(k, p, w.sigma, w.t_d, nt, w.tol, out=out)
        cur = out.cpu().numpy()
        assert st["iters"].shape == (nt, nb)
    for wv in (0, 1):
        rows, ref = g[("sphere7680_b64", wv)]
        err = rel(cur[:, wv, rows], ref)
        print(f"sphere7680_b64 wave {wv} (batch of {nb}) vs oracle: {err:.3e}")
        assert err < 1e-4, (wv, err)
    with _ctx(w, batch_max=1) as c1:
        for b in range(nb):
            one = torch.empty((nt, 1, c1.ns), dtype=torch.complex128, device="cuda")
            c1.march(k[b:b + 1], p[b:b + 1], w.sigma, w.t_d, nt, w.tol, out=one)
            e = rel(cur[:, b], one.cpu().numpy()[:, 0])
            assert e < 1e-10, (b, e)
