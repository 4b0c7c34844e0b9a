"""The synthetic meshes are valid RWG surfaces: closed, two-manifold, outward
oriented, and (for the ellipsoid) Delaunay on the surface with no slivers."""
import numpy as np

from paper_1408_7060_gb300.inputs import ellipsoid_mesh, icosphere, sphere_array


def _angles(V, F):
    P = V[F]
    out = []
    for j in range(3):
        u = P[:, (j + 1) % 3] - P[:, j]
        v = P[:, (j + 2) % 3] - P[:, j]
        out.append(np.arccos(np.clip((u * v).sum(1) / np.linalg.norm(u, axis=1) / np.linalg.norm(v, axis=1), -1, 1)))
    return np.stack(out, axis=1)  # angle at vertex j of each face


def _check_closed_outward(V, F, centres):
    half = {}
    for f in F:
        for j in range(3):
            e = (int(f[j]), int(f[(j + 1) % 3]))
            assert e not in half
            half[e] = True
    assert all((b, a) in half for (a, b) in half)
    P = V[F]
    n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    c = P.mean(axis=1)
    ctr = centres[np.argmin(((c[:, None, :] - centres[None]) ** 2).sum(2), axis=1)]
    assert ((n * (c - ctr)).sum(1) > 0).all()


def test_ellipsoid_mesh_is_surface_delaunay():
    V, F = ellipsoid_mesh(n_points=1500)
    _check_closed_outward(V, F, np.zeros((1, 3)))
    assert len(F) == 2 * len(V) - 4
    A = _angles(V, F)
    assert np.degrees(A.min()) > 20.0
    # Delaunay: for every interior edge the two opposite angles sum to at most pi
    opp = {}
    for fi, f in enumerate(F):
        for j in range(3):
            a, b = int(f[j]), int(f[(j + 1) % 3])
            opp[(a, b)] = A[fi, (j + 2) % 3]
    assert max(opp[(a, b)] + opp[(b, a)] for (a, b) in opp if a < b) <= np.pi + 1e-9


def test_sphere_meshes_closed_outward():
    V, F = icosphere(2, 1.0)
    _check_closed_outward(V, F, np.zeros((1, 3)))
    V, F = sphere_array(2, 0.5, 1.5)
    g = (np.arange(4) - 1.5) * 1.5
    centres = np.array([(x, y, 0.0) for y in g for x in g])
    _check_closed_outward(V, F, centres)


def test_plate_meshes_match_table_ii():
    """Square plates: open, every interior edge shared by two faces of opposite
    traversal, boundary edges on the outline only, faces counter-clockwise about +z, and
    the RWG counts 3 n^2 - 2 n of Table II (280, 1160, 4720, 19 040 for 1, 2, 4, 8 m)."""
    from oracle.rwg import build_rwg
    from paper_1408_7060_gb300.inputs import plate_mesh

    for side, ns in ((1.0, 280), (2.0, 1160), (4.0, 4720), (8.0, 19040)):
        n = int(round(side / 0.1))
        V, F = plate_mesh(side, n)
        P = V[F]
        nz = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])[:, 2]
        assert (nz > 0).all() and np.allclose(V[:, 2], 0.0)
        count = {}
        for f in F:
            for j in range(3):
                a, b = int(f[j]), int(f[(j + 1) % 3])
                count[(a, b)] = count.get((a, b), 0) + 1
        assert max(count.values()) == 1                       # no half-edge twice
        boundary = [(a, b) for (a, b) in count if (b, a) not in count]
        mid = np.array([(V[a] + V[b]) / 2 for a, b in boundary])
        assert np.all(np.isclose(np.abs(mid[:, :2]).max(axis=1), side / 2))
        assert len(boundary) == 4 * n
        assert build_rwg(V, F).ns == ns == 3 * n * n - 2 * n
