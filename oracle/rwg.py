"""RWG (Rao-Wilton-Glisson) spatial basis on a triangle mesh, Sec. 3 (Eq. 3).

One basis per interior edge (an edge shared by two faces); an edge of one face only
lies on the boundary of an open surface (the plates of Sec. 5.1) and carries none, its
face slot left empty.  Ordering and orientation (a reading; the paper defers the basis
to its reference [14]):

* edges are sorted by (lower vertex index, higher vertex index);
* T+ is the face whose counter-clockwise vertex cycle runs along the edge from
  the lower to the higher vertex index, T- the other face;
* on T+:  S(r) = l / (2 A+) (r - v+),  div S = +l / A+;
  on T-:  S(r) = l / (2 A-) (v- - r),  div S = -l / A-,
  with v+- the vertex of T+- opposite the edge and l the edge length.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class RWG:
    V: np.ndarray        # [nv,3]
    F: np.ndarray        # [nt,3]
    edge: np.ndarray     # [ns,2] (lo, hi)
    tri: np.ndarray      # [ns,2] (T+, T-)
    free: np.ndarray     # [ns,2] opposite vertex of (T+, T-)
    length: np.ndarray   # [ns]
    area: np.ndarray     # [nt]

    @property
    def ns(self) -> int:
        return len(self.edge)

    def midpoint(self) -> np.ndarray:
        return 0.5 * (self.V[self.edge[:, 0]] + self.V[self.edge[:, 1]])

    def tri_bases(self):
        """For every face, the (rwg, sign, free vertex) of its three edges.

        Returns ``k[nt,3], s[nt,3], vfree[nt,3]`` (vertex indices); a slot of a
        boundary edge keeps k = -1, s = 0, vfree = -1 (its coefficient s l / 2A is 0).
        """
        nt = len(self.F)
        k = np.full((nt, 3), -1, dtype=np.int64)
        s = np.zeros((nt, 3))
        fv = np.full((nt, 3), -1, dtype=np.int64)
        cnt = np.zeros(nt, dtype=np.int64)
        for e in range(self.ns):
            for side, sign in ((0, 1.0), (1, -1.0)):
                t = self.tri[e, side]
                k[t, cnt[t]] = e
                s[t, cnt[t]] = sign
                fv[t, cnt[t]] = self.free[e, side]
                cnt[t] += 1
        return k, s, fv


def build_rwg(V: np.ndarray, F: np.ndarray) -> RWG:
    V = np.asarray(V, dtype=np.float64)
    F = np.asarray(F, dtype=np.int64)
    owners: dict[tuple[int, int], list[tuple[int, int]]] = {}
    for t, (a, b, c) in enumerate(F):
        for p, q, r in ((a, b, c), (b, c, a), (c, a, b)):
            key = (min(p, q), max(p, q))
            # +1 when the face runs lo -> hi along this edge
            owners.setdefault(key, []).append((t, 1 if p < q else -1, r))
    keys = sorted(owners)
    edge, tri, free = [], [], []
    for key in keys:
        own = owners[key]
        if len(own) == 1:
            continue  # boundary edge of an open surface: no basis
        if len(own) != 2 or own[0][1] == own[1][1]:
            raise ValueError(f"edge {key} is not a consistently oriented manifold edge")
        plus = own[0] if own[0][1] > 0 else own[1]
        minus = own[1] if plus is own[0] else own[0]
        edge.append(key)
        tri.append((plus[0], minus[0]))
        free.append((plus[2], minus[2]))
    edge = np.asarray(edge, dtype=np.int64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    length = np.linalg.norm(V[edge[:, 1]] - V[edge[:, 0]], axis=1)
    return RWG(V, F, edge, np.asarray(tri, dtype=np.int64), np.asarray(free, dtype=np.int64),
               length, area)
