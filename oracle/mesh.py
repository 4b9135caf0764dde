"""FP64 brute-force signed distance to a watertight triangle mesh.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3.1 of the paper samples points around the object and computes their
signed distance to the mesh, without saying how.  This module takes the
plain definition:

* unsigned distance = min over all triangles of || p - c_t(p) ||, where
  c_t(p) is the closest point of triangle t to p.  c_t is found by the
  region test on the barycentric Voronoi regions of the triangle (vertex,
  edge or face region), as in Ericson, "Real-Time Collision Detection",
  Sec. 5.1.5;
* sign: negative inside (Sec. 3.2 defines the interior as negative), where
  "inside" means a generalized winding number w(p) > 1/2 (Jacobson, Kavan &
  Sorkine-Hornung, SIGGRAPH 2013).  w(p) = sum_t Omega_t(p) / (4 pi), with
  the solid angle of each triangle from the Van Oosterom & Strackee (1983)
  formula  tan(Omega/2) = A.(B x C) / (|A||B||C| + (A.B)|C| + (A.C)|B| + (B.C)|A|),
  A, B, C the triangle's corners relative to p.
"""

import numpy as np


def _dot(u, v):
    return np.einsum("...i,...i->...", u, v)


def closest_point_triangle(p, a, b, c):
    """Closest point of triangles (a, b, c) to points p, all broadcast [..., 3].

    Vertex regions are tested first, then edges, then the face, so a point
    on a region boundary gets the feature listed first; the distance is the
    same either way.
    """
    p, a, b, c = np.broadcast_arrays(*(np.asarray(x, dtype=np.float64) for x in (p, a, b, c)))
    ab, ac = b - a, c - a
    ap, bp, cp = p - a, p - b, p - c
    d1, d2 = _dot(ab, ap), _dot(ac, ap)
    d3, d4 = _dot(ab, bp), _dot(ac, bp)
    d5, d6 = _dot(ab, cp), _dot(ac, cp)
    vc = d1 * d4 - d3 * d2
    vb = d5 * d2 - d1 * d6
    va = d3 * d6 - d5 * d4

    in_a = (d1 <= 0) & (d2 <= 0)
    in_b = (d3 >= 0) & (d4 <= d3)
    in_c = (d6 >= 0) & (d5 <= d6)
    on_ab = (vc <= 0) & (d1 >= 0) & (d3 <= 0)
    on_ac = (vb <= 0) & (d2 >= 0) & (d6 <= 0)
    on_bc = (va <= 0) & ((d4 - d3) >= 0) & ((d5 - d6) >= 0)

    with np.errstate(divide="ignore", invalid="ignore"):
        t_ab = d1 / (d1 - d3)
        t_ac = d2 / (d2 - d6)
        t_bc = (d4 - d3) / ((d4 - d3) + (d5 - d6))
        den = va + vb + vc
        v_face = vb / den
        w_face = vc / den

    def e(t):
        return np.nan_to_num(t)[..., None]

    face = a + ab * e(v_face) + ac * e(w_face)
    choices = [a, b, a + ab * e(t_ab), c, a + ac * e(t_ac), b + (c - b) * e(t_bc)]
    conds = [in_a, in_b & ~in_a, on_ab, in_c, on_ac, on_bc]
    out = face
    # apply in reverse so that the first listed region wins
    for cond, val in reversed(list(zip(conds, choices))):
        out = np.where(cond[..., None], val, out)
    return out


def solid_angle(p, a, b, c):
    """Signed solid angle of triangles (a, b, c) seen from p (Van Oosterom-Strackee)."""
    A, B, C = a - p, b - p, c - p
    la, lb, lc = (np.linalg.norm(X, axis=-1) for X in (A, B, C))
    num = _dot(A, np.cross(B, C))
    den = la * lb * lc + _dot(A, B) * lc + _dot(A, C) * lb + _dot(B, C) * la
    return 2.0 * np.arctan2(num, den)


def winding_number(p, V, F, chunk=256):
    """Generalized winding number w(p) = sum_t Omega_t(p) / (4 pi), p [n, 3]."""
    p = np.asarray(p, dtype=np.float64)[:, :3]
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    out = np.empty(p.shape[0])
    for s in range(0, p.shape[0], chunk):
        q = p[s:s + chunk, None, :]
        out[s:s + chunk] = solid_angle(q, a[None], b[None], c[None]).sum(1) / (4 * np.pi)
    return out


def unsigned_distance(p, V, F, chunk=256):
    """min_t || p - c_t(p) || over all triangles, p [n, 3]; also the argmin."""
    p = np.asarray(p, dtype=np.float64)[:, :3]
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    d = np.empty(p.shape[0])
    arg = np.empty(p.shape[0], dtype=np.int64)
    for s in range(0, p.shape[0], chunk):
        q = p[s:s + chunk, None, :]
        cp = closest_point_triangle(q, a[None], b[None], c[None])
        dist = np.linalg.norm(q - cp, axis=-1)
        arg[s:s + chunk] = dist.argmin(1)
        d[s:s + chunk] = dist.min(1)
    return d, arg


def signed_distance(p, V, F, chunk=256):
    """Exact signed distance: -dist inside (w > 1/2), +dist outside."""
    d, _ = unsigned_distance(p, V, F, chunk)
    w = winding_number(p, V, F, chunk)
    return np.where(w > 0.5, -d, d)
