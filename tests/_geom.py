"""Independent circle/triangle crossing count in world coordinates (test helper).

Used to pin the oracle with a method that shares none of its steps: no two-rotation frame,
no layer slicing and no radius intervals.  For an oriented point (S, n) the circle of layer
beta and radius alpha is C(t) = S + beta*n_hat + alpha*(cos t * u + sin t * v) with (u, v,
n_hat) orthonormal.  Against a triangle with vertices A, B, C and plane normal m,
f(t) = m . (C(t) - A) = d + p cos t + q sin t, whose roots are found in closed form; each
root point is kept if it lies inside the triangle (barycentric test).  The count of a bin is
the number of such points over all triangles.

It also returns a per-bin margin (distance from tangency and from the triangle boundary) so
that comparisons can skip near-degenerate bins where the conventions for shared edges and
tangency decide the answer.
"""
import math

import numpy as np


def _basis(n):
    n = n / np.linalg.norm(n)
    a = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u = np.cross(n, a)
    u /= np.linalg.norm(u)
    v = np.cross(n, u)
    return n, u, v


def circle_counts(vertices, normal_of_origin, origin_pos, triangles, R, N):
    V = np.asarray(vertices, np.float64)
    S = np.asarray(origin_pos, np.float64)
    nh, u, v = _basis(np.asarray(normal_of_origin, np.float64))
    T = np.asarray(triangles, np.int64)
    A, B, Cc = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    m = np.cross(B - A, Cc - A)
    mlen = np.linalg.norm(m, axis=1)
    ok = mlen > 0
    A, B, Cc, m, mlen = A[ok], B[ok], Cc[ok], m[ok], mlen[ok]
    mu = m @ u
    mv = m @ v
    counts = np.zeros((N, N), np.int64)
    margin = np.full((N, N), np.inf)
    e0, e1 = B - A, Cc - A
    d00 = (e0 * e0).sum(1)
    d01 = (e0 * e1).sum(1)
    d11 = (e1 * e1).sum(1)
    den = d00 * d11 - d01 * d01
    for r in range(N):
        beta = R * (2 * r + 1 - N) / (2 * N)
        centre = S + beta * nh
        dconst = ((centre[None, :] - A) * m).sum(1)
        for c in range(N):
            alpha = R * (2 * c + 1) / (2 * N)
            p = alpha * mu
            q = alpha * mv
            amp = np.hypot(p, q)
            cnt = 0
            mg = np.inf
            rel = np.where(amp > 0, np.abs(dconst) / np.where(amp > 0, amp, 1), np.inf)
            cand = np.nonzero(rel < 1.0 + 1e-9)[0]
            # tangency margin: how far |d|/amp is from 1, scaled to a length
            near = np.nonzero(np.abs(rel - 1.0) < 1e-6)[0]
            if near.size:
                mg = 0.0
            for k in cand:
                if rel[k] > 1.0:
                    continue
                phi = math.atan2(q[k], p[k])
                w = math.acos(max(-1.0, min(1.0, -dconst[k] / amp[k])))
                for t in (phi + w, phi - w):
                    X = centre + alpha * (math.cos(t) * u + math.sin(t) * v)
                    w2 = X - A[k]
                    b1 = ((w2 * e0[k]).sum() * d11[k] - (w2 * e1[k]).sum() * d01[k]) / den[k]
                    b2 = ((w2 * e1[k]).sum() * d00[k] - (w2 * e0[k]).sum() * d01[k]) / den[k]
                    b0 = 1.0 - b1 - b2
                    bmin = min(b0, b1, b2)
                    mg = min(mg, abs(bmin))
                    if bmin > 0:
                        cnt += 1
                if w < 1e-4:
                    mg = 0.0
            counts[r, c] = cnt
            margin[r, c] = mg
    return counts, margin
