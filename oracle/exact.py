"""Exact-rational RICI for tiny inputs (test infrastructure only).

The same definition as ``rici_oracle.c`` (Section 3.1 of the paper, with the same readings),
evaluated in exact rational arithmetic with ``fractions.Fraction`` instead of FP64.  Inputs
are FP32 numbers (exact rationals); spin normals must have rational frame coefficients,
i.e. nx^2+ny^2 and nx^2+ny^2+nz^2 perfect squares (for example (3, 4, 12)).  The support
radius must be an exact binary fraction.

Besides the counts it returns, per bin, the smallest |value| of any predicate that decided a
count in that bin (or was evaluated there).  Where that margin is comfortably above the
rounding error of FP64 evaluation, the FP64 oracle must agree with these exact counts.
"""
from __future__ import annotations

from fractions import Fraction
from math import isqrt

import numpy as np


def _sqrt_exact(q: Fraction) -> Fraction:
    n, d = q.numerator, q.denominator
    rn, rd = isqrt(n), isqrt(d)
    if rn * rn != n or rd * rd != d:
        raise ValueError(f"{q} is not a rational square; use a Pythagorean spin normal")
    return Fraction(rn, rd)


def frame(nx, ny, nz):
    nx, ny, nz = Fraction(nx), Fraction(ny), Fraction(nz)
    h = _sqrt_exact(nx * nx + ny * ny)
    Nax, Nay = (Fraction(1), Fraction(0)) if h == 0 else (nx / h, ny / h)
    n2x = Nax * nx + Nay * ny
    g = _sqrt_exact(n2x * n2x + nz * nz)
    Nbx, Nbz = (Fraction(0), Fraction(1)) if g == 0 else (n2x / g, nz / g)
    return Nax, Nay, Nbx, Nbz


def project(P, S, fr):
    Nax, Nay, Nbx, Nbz = fr
    px, py, pz = (Fraction(float(P[k])) - S[k] for k in range(3))
    qx = Nax * px + Nay * py
    qy = -Nay * px + Nax * py
    return (Nbz * qx - Nbx * pz, qy, Nbx * qx + Nbz * pz)


def rici_exact(vertices, normals, triangles, origins, support_radius, N):
    """Returns (counts int64 [O,N,N] unsaturated, margins float [O,N,N])."""
    V = np.asarray(vertices, np.float32)
    Nrm = np.asarray(normals, np.float32)
    Tri = np.asarray(triangles, np.int64)
    R = Fraction(float(np.float32(support_radius)))
    alpha2 = [(R * (2 * c + 1) / (2 * N)) ** 2 for c in range(N)]
    beta = [R * (2 * r + 1 - N) / (2 * N) for r in range(N)]
    out = np.zeros((len(origins), N, N), np.int64)
    margin = np.full((len(origins), N, N), np.inf)
    for oi, o in enumerate(origins):
        S = [Fraction(float(V[o, k])) for k in range(3)]
        fr = frame(*(float(Nrm[o, k]) for k in range(3)))
        proj = {}
        for tri in Tri:
            gid = [int(x) for x in tri]
            T = []
            for g in gid:
                if g not in proj:
                    proj[g] = project(V[g], S, fr)
                T.append(proj[g])
            for r in range(N):
                b = beta[r]
                zs = [T[k][2] - b for k in range(3)]
                # a side decision decides whether the triangle crosses this layer at all
                zmin = float(min(abs(z) for z in zs))
                margin[oi, r, :] = np.minimum(margin[oi, r, :], zmin)
                side = [z >= 0 for z in zs]
                if side[0] == side[1] == side[2]:
                    continue
                lone = 0 if (side[0] != side[1] and side[0] != side[2]) else (
                    1 if (side[1] != side[0] and side[1] != side[2]) else 2)
                others = [(lone + 1) % 3, (lone + 2) % 3]
                edges = []
                for ob in others:
                    u, v = (lone, ob) if gid[lone] < gid[ob] else (ob, lone)
                    lam = (b - T[u][2]) / (T[v][2] - T[u][2])
                    E = (T[u][0] + lam * (T[v][0] - T[u][0]), T[u][1] + lam * (T[v][1] - T[u][1]))
                    edges.append(((gid[u], gid[v]), E))
                edges.sort(key=lambda kv: kv[0])
                E0, E1 = edges[0][1], edges[1][1]
                e0 = E0[0] ** 2 + E0[1] ** 2
                e1 = E1[0] ** 2 + E1[1] ** 2
                Dx, Dy = E1[0] - E0[0], E1[1] - E0[1]
                d0 = E0[0] * Dx + E0[1] * Dy
                d1 = E1[0] * Dx + E1[1] * Dy
                cr = E0[0] * Dy - E0[1] * Dx
                dd = Dx * Dx + Dy * Dy
                for c in range(N):
                    a2 = alpha2[c]
                    m = min(abs(e0 - a2), abs(e1 - a2))
                    in0, in1 = e0 >= a2, e1 >= a2
                    if in0 != in1:
                        out[oi, r, c] += 1
                    elif in0 and in1:
                        m = min(m, abs(d0), abs(d1))
                        if d0 < 0 and d1 > 0:
                            q = a2 * dd - cr * cr
                            m = min(m, abs(q))
                            if q > 0:
                                out[oi, r, c] += 2
                    margin[oi, r, c] = min(margin[oi, r, c], float(m))
    return out, margin
