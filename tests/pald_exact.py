"""Independent reference formulations used only to pin the oracle.

* ``exact_pald``: exact rational arithmetic, enumerating the random variables
  of the paper's probabilistic definition (Sec. 2, eqs. (LD) and (cohesion))
  directly: Y uniform on S minus {x}, then Z uniform on the focus U_xY, then
  the event "Z is closer to x than to Y" (half on a tie, Sec. 5).
* ``pairwise_alg`` and ``triplet_alg``: the two entry-wise algorithms of
  Sec. 3 (Alg. 1 and Alg. 2), restated.  They use strict comparisons and no
  tie split, so they agree with the definition only on tie-free inputs; they
  also leave out the 1/(n-1) factor, and Alg. 2 never visits the diagonal
  of C.  On tie-free inputs they give two further formulations the oracle must
  agree with.

None of this code is shared with the oracle or with the CUDA path.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def load_golden(path):
    """Parse tests/golden/hand_worked.txt into a list of dicts."""
    cases, cur, key, rows = [], None, None, []

    def flush():
        nonlocal key, rows
        if cur is not None and key is not None:
            cur[key] = rows
        key, rows = None, []

    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("case "):
                flush()
                cur = {"name": line.split()[1]}
                cases.append(cur)
            elif line in ("D", "u", "C"):
                flush()
                key = line
            else:
                rows.append([Fraction(t) for t in line.split()])
        flush()
    return cases


def _support(dzx, dzy) -> Fraction:
    if dzx < dzy:
        return Fraction(1)
    if dzx == dzy:
        return Fraction(1, 2)
    return Fraction(0)


def exact_pald(D):
    """Exact (u, C) by enumeration of (Y, Z); D holds exact numbers."""
    n = len(D)
    d = [[Fraction(v) for v in row] for row in D]
    focus = [[[z for z in range(n) if d[x][z] <= d[x][y] or d[y][z] <= d[x][y]]
              for y in range(n)] for x in range(n)]
    u = [[len(focus[x][y]) for y in range(n)] for x in range(n)]
    C = [[Fraction(0) for _ in range(n)] for _ in range(n)]
    for x in range(n):
        p_y = Fraction(1, n - 1)
        for y in range(n):
            if y == x:
                continue
            members = focus[x][y]
            p_z = Fraction(1, len(members))
            for z in members:
                C[x][z] += p_y * p_z * _support(d[z][x], d[z][y])
    return u, C


def local_depth_exact(D, x):
    """Eq. (LD): Pr[d_Zx < d_ZY] (ties counted half), evaluated directly."""
    n = len(D)
    d = [[Fraction(v) for v in row] for row in D]
    total = Fraction(0)
    for y in range(n):
        if y == x:
            continue
        members = [z for z in range(n) if d[x][z] <= d[x][y] or d[y][z] <= d[x][y]]
        hits = sum((_support(d[z][x], d[z][y]) for z in members), Fraction(0))
        total += Fraction(1, n - 1) * hits / len(members)
    return total


def pairwise_alg(D):
    """Alg. 1 (pairwise): returns (u for x<y, unnormalised C incl. diagonal)."""
    D = np.asarray(D, dtype=np.float64)
    n = D.shape[0]
    U = np.zeros((n, n), dtype=np.int64)
    C = np.zeros((n, n), dtype=np.float64)
    for x in range(n - 1):
        for y in range(x + 1, n):
            inside = (D[x] < D[x, y]) | (D[y] < D[x, y])      # focus, strict
            u = int(inside.sum())
            U[x, y] = U[y, x] = u
            closer_x = D[x] < D[y]                           # which side z supports
            C[x] += np.where(inside & closer_x, 1.0 / u, 0.0)
            C[y] += np.where(inside & ~closer_x, 1.0 / u, 0.0)
    return U, C


def triplet_alg(D):
    """Alg. 2 (triplet): returns (u for x<y, unnormalised off-diagonal C)."""
    D = np.asarray(D, dtype=np.float64)
    n = D.shape[0]
    U = np.zeros((n, n), dtype=np.int64)
    for x in range(n):
        for y in range(x + 1, n):
            U[x, y] = 2                                      # x and y themselves
    for x in range(n - 1):
        for y in range(x + 1, n):
            for z in range(y + 1, n):
                if D[x, y] < D[x, z] and D[x, y] < D[y, z]:   # x,y closest
                    U[x, z] += 1
                    U[y, z] += 1
                elif D[x, z] < D[y, z]:                       # x,z closest
                    U[x, y] += 1
                    U[y, z] += 1
                else:                                         # y,z closest
                    U[x, y] += 1
                    U[x, z] += 1
    U = U + U.T
    C = np.zeros((n, n), dtype=np.float64)
    for x in range(n - 1):
        for y in range(x + 1, n):
            for z in range(y + 1, n):
                if D[x, y] < D[x, z] and D[x, y] < D[y, z]:
                    C[x, y] += 1.0 / U[x, z]
                    C[y, x] += 1.0 / U[y, z]
                elif D[x, z] < D[y, z]:
                    C[x, z] += 1.0 / U[x, y]
                    C[z, x] += 1.0 / U[y, z]
                else:
                    C[y, z] += 1.0 / U[x, y]
                    C[z, y] += 1.0 / U[x, z]
    return U, C
