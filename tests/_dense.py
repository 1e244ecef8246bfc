"""Dense-matrix helpers for tiny grids (test infrastructure).

They rebuild A, L and U as dense numpy matrices by explicit (i, j, k)
neighbour enumeration, so that statements about the SIP factorisation can be
checked with plain linear algebra instead of re-running the recurrences.
"""
import numpy as np

# neighbour offsets (di, dj, dk) of the 7-point stencil
OFF = {"W": (-1, 0, 0), "E": (1, 0, 0), "S": (0, -1, 0), "N": (0, 1, 0), "B": (0, 0, -1), "T": (0, 0, 1)}
COEF_OF = {"W": "aw", "E": "ae", "S": "as", "N": "an", "B": "ab", "T": "at"}
# Stone's six fill positions of L U and the two stencil neighbours that
# flank each of them (linear extrapolation x_fill ~ x_a + x_b - x_P)
FILLS = {
    "BE": ((1, 0, -1), ("B", "E")),
    "BN": ((0, 1, -1), ("B", "N")),
    "SE": ((1, -1, 0), ("S", "E")),
    "ST": ((0, -1, 1), ("S", "T")),
    "WN": ((-1, 1, 0), ("W", "N")),
    "WT": ((-1, 0, 1), ("W", "T")),
}


def idx(nx, ny, i, j, k):
    return i + nx * (j + ny * k)


def cells(nx, ny, nz):
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                yield i, j, k


def inside(nx, ny, nz, i, j, k):
    return 0 <= i < nx and 0 <= j < ny and 0 <= k < nz


def dense_A(nx, ny, nz, coefs):
    n = nx * ny * nz
    A = np.zeros((n, n))
    for i, j, k in cells(nx, ny, nz):
        p = idx(nx, ny, i, j, k)
        A[p, p] = coefs["ap"][p]
        for nb, (di, dj, dk) in OFF.items():
            if inside(nx, ny, nz, i + di, j + dj, k + dk):
                A[p, idx(nx, ny, i + di, j + dj, k + dk)] = coefs[COEF_OF[nb]][p]
    return A


def dense_LU(nx, ny, nz, factors):
    lb, lw, ls, lp, un, ue, ut = factors
    n = nx * ny * nz
    L = np.zeros((n, n))
    U = np.eye(n)
    for i, j, k in cells(nx, ny, nz):
        p = idx(nx, ny, i, j, k)
        L[p, p] = lp[p]
        for nb, arr in (("W", lw), ("S", ls), ("B", lb)):
            di, dj, dk = OFF[nb]
            if inside(nx, ny, nz, i + di, j + dj, k + dk):
                L[p, idx(nx, ny, i + di, j + dj, k + dk)] = arr[p]
        for nb, arr in (("E", ue), ("N", un), ("T", ut)):
            di, dj, dk = OFF[nb]
            if inside(nx, ny, nz, i + di, j + dj, k + dk):
                U[p, idx(nx, ny, i + di, j + dj, k + dk)] = arr[p]
    return L, U


def pattern7(nx, ny, nz):
    n = nx * ny * nz
    P = np.zeros((n, n), dtype=bool)
    for i, j, k in cells(nx, ny, nz):
        p = idx(nx, ny, i, j, k)
        P[p, p] = True
        for di, dj, dk in OFF.values():
            if inside(nx, ny, nz, i + di, j + dj, k + dk):
                P[p, idx(nx, ny, i + di, j + dj, k + dk)] = True
    return P


def ilu0(A, pattern):
    """Textbook ILU(0) (IKJ variant, e.g. Saad, Iterative Methods, Alg. 10.4):
    returns the product L_unit @ U restricted to the given sparsity pattern."""
    a = A.copy()
    n = a.shape[0]
    for i in range(1, n):
        for k in range(i):
            if not pattern[i, k]:
                continue
            a[i, k] /= a[k, k]
            for j in range(k + 1, n):
                if pattern[i, j]:
                    a[i, j] -= a[i, k] * a[k, j]
    Lu = np.tril(a, -1) + np.eye(n)
    U = np.triu(a)
    return Lu @ U
