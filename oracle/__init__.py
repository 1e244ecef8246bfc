"""CPU oracle for Stone's SIP (plain C in sip_oracle.c, FP64; ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by the cpu_baseline / reference legs of bench.py, nowhere else.  It shares no
code with the CUDA path (paper_1303_4538_gb300/csrc) and does not import it.

Every function follows the paper's SIP (arXiv:1303.4538, Sec. 1 and Sec. 4.1:
factorisation lu3d, fused residual + forward substitution resforward3d,
backward substitution backward3d, single-precision relaxation).  The formulas
are restated in the header comment of sip_oracle.c.  Arrays are numpy, flat,
natural layout p = i + nx*(j + ny*k).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sip_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
COEF_NAMES = ("ap", "aw", "ae", "as", "an", "ab", "at")
_lib = None


def build(force: bool = False) -> str:
    """Compile sip_oracle.c with gcc -O2 -ffp-contract=off (no FMA contraction,
    so x86 and Arm hosts round identically)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        L.oracle_dot_sq.argtypes = [ctypes.c_int64, P]
        L.oracle_dot_sq.restype = D
        L.oracle_factor.argtypes = [I, I, I, D] + [P] * 14
        L.oracle_factor.restype = I
        L.oracle_residual.argtypes = [I, I, I] + [P] * 10
        L.oracle_residual.restype = D
        L.oracle_residual_sym.argtypes = [I, I, I] + [P] * 7
        L.oracle_residual_sym.restype = D
        L.oracle_forward.argtypes = [I, I, I] + [P] * 6
        L.oracle_forward.restype = None
        L.oracle_backward.argtypes = [I, I, I] + [P] * 5
        L.oracle_backward.restype = None
        L.oracle_iterate.argtypes = [I, I, I] + [P] * 19
        L.oracle_iterate.restype = D
        L.oracle_solve.argtypes = [I, I, I] + [P] * 16 + [D, I, P, P]
        L.oracle_solve.restype = I
        L.oracle_iterate_f32.argtypes = [I, I, I] + [P] * 16 + [I, P, P, P]
        L.oracle_iterate_f32.restype = None
        L.oracle_solve_refined.argtypes = [I, I, I] + [P] * 23 + [D, I, I, P, P]
        L.oracle_solve_refined.restype = I
        L.oracle_solve_f32.argtypes = [I, I, I] + [P] * 16 + [D, I, P, P]
        L.oracle_solve_f32.restype = I
        L.oracle_solve_mb.argtypes = [I, P, P, P, P, P, I, P, I, D, I, P, P]
        L.oracle_solve_mb.restype = I
        L.oracle_solve_refined_mb.argtypes = [I, P, P, P, P, P, P, I, P, I, D, I, I, P, P]
        L.oracle_solve_refined_mb.restype = I
        L.oracle_assemble_pcorr.argtypes = [I, I, I] + [P] * 8 + [I] + [P] * 8
        L.oracle_assemble_pcorr.restype = None
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64).reshape(-1)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32).reshape(-1)


def _coefs(coefs, conv=_f64) -> List[np.ndarray]:
    if isinstance(coefs, dict):
        return [conv(coefs[k]) for k in COEF_NAMES]
    return [conv(c) for c in coefs]


class BreakdownError(ArithmeticError):
    pass


def factor(nx: int, ny: int, nz: int, coefs, alpha: float) -> Tuple[np.ndarray, ...]:
    """Stone factorisation; returns (LB, LW, LS, LP, UN, UE, UT), FP64."""
    A = _coefs(coefs)
    n = nx * ny * nz
    F = [np.zeros(n) for _ in range(7)]
    rc = lib().oracle_factor(nx, ny, nz, float(alpha), *[_p(a) for a in A], *[_p(f) for f in F])
    if rc != 0:
        raise BreakdownError(f"SIP factorisation breaks down at cell {-1 - rc}")
    return tuple(F)


def residual(nx, ny, nz, coefs, b, x) -> Tuple[np.ndarray, float]:
    """r = b - A x and ||r||_2."""
    A = _coefs(coefs)
    b = _f64(b)
    x = _f64(x)
    r = np.zeros(nx * ny * nz)
    rr = lib().oracle_residual(nx, ny, nz, *[_p(a) for a in A], _p(b), _p(x), _p(r))
    return r, float(np.sqrt(rr))


def residual_sym(nx, ny, nz, ap, ae, an, at, b, x) -> Tuple[np.ndarray, float]:
    """Residual in the symmetric form of the paper's Listing 1."""
    arrs = [_f64(a) for a in (ap, ae, an, at, b, x)]
    r = np.zeros(nx * ny * nz)
    rr = lib().oracle_residual_sym(nx, ny, nz, *[_p(a) for a in arrs], _p(r))
    return r, float(np.sqrt(rr))


def forward(nx, ny, nz, factors, r) -> np.ndarray:
    lb, lw, ls, lp = [_f64(f) for f in factors[:4]]
    r = _f64(r)
    y = np.zeros(nx * ny * nz)
    lib().oracle_forward(nx, ny, nz, _p(lb), _p(lw), _p(ls), _p(lp), _p(r), _p(y))
    return y


def backward(nx, ny, nz, factors, y) -> np.ndarray:
    un, ue, ut = [_f64(f) for f in factors[4:7]]
    y = _f64(y)
    d = np.zeros(nx * ny * nz)
    lib().oracle_backward(nx, ny, nz, _p(un), _p(ue), _p(ut), _p(y), _p(d))
    return d


def iterate(nx, ny, nz, coefs, factors, b, x: np.ndarray) -> float:
    """One SIP iteration on x (in place, x must be a contiguous float64 array).
    Returns ||b - A x_in||_2."""
    assert x.dtype == np.float64 and x.flags.c_contiguous
    A = _coefs(coefs)
    F = [_f64(f) for f in factors]
    b = _f64(b)
    n = nx * ny * nz
    w = [np.zeros(n) for _ in range(3)]
    rr = lib().oracle_iterate(nx, ny, nz, *[_p(a) for a in A], *[_p(f) for f in F], _p(b), _p(x),
                              *[_p(v) for v in w])
    return float(np.sqrt(rr))


def solve(nx, ny, nz, coefs, factors, b, x0=None, rtol=1e-8, max_iters=100):
    """SIP to relres <= rtol (stop rule: relres of x_n from the residual of
    x_n; stop at the first n with relres <= rtol or n == max_iters).
    Returns (x, n, relres, hist[0..n])."""
    A = _coefs(coefs)
    F = [_f64(f) for f in factors]
    b = _f64(b)
    n = nx * ny * nz
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    hist = np.zeros(max_iters + 1)
    rel = ctypes.c_double(0.0)
    it = lib().oracle_solve(nx, ny, nz, *[_p(a) for a in A], *[_p(f) for f in F], _p(b), _p(x),
                            float(rtol), int(max_iters), _p(hist), ctypes.byref(rel))
    return x, it, rel.value, hist[: it + 1].copy()


def factors_f32(factors) -> Tuple[np.ndarray, ...]:
    """Single-precision factors: the FP64 factors rounded to float."""
    return tuple(_f32(f) for f in factors)


def iterate_f32(nx, ny, nz, coefs32, factors32, b32, x32: np.ndarray, x_is_zero=False) -> None:
    """One SIP iteration in float arithmetic on x32 (in place)."""
    assert x32.dtype == np.float32 and x32.flags.c_contiguous
    A = _coefs(coefs32, _f32)
    F = [_f32(f) for f in factors32]
    b32 = _f32(b32)
    n = nx * ny * nz
    w = [np.zeros(n, np.float32) for _ in range(3)]
    lib().oracle_iterate_f32(nx, ny, nz, *[_p(a) for a in A], *[_p(f) for f in F], _p(b32),
                             _p(x32), int(bool(x_is_zero)), *[_p(v) for v in w])


def solve_refined(nx, ny, nz, coefs64, coefs32, factors32, b, x0=None, rtol=1e-8,
                  max_outer=100, m_inner=4):
    """FP64 iterative refinement around m single-precision SIP iterations.
    Returns (x, outer_corrections, relres, hist)."""
    A64 = _coefs(coefs64)
    A32 = _coefs(coefs32, _f32)
    F = [_f32(f) for f in factors32]
    b = _f64(b)
    n = nx * ny * nz
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    hist = np.zeros(max_outer + 1)
    rel = ctypes.c_double(0.0)
    it = lib().oracle_solve_refined(nx, ny, nz, *[_p(a) for a in A64], *[_p(a) for a in A32],
                                    *[_p(f) for f in F], _p(b), _p(x), float(rtol), int(max_outer),
                                    int(m_inner), _p(hist), ctypes.byref(rel))
    return x, it, rel.value, hist[: it + 1].copy()


def solve_f32(nx, ny, nz, coefs32, factors32, b, x0=None, rtol=1e-8, max_iters=100):
    """The paper's single-precision SIP (Sec. 4.1): float copies of A, of the
    factors, of b and x; returns (x (FP64), n, relres, hist)."""
    A32 = _coefs(coefs32, _f32)
    F = [_f32(f) for f in factors32]
    b = _f64(b)
    n = nx * ny * nz
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    hist = np.zeros(max_iters + 1)
    rel = ctypes.c_double(0.0)
    it = lib().oracle_solve_f32(nx, ny, nz, *[_p(a) for a in A32], *[_p(f) for f in F], _p(b), _p(x),
                                float(rtol), int(max_iters), _p(hist), ctypes.byref(rel))
    return x, it, rel.value, hist[: it + 1].copy()


def solve_multiblock(blocks, ifaces, factors, x0=None, rtol=1e-8, max_iters=100, symmetric=False):
    """Lagged block-Jacobi SIP over blocks coupled across x interfaces.

    blocks: list of (nx, ny, nz, coefs, b); ifaces: list of (lo, hi, nj, nk);
    factors: per block the 7 FP64 factor arrays (oracle.factor); x0: list of
    per-block initial guesses (default zeros).  Returns (xs, n, relres, hist)."""
    nb = len(blocks)
    dims = np.array([[bl[0], bl[1], bl[2]] for bl in blocks], dtype=np.int32).reshape(-1)
    A = [_coefs(bl[3]) for bl in blocks]
    F = [[_f64(f) for f in fs] for fs in factors]
    B = [_f64(bl[4]) for bl in blocks]
    X = [np.zeros(bl[0] * bl[1] * bl[2]) if x0 is None else _f64(x0[i]).copy() for i, bl in enumerate(blocks)]
    Pa = (ctypes.c_void_p * (7 * nb))(*[a.ctypes.data for arrs in A for a in arrs])
    Pf = (ctypes.c_void_p * (7 * nb))(*[f.ctypes.data for fs in F for f in fs])
    Pb = (ctypes.c_void_p * nb)(*[b.ctypes.data for b in B])
    Px = (ctypes.c_void_p * nb)(*[x.ctypes.data for x in X])
    ifc = np.array([list(q) for q in ifaces], dtype=np.int32).reshape(-1) if ifaces else np.zeros(4, np.int32)
    hist = np.zeros(max_iters + 1)
    rel = ctypes.c_double(0.0)
    it = lib().oracle_solve_mb(nb, _p(dims), Pa, Pf, Pb, Px, len(ifaces), _p(ifc), 1 if symmetric else 0,
                               float(rtol), int(max_iters), _p(hist), ctypes.byref(rel))
    return X, it, rel.value, hist[: it + 1].copy()


def solve_refined_multiblock(blocks, ifaces, coefs32, factors32, x0=None, rtol=1e-8, max_outer=100, m_inner=4,
                             symmetric=False):
    """FP64 refinement around m single-precision SIP iterations over blocks
    coupled across x interfaces, the blocks exchanging their interface values
    of the correction after every inner iteration.

    blocks: list of (nx, ny, nz, coefs64, b); coefs32: per block the FP32
    coefficient dict; factors32: per block the 7 FP32 factor arrays.
    Returns (xs, outer_corrections, relres, hist)."""
    nb = len(blocks)
    dims = np.array([[bl[0], bl[1], bl[2]] for bl in blocks], dtype=np.int32).reshape(-1)
    A = [_coefs(bl[3]) for bl in blocks]
    A32 = [_coefs(c, _f32) for c in coefs32]
    F = [[_f32(f) for f in fs] for fs in factors32]
    B = [_f64(bl[4]) for bl in blocks]
    X = [np.zeros(bl[0] * bl[1] * bl[2]) if x0 is None else _f64(x0[i]).copy() for i, bl in enumerate(blocks)]
    Pa = (ctypes.c_void_p * (7 * nb))(*[a.ctypes.data for arrs in A for a in arrs])
    Pa32 = (ctypes.c_void_p * (7 * nb))(*[a.ctypes.data for arrs in A32 for a in arrs])
    Pf = (ctypes.c_void_p * (7 * nb))(*[f.ctypes.data for fs in F for f in fs])
    Pb = (ctypes.c_void_p * nb)(*[b.ctypes.data for b in B])
    Px = (ctypes.c_void_p * nb)(*[x.ctypes.data for x in X])
    ifc = np.array([list(q) for q in ifaces], dtype=np.int32).reshape(-1) if ifaces else np.zeros(4, np.int32)
    hist = np.zeros(max_outer + 1)
    rel = ctypes.c_double(0.0)
    it = lib().oracle_solve_refined_mb(nb, _p(dims), Pa, Pa32, Pf, Pb, Px, len(ifaces), _p(ifc),
                                       1 if symmetric else 0, float(rtol), int(max_outer), int(m_inner),
                                       _p(hist), ctypes.byref(rel))
    return X, it, rel.value, hist[: it + 1].copy()


def assemble_pcorr(nx, ny, nz, dx, dy, dz, rho, g, ux, uy, uz, dirichlet_bottom=True):
    """Pressure-correction coefficients and right-hand side of one block on a
    rectilinear grid (the routine celp2 of Sec. 3.1).  Returns (coefs, b):
    coefs a dict ap, aw, ae, as, an, ab, at of natural-layout FP64 arrays."""
    n = nx * ny * nz
    ins = [_f64(v) for v in (dx, dy, dz, rho, g, ux, uy, uz)]
    assert ins[0].size == nx and ins[1].size == ny and ins[2].size == nz
    assert ins[3].size == n and ins[4].size == n
    assert ins[5].size == (nx + 1) * ny * nz and ins[6].size == nx * (ny + 1) * nz
    assert ins[7].size == nx * ny * (nz + 1)
    out = [np.zeros(n) for _ in range(8)]
    lib().oracle_assemble_pcorr(nx, ny, nz, *[_p(v) for v in ins], 1 if dirichlet_bottom else 0,
                                *[_p(v) for v in out])
    return dict(zip(COEF_NAMES, out[:7])), out[7]


def norm2(v) -> float:
    v = _f64(v)
    return float(np.sqrt(lib().oracle_dot_sq(v.size, _p(v))))
