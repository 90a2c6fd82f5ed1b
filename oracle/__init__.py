"""FP64 CPU oracle for the simplex-domain hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package.  It wraps ``oracle.c`` (plain C, nested loops, FP64)
through ctypes and shares nothing with the CUDA library.

Every function takes NumPy arrays; point arrays are converted to FP64 (the
FP32 inputs of the CUDA path are exactly representable).

Parity status of each function (what pins it, see ``tests/test_oracle.py``):

* ``table2`` / ``table3`` (recursive construction of S_n^2, S_n^3, Sec. III-A
  and III-C), ``bbox``/``linear`` tables: pinned by brute-force bijection
  checks, the closed-form volumes of Eq. 2 and eq. (m2)/(m3), the extra-volume
  limits of Sec. III-C, and the paper's closed-form lambda of eq. (map2d).
* ``table4`` (S_n^4 with r = 1/2, beta = 2, Sec. III-D, built from its cross
  terms): pinned by a brute-force check that every block I <= J <= K < L
  appears once and no grid point twice, V(S_n^4) = (n^4 - n)/14 and the
  extra-volume limit 5/7 of Sec. III-D.
* ``cover2`` / ``cover3`` / ``cover4``: pinned by V(Delta_n^2) = n(n+1)/2,
  V(Delta_n^3) = n(n+1)(n+2)/6, V(Delta_n^4) = C(n+3, 4) and by brute-force
  idle counts.
* ``edm_packed`` / ``edm_pairs``: pinned by closed forms on a line and a
  lattice, scaling, translation and permutation invariance.
* ``edm_tiles``: pinned by points on a line, where each entry's value
  (i - j)^2 names its pair: the tiles, walked in the triangle's order by
  nested loops, equal the blocks of the full square matrix; padding 0.
* ``atm_energy`` / ``atm_atom_energy`` / ``atm_grad`` / ``atm_grad_atoms``:
  pinned by closed-form triangles (equilateral, collinear, right angle), a
  pure-Python brute force using angles, invariances, Euler's theorem for a
  homogeneous function and FD of the energy.
* ``atm_energy_grad_slice``: pinned by FD of its own energy (a sum of terms
  whose gradient it returns) and by slices that partition the total energy
  and gradient.
* ``atm_grad_abs`` (per atom, the sum of the magnitudes of its gradient's
  per-side parts): pinned by the equilateral triangle, where the two parts
  at each atom have equal length at 60 degrees so the sum is 2/sqrt(3) times
  the gradient's norm whatever the derivative's value, by a collinear
  triple with an end atom (parallel parts: equal to the norm, or the norm
  of the difference when the parts oppose), and by sum >= |gradient| on a
  cloud.
* ``atm_abs_energy`` (sum of |e|): pinned by the closed-form triangles in
  absolute value, a pure-Python brute force of sum |e| on a cloud with terms
  of both signs, and equality with E on a regular tetrahedron.
* ``stress_loss`` / ``stress_grad_rows``: pinned by the two-point closed form,
  the zero at y = x, translation invariance and FD.
* ``stress_loss_rows``: pinned by the moment-matrix form of the loss (rows
  partition it) and the two-point closed form on its one row.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MAP_LAMBDA, MAP_BBOX, MAP_LINEAR, MAP_RB = 0, 1, 2, 3
MAPS = {"lambda": MAP_LAMBDA, "bbox": MAP_BBOX, "linear": MAP_LINEAR, "rb": MAP_RB}


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (no FP contraction, so the
    results agree across hosts)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC",
                               "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_i64, _i32p, _i64p = ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
_dp, _d = ctypes.POINTER(ctypes.c_double), ctypes.c_double


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        sig = {
            "oracle_grid2": (_i64, [_i64, ctypes.c_int, _i64p, _i64p]),
            "oracle_grid3": (_i64, [_i64, ctypes.c_int, _i64p, _i64p, _i64p]),
            "oracle_table2": (_i64, [_i64, ctypes.c_int, _i32p]),
            "oracle_table3": (_i64, [_i64, ctypes.c_int, _i32p]),
            "oracle_cover2": (_i64, [_i64, _i64, ctypes.c_int, _i32p]),
            "oracle_cover3": (_i64, [_i64, _i64, ctypes.c_int, _i32p]),
            "oracle_grid4": (_i64, [_i64, ctypes.c_int, _i64p, _i64p, _i64p, _i64p]),
            "oracle_table4": (_i64, [_i64, ctypes.c_int, _i32p]),
            "oracle_volume4": (_i64, [_i64]),
            "oracle_cover4": (_i64, [_i64, _i64, ctypes.c_int, _i32p]),
            "oracle_edm_packed": (None, [_i64, _i64, _dp, _dp]),
            "oracle_edm_tiles": (None, [_i64, _i64, _dp, _dp]),
            "oracle_atm_energy_grad_slice": (_d, [_i64, _dp, _d, _d, _i64, _i64, _dp]),
            "oracle_stress_loss_rows": (_d, [_i64, _i64, _dp, _dp, _i64, _i64]),
            "oracle_edm_pairs": (None, [_i64, _dp, _i64p, _i64, _dp]),
            "oracle_atm_energy": (_d, [_i64, _dp, _d, _d]),
            "oracle_atm_energy_slice": (_d, [_i64, _dp, _d, _d, _i64, _i64]),
            "oracle_atm_abs_energy": (_d, [_i64, _dp, _d, _d]),
            "oracle_atm_atom_energy": (_d, [_i64, _dp, _i64, _d, _d]),
            "oracle_atm_grad": (None, [_i64, _dp, _d, _d, _dp]),
            "oracle_atm_grad_atoms": (None, [_i64, _dp, _d, _d, _i64p, _i64, _dp]),
            "oracle_atm_grad_abs": (None, [_i64, _dp, _d, _d, _dp]),
            "oracle_stress_loss": (_d, [_i64, _i64, _dp, _dp]),
            "oracle_stress_grad_rows": (None, [_i64, _i64, _dp, _dp, _i64p, _i64, _dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _map(m):
    return MAPS[m] if isinstance(m, str) else int(m)


# ---------------------------------------------------------------- maps

def grid2(nb: int, m) -> tuple[int, int]:
    gx, gy = ctypes.c_int64(), ctypes.c_int64()
    lib().oracle_grid2(nb, _map(m), ctypes.byref(gx), ctypes.byref(gy))
    return gx.value, gy.value


def grid3(nb: int, m) -> tuple[int, int, int]:
    gx, gy, gz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib().oracle_grid3(nb, _map(m), ctypes.byref(gx), ctypes.byref(gy), ctypes.byref(gz))
    return gx.value, gy.value, gz.value


def table2(nb: int, m) -> np.ndarray:
    """(grid, 4) int32: per grid block (X0, Y0, X1, Y1), -1 where unused."""
    gx, gy = grid2(nb, m)
    t = np.empty((gx * gy, 4), dtype=np.int32)
    lib().oracle_table2(nb, _map(m), _p(t, ctypes.c_int32))
    return t


def table3(nb: int, m) -> np.ndarray:
    """(grid, 6) int32: per grid block (I0, J0, K0, I1, J1, K1), -1 where unused."""
    gx, gy, gz = grid3(nb, m)
    t = np.empty((gx * gy * gz, 6), dtype=np.int32)
    lib().oracle_table3(nb, _map(m), _p(t, ctypes.c_int32))
    return t


def grid4(nb: int, m) -> tuple[int, int, int, int]:
    g = [ctypes.c_int64() for _ in range(4)]
    lib().oracle_grid4(nb, _map(m), *[ctypes.byref(v) for v in g])
    return tuple(v.value for v in g)


def table4(nb: int, m) -> np.ndarray:
    """(grid, 8) int32: per grid block (I, J, K, L, -1, -1, -1, -1), -1 where
    unused; lambda holds the blocks I <= J <= K < L.  Raises if two cross
    terms land on one grid point."""
    gx, gy, gz, gw = grid4(nb, m)
    t = np.empty((gx * gy * gz * gw, 8), dtype=np.int32)
    if lib().oracle_table4(nb, _map(m), _p(t, ctypes.c_int32)) < 0:
        raise RuntimeError("m = 4 placement collision")
    return t


def volume4(s: int) -> int:
    """Grid points of the recursive set S_s^4 (mapped or idle)."""
    return int(lib().oracle_volume4(s))


def cover4(n: int, rho: int, m) -> tuple[np.ndarray, int]:
    c = np.zeros(n * (n + 1) * (n + 2) * (n + 3) // 24, dtype=np.int32)
    idle = lib().oracle_cover4(n, rho, _map(m), _p(c, ctypes.c_int32))
    if idle < 0:
        raise RuntimeError("m = 4 placement collision")
    return c, int(idle)


def cover2(n: int, rho: int, m) -> tuple[np.ndarray, int]:
    c = np.zeros(n * (n + 1) // 2, dtype=np.int32)
    idle = lib().oracle_cover2(n, rho, _map(m), _p(c, ctypes.c_int32))
    return c, int(idle)


def cover3(n: int, rho: int, m) -> tuple[np.ndarray, int]:
    c = np.zeros(n * (n + 1) * (n + 2) // 6, dtype=np.int32)
    idle = lib().oracle_cover3(n, rho, _map(m), _p(c, ctypes.c_int32))
    return c, int(idle)


# ---------------------------------------------------------------- EDM

def edm_packed(x: np.ndarray) -> np.ndarray:
    x = _f64(x)
    n, d = x.shape
    out = np.empty(n * (n + 1) // 2, dtype=np.float64)
    lib().oracle_edm_packed(n, d, _p(x, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def edm_tiles(x: np.ndarray) -> np.ndarray:
    """Tile-packed EDM: tiles (I, J), J <= I, of 128 x 128 in packed lower
    order, each row-major; diagonal tiles whole, padding 0."""
    x = _f64(x)
    n, d = x.shape
    nt = (n + 127) // 128
    out = np.empty(nt * (nt + 1) // 2 * 128 * 128, dtype=np.float64)
    lib().oracle_edm_tiles(n, d, _p(x, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def edm_pairs(x: np.ndarray, pairs: np.ndarray) -> np.ndarray:
    x = _f64(x)
    pr = np.ascontiguousarray(pairs, dtype=np.int64)
    out = np.empty(len(pr), dtype=np.float64)
    lib().oracle_edm_pairs(x.shape[1], _p(x, ctypes.c_double), _p(pr, ctypes.c_int64),
                           len(pr), _p(out, ctypes.c_double))
    return out


# ---------------------------------------------------------------- ATM

def atm_energy(x: np.ndarray, nu: float = 1.0, eps: float = 1e-4) -> float:
    x = _f64(x)
    return lib().oracle_atm_energy(len(x), _p(x, ctypes.c_double), nu, eps)


def atm_energy_slice(x: np.ndarray, i_lo: int, i_hi: int, nu: float = 1.0,
                     eps: float = 1e-4) -> float:
    x = _f64(x)
    return lib().oracle_atm_energy_slice(len(x), _p(x, ctypes.c_double), nu, eps, i_lo, i_hi)


def atm_abs_energy(x: np.ndarray, nu: float = 1.0, eps: float = 1e-4) -> float:
    x = _f64(x)
    return lib().oracle_atm_abs_energy(len(x), _p(x, ctypes.c_double), nu, eps)


def atm_atom_energy(x: np.ndarray, a: int, nu: float = 1.0, eps: float = 1e-4) -> float:
    x = _f64(x)
    return lib().oracle_atm_atom_energy(len(x), _p(x, ctypes.c_double), a, nu, eps)


def atm_grad(x: np.ndarray, nu: float = 1.0, eps: float = 1e-4) -> np.ndarray:
    x = _f64(x)
    g = np.empty_like(x)
    lib().oracle_atm_grad(len(x), _p(x, ctypes.c_double), nu, eps, _p(g, ctypes.c_double))
    return g


def atm_grad_abs(x: np.ndarray, nu: float = 1.0, eps: float = 1e-4) -> np.ndarray:
    """Per atom, the sum of the magnitudes of the per-side parts of its
    gradient (2 |de/ds| |x_a - x_b| over its triples): the scale of the
    rounding error of an FP32 evaluation of that gradient."""
    x = _f64(x)
    out = np.empty(len(x))
    lib().oracle_atm_grad_abs(len(x), _p(x, ctypes.c_double), nu, eps, _p(out, ctypes.c_double))
    return out


def atm_energy_grad_slice(x: np.ndarray, i_lo: int, i_hi: int, nu: float = 1.0,
                          eps: float = 1e-4, grad: np.ndarray | None = None):
    """(energy, gradient) of the triples with i in [i_lo, i_hi); the gradient
    is added into `grad` when one is given (n x 3 FP64)."""
    x = _f64(x)
    g = np.zeros_like(x) if grad is None else grad
    e = lib().oracle_atm_energy_grad_slice(len(x), _p(x, ctypes.c_double), nu, eps, i_lo, i_hi,
                                           _p(g, ctypes.c_double))
    return e, g


def atm_grad_atoms(x: np.ndarray, atoms, nu: float = 1.0, eps: float = 1e-4) -> np.ndarray:
    x = _f64(x)
    a = np.ascontiguousarray(atoms, dtype=np.int64)
    g = np.empty((len(a), 3), dtype=np.float64)
    lib().oracle_atm_grad_atoms(len(x), _p(x, ctypes.c_double), nu, eps,
                                _p(a, ctypes.c_int64), len(a), _p(g, ctypes.c_double))
    return g


# ---------------------------------------------------------------- stress

def stress_loss_rows(x: np.ndarray, y: np.ndarray, i_lo: int, i_hi: int) -> float:
    """Loss terms of the rows i in [i_lo, i_hi) (pairs j < i)."""
    x, y = _f64(x), _f64(y)
    n, d = x.shape
    return lib().oracle_stress_loss_rows(n, d, _p(x, ctypes.c_double), _p(y, ctypes.c_double), i_lo, i_hi)


def stress_loss(x: np.ndarray, y: np.ndarray) -> float:
    x, y = _f64(x), _f64(y)
    n, d = x.shape
    return lib().oracle_stress_loss(n, d, _p(x, ctypes.c_double), _p(y, ctypes.c_double))


def stress_grad_rows(x: np.ndarray, y: np.ndarray, rows) -> np.ndarray:
    x, y = _f64(x), _f64(y)
    n, d = x.shape
    r = np.ascontiguousarray(rows, dtype=np.int64)
    g = np.empty((len(r), d), dtype=np.float64)
    lib().oracle_stress_grad_rows(n, d, _p(x, ctypes.c_double), _p(y, ctypes.c_double),
                                  _p(r, ctypes.c_int64), len(r), _p(g, ctypes.c_double))
    return g
