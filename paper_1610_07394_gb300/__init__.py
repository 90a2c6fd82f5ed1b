"""libsimplex: recursive block-space maps over discrete orthogonal simplices
and the simplex-domain kernels they drive, on one GB300 (sm_103a).

Paper: Navarro, Bustos, Hitschfeld, "Possibilities of Recursive GPU Mapping
for Discrete Orthogonal Simplices" (arXiv 1610.07394).

This module is a thin ctypes binding of ``include/simplex.h``: the
``simplex_*`` functions take torch CUDA tensors, check dtypes/devices, pass
raw pointers and the current CUDA stream, and turn status codes into
exceptions.  Every step of the computation runs in ``libsimplex.so``; there is
no CPU or PyTorch fallback, and a missing library raises at the first call.

Convenience wrappers allocate outputs and workspace with torch
(``edm_packed``, ``atm_energy``, ``atm_forces``, ``stress_loss``...), and
``ATMEnergy`` / ``StressLoss`` are ``torch.autograd.Function`` s whose
backward passes call the library's adjoint kernels.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsimplex.so")

MAPS = {"lambda": 0, "bbox": 1, "linear": 2, "rb": 3}
PRECS = {"fp32": 0, "bf16x3": 1, "auto": 2}
OPS = {"map2": 0, "map3": 1, "edm": 2, "atm_energy": 3, "atm_forces": 4,
       "stress_fwd": 5, "stress_bwd": 6, "stress_fwd_bwd": 7}

# Every symbol the header declares (the tests check the library exports them).
EXPORTS = [
    "simplex_abi_version", "simplex_strerror", "simplex_last_cuda_error", "simplex_block_rho",
    "simplex_grid_blocks", "simplex_map_blocks", "simplex_map_blocks_host", "simplex_map2",
    "simplex_map3", "simplex_map4", "simplex_edm_packed", "simplex_atm_energy", "simplex_atm_forces",
    "simplex_stress_fwd", "simplex_stress_bwd", "simplex_workspace_bytes", "simplex_profile",
    "simplex_profile_read", "simplex_atm_energy_noalloc", "simplex_device_errors",
    "simplex_stress_fwd_bwd", "simplex_edm_tiles", "simplex_edm_tiles_len",
]


class SimplexError(RuntimeError):
    def __init__(self, fn: str, status: int, text: str, cuda: int):
        super().__init__(f"{fn} failed: status {status} ({text})"
                         + (f", cudaError {cuda}" if cuda else ""))
        self.status = status
        self.cuda_error = cuda


_lib = None
_i64, _i32, _f32, _f64, _vp = ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_void_p


def _signatures(L):
    sig = {
        "simplex_abi_version": (_i32, []),
        "simplex_strerror": (ctypes.c_char_p, [_i32]),
        "simplex_last_cuda_error": (_i32, []),
        "simplex_block_rho": (_i32, [_i32, _i64, _i32]),
        "simplex_grid_blocks": (_i64, [_i32, _i64, _i32]),
        "simplex_map_blocks": (_i32, [_i32, _i64, _i32, _vp, _vp]),
        "simplex_map_blocks_host": (_i32, [_i32, _i64, _i32, _vp]),
        "simplex_map2": (_i32, [_i64, _i32, _i32, _vp, _vp, _vp]),
        "simplex_map3": (_i32, [_i64, _i32, _i32, _vp, _vp, _vp]),
        "simplex_map4": (_i32, [_i64, _i32, _i32, _vp, _vp, _vp]),
        "simplex_edm_packed": (_i32, [_i64, _i64, _vp, _vp, _i32, _i32, _vp, _i64, _vp]),
        "simplex_edm_tiles": (_i32, [_i64, _i64, _vp, _vp, _i32, _i32, _vp, _i64, _vp]),
        "simplex_edm_tiles_len": (_i64, [_i64]),
        "simplex_atm_energy": (_i32, [_i64, _i64, _vp, _f32, _f32, _vp, _i32, _vp, _i64, _vp]),
        "simplex_atm_forces": (_i32, [_i64, _i64, _vp, _f32, _f32, _vp, _vp, _i32, _vp, _i64, _vp]),
        "simplex_stress_fwd": (_i32, [_i64, _i64, _vp, _vp, _vp, _vp, _i32, _i32, _vp, _i64, _vp]),
        "simplex_stress_bwd": (_i32, [_i64, _i64, _vp, _vp, _f64, _vp, _i32, _i32, _vp, _i64, _vp]),
        "simplex_stress_fwd_bwd": (_i32, [_i64, _i64, _vp, _vp, _f64, _vp, _vp, _i32, _i32, _vp, _i64, _vp]),
        "simplex_workspace_bytes": (_i64, [_i32, _i64, _i64, _i32, _i32]),
        "simplex_profile": (_i32, [_i32]),
        "simplex_device_errors": (_i32, [_vp]),
        "simplex_atm_energy_noalloc": (_i32, [_i64, _i64, _vp, _f32, _f32, _vp, _i32, _vp]),
        "simplex_profile_read": (_i32, [ctypes.POINTER(_f64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def lib():
    """The loaded libsimplex (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsimplex.so not found at {LIB_PATH}; build it with "
                               "`python -m paper_1610_07394_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        _signatures(L)
        _lib = L
    return _lib


def _check(fn: str, st: int):
    if st != 0:
        L = lib()
        raise SimplexError(fn, st, L.simplex_strerror(st).decode(), L.simplex_last_cuda_error())


def _map(m) -> int:
    return MAPS[m] if isinstance(m, str) else int(m)


def _prec(p) -> int:
    return PRECS[p] if isinstance(p, str) else int(p)


def _stream(stream=None) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _cuda(t: torch.Tensor, dtype, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _ptr_or_null(t, dtype, name):
    return None if t is None else _cuda(t, dtype, name)


# ------------------------------------------------------------ raw C-ABI calls

def simplex_abi_version() -> int:
    return lib().simplex_abi_version()


def simplex_block_rho(op, d: int = 3, prec="fp32") -> int:
    return lib().simplex_block_rho(OPS[op] if isinstance(op, str) else op, d, _prec(prec))


def simplex_grid_blocks(m: int, nb: int, map="lambda") -> int:
    return lib().simplex_grid_blocks(m, nb, _map(map))


def simplex_workspace_bytes(op, n: int, d: int, map="lambda", prec="fp32") -> int:
    return lib().simplex_workspace_bytes(OPS[op] if isinstance(op, str) else op, n, d,
                                         _map(map), _prec(prec))


def simplex_map_blocks(m: int, nb: int, map, out: torch.Tensor, stream=None):
    _check("simplex_map_blocks", lib().simplex_map_blocks(
        m, nb, _map(map), _cuda(out, torch.int32, "out"), _stream(stream)))


def simplex_map_blocks_host(m: int, nb: int, map, out: torch.Tensor):
    if out.is_cuda or out.dtype != torch.int32 or not out.is_contiguous():
        raise TypeError("out must be a contiguous host int32 tensor")
    _check("simplex_map_blocks_host", lib().simplex_map_blocks_host(m, nb, _map(map), out.data_ptr()))


def simplex_map2(n: int, rho: int, map, count: torch.Tensor, idle: torch.Tensor, stream=None):
    _check("simplex_map2", lib().simplex_map2(
        n, rho, _map(map), _cuda(count, torch.int32, "count"), _cuda(idle, torch.int64, "idle"),
        _stream(stream)))


def simplex_map3(n: int, rho: int, map, count: torch.Tensor, idle: torch.Tensor, stream=None):
    _check("simplex_map3", lib().simplex_map3(
        n, rho, _map(map), _cuda(count, torch.int32, "count"), _cuda(idle, torch.int64, "idle"),
        _stream(stream)))


def simplex_map4(n: int, rho: int, map, count: torch.Tensor, idle: torch.Tensor, stream=None):
    _check("simplex_map4", lib().simplex_map4(
        n, rho, _map(map), _cuda(count, torch.int32, "count"), _cuda(idle, torch.int64, "idle"),
        _stream(stream)))


def simplex_edm_packed(x, out, map="lambda", prec="fp32", workspace=None, stream=None):
    n, d = x.shape
    ws = _ptr_or_null(workspace, torch.uint8, "workspace")
    _check("simplex_edm_packed", lib().simplex_edm_packed(
        n, d, _cuda(x, torch.float32, "x"), _cuda(out, torch.float32, "out"), _map(map),
        _prec(prec), ws, 0 if workspace is None else workspace.numel(), _stream(stream)))


def simplex_edm_tiles(x, out, map="lambda", prec="fp32", workspace=None, stream=None):
    n, d = x.shape
    ws = _ptr_or_null(workspace, torch.uint8, "workspace")
    _check("simplex_edm_tiles", lib().simplex_edm_tiles(
        n, d, _cuda(x, torch.float32, "x"), _cuda(out, torch.float32, "out"), _map(map),
        _prec(prec), ws, 0 if workspace is None else workspace.numel(), _stream(stream)))


def simplex_edm_tiles_len(n: int) -> int:
    return lib().simplex_edm_tiles_len(n)


def simplex_atm_energy(x, nu, eps, energy, map="lambda", workspace=None, stream=None):
    n, d = x.shape
    ws = _ptr_or_null(workspace, torch.uint8, "workspace")
    _check("simplex_atm_energy", lib().simplex_atm_energy(
        n, d, _cuda(x, torch.float32, "x"), nu, eps, _cuda(energy, torch.float64, "energy"),
        _map(map), ws, 0 if workspace is None else workspace.numel(), _stream(stream)))


def simplex_atm_energy_noalloc(x, nu, eps, energy, map="lambda", stream=None):
    """simplex_atm_energy with the library's static scratch (no allocation)."""
    n, d = x.shape
    _check("simplex_atm_energy_noalloc", lib().simplex_atm_energy_noalloc(
        n, d, _cuda(x, torch.float32, "x"), nu, eps, _cuda(energy, torch.float64, "energy"),
        _map(map), _stream(stream)))


def simplex_atm_forces(x, nu, eps, energy, forces, map="lambda", workspace=None, stream=None):
    n, d = x.shape
    ws = _ptr_or_null(workspace, torch.uint8, "workspace")
    _check("simplex_atm_forces", lib().simplex_atm_forces(
        n, d, _cuda(x, torch.float32, "x"), nu, eps, _ptr_or_null(energy, torch.float64, "energy"),
        _cuda(forces, torch.float64, "forces"), _map(map), ws,
        0 if workspace is None else workspace.numel(), _stream(stream)))


def simplex_stress_fwd(x, y, d_out, loss, map="lambda", prec="fp32", workspace=None, stream=None):
    n, d = x.shape
    ws = _ptr_or_null(workspace, torch.uint8, "workspace")
    _check("simplex_stress_fwd", lib().simplex_stress_fwd(
        n, d, _cuda(x, torch.float32, "x"), _cuda(y, torch.float32, "y"),
        _ptr_or_null(d_out, torch.float32, "d_out"), _cuda(loss, torch.float64, "loss"),
        _map(map), _prec(prec), ws, 0 if workspace is None else workspace.numel(), _stream(stream)))


def simplex_stress_bwd(x, y, gscale, grad, map="lambda", prec="fp32", workspace=None, stream=None):
    n, d = x.shape
    ws = _ptr_or_null(workspace, torch.uint8, "workspace")
    _check("simplex_stress_bwd", lib().simplex_stress_bwd(
        n, d, _cuda(x, torch.float32, "x"), _cuda(y, torch.float32, "y"), float(gscale),
        _cuda(grad, torch.float32, "grad"), _map(map), _prec(prec), ws,
        0 if workspace is None else workspace.numel(), _stream(stream)))


def simplex_stress_fwd_bwd(x, y, gscale, grad, loss, map="lambda", prec="fp32", workspace=None,
                           stream=None):
    n, d = x.shape
    ws = _ptr_or_null(workspace, torch.uint8, "workspace")
    _check("simplex_stress_fwd_bwd", lib().simplex_stress_fwd_bwd(
        n, d, _cuda(x, torch.float32, "x"), _cuda(y, torch.float32, "y"), float(gscale),
        _cuda(grad, torch.float32, "grad"), _cuda(loss, torch.float64, "loss"), _map(map), _prec(prec),
        ws, 0 if workspace is None else workspace.numel(), _stream(stream)))


def simplex_device_errors(stream=None):
    """Raises if a bounded device-side wait ran out (synchronises the stream)."""
    _check("simplex_device_errors", lib().simplex_device_errors(_stream(stream)))


def simplex_profile(on: bool):
    _check("simplex_profile", lib().simplex_profile(1 if on else 0))


def simplex_profile_read():
    """(summed main-kernel ms, main-kernel launches timed, all kernel launches)."""
    ms, k, a = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    _check("simplex_profile_read", lib().simplex_profile_read(ctypes.byref(ms), ctypes.byref(k),
                                                              ctypes.byref(a)))
    return ms.value, k.value, a.value


# ------------------------------------------------------------ conveniences

def workspace(op, n: int, d: int, map="lambda", prec="fp32", device="cuda") -> torch.Tensor | None:
    """A workspace buffer of the size the library asks for (None if none)."""
    b = simplex_workspace_bytes(op, n, d, map, prec)
    if b < 0:
        raise ValueError("bad arguments for workspace sizing")
    return torch.empty(b, dtype=torch.uint8, device=device) if b else None


def map2(n: int, rho: int = 0, map="lambda"):
    """Coverage of Delta_n^2: (count[n(n+1)/2] int32, idle threads)."""
    count = torch.empty(n * (n + 1) // 2, dtype=torch.int32, device="cuda")
    idle = torch.empty(1, dtype=torch.int64, device="cuda")
    simplex_map2(n, rho, map, count, idle)
    return count, idle


def map3(n: int, rho: int = 0, map="lambda"):
    """Coverage of Delta_n^3: (count[n(n+1)(n+2)/6] int32, idle threads)."""
    count = torch.empty(n * (n + 1) * (n + 2) // 6, dtype=torch.int32, device="cuda")
    idle = torch.empty(1, dtype=torch.int64, device="cuda")
    simplex_map3(n, rho, map, count, idle)
    return count, idle


def map4(n: int, rho: int = 0, map="lambda"):
    """Coverage of Delta_n^4: (count[n(n+1)(n+2)(n+3)/24] int32, idle threads)."""
    count = torch.empty(n * (n + 1) * (n + 2) * (n + 3) // 24, dtype=torch.int32, device="cuda")
    idle = torch.empty(1, dtype=torch.int64, device="cuda")
    simplex_map4(n, rho, map, count, idle)
    return count, idle


def map_blocks(m: int, nb: int, map="lambda", device="cuda") -> torch.Tensor:
    """Decode table of a map: (grid blocks, 2m) int32."""
    g = simplex_grid_blocks(m, nb, map)
    out = torch.empty((g, 2 * m), dtype=torch.int32, device=device)
    if device == "cpu":
        simplex_map_blocks_host(m, nb, map, out)
    else:
        simplex_map_blocks(m, nb, map, out)
    return out


def edm_packed(x: torch.Tensor, map="lambda", prec="fp32") -> torch.Tensor:
    """Packed lower EDM of squared distances, n(n+1)/2 FP32."""
    n, d = x.shape
    out = torch.empty(n * (n + 1) // 2, dtype=torch.float32, device=x.device)
    simplex_edm_packed(x, out, map, prec, workspace("edm", n, d, map, prec))
    return out


def edm_tiles(x: torch.Tensor, map="lambda", prec="fp32") -> torch.Tensor:
    """Tile-packed EDM of squared distances: simplex_edm_tiles_len(n) FP32,
    tile (I, J) of 128 x 128 at floats [s * 16384, (s + 1) * 16384),
    s = I(I+1)/2 + J."""
    n, d = x.shape
    out = torch.empty(simplex_edm_tiles_len(n), dtype=torch.float32, device=x.device)
    simplex_edm_tiles(x, out, map, prec, workspace("edm", n, d, map, prec))
    return out


def atm_energy_raw(x: torch.Tensor, nu=1.0, eps=1e-4, map="lambda") -> torch.Tensor:
    n, d = x.shape
    e = torch.empty((), dtype=torch.float64, device=x.device)
    simplex_atm_energy(x, nu, eps, e, map, workspace("atm_energy", n, d, map))
    return e


def atm_forces(x: torch.Tensor, nu=1.0, eps=1e-4, map="lambda", with_energy=True):
    """(forces n x 3 FP64, energy FP64 or None)."""
    n, d = x.shape
    f = torch.empty((n, 3), dtype=torch.float64, device=x.device)
    e = torch.empty((), dtype=torch.float64, device=x.device) if with_energy else None
    simplex_atm_forces(x, nu, eps, e, f, map, workspace("atm_forces", n, d, map))
    return f, e


class ATMEnergy(torch.autograd.Function):
    """E(x) with backward dE/dx = -F from the adjoint kernel (same map)."""

    @staticmethod
    def forward(ctx, x, nu=1.0, eps=1e-4, map="lambda"):
        ctx.save_for_backward(x)
        ctx.args = (nu, eps, map)
        return atm_energy_raw(x, nu, eps, map)

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        nu, eps, map = ctx.args
        f, _ = atm_forces(x, nu, eps, map, with_energy=False)
        return (-f * g).to(x.dtype), None, None, None


def atm_energy(x: torch.Tensor, nu=1.0, eps=1e-4, map="lambda") -> torch.Tensor:
    return ATMEnergy.apply(x, nu, eps, map)


def stress_fwd(x, y, map="lambda", prec="fp32", store_d=False):
    n, d = x.shape
    loss = torch.empty((), dtype=torch.float64, device=x.device)
    D = torch.empty(n * (n + 1) // 2, dtype=torch.float32, device=x.device) if store_d else None
    simplex_stress_fwd(x, y, D, loss, map, prec, workspace("stress_fwd", n, d, map, prec))
    return loss, D


def stress_bwd(x, y, gscale=1.0, map="lambda", prec="fp32"):
    n, d = x.shape
    grad = torch.empty_like(x)
    simplex_stress_bwd(x, y, gscale, grad, map, prec, workspace("stress_bwd", n, d, map, prec))
    return grad


def stress_fwd_bwd(x, y, gscale=1.0, map="lambda", prec="fp32"):
    """(loss, gradient times gscale) from one pass over the pairs."""
    n, d = x.shape
    loss = torch.empty((), dtype=torch.float64, device=x.device)
    grad = torch.empty_like(x)
    simplex_stress_fwd_bwd(x, y, gscale, grad, loss, map, prec, workspace("stress_fwd_bwd", n, d, map, prec))
    return loss, grad


class StressLoss(torch.autograd.Function):
    """L(x; y) = sum_{i<j} (|x_i-x_j|^2 - |y_i-y_j|^2)^2, backward dL/dx."""

    @staticmethod
    def forward(ctx, x, y, map="lambda", prec="fp32"):
        ctx.save_for_backward(x, y)
        ctx.args = (map, prec)
        loss, _ = stress_fwd(x, y, map, prec)
        return loss

    @staticmethod
    def backward(ctx, g):
        x, y = ctx.saved_tensors
        map, prec = ctx.args
        # the upstream gradient stays on the device: the kernel's scale
        # argument is a host double, so it runs at 1 and g is applied after
        grad = stress_bwd(x, y, 1.0, map, prec)
        return grad.mul_(g.to(grad.dtype)), None, None, None


def stress_loss(x, y, map="lambda", prec="fp32"):
    return StressLoss.apply(x, y, map, prec)
