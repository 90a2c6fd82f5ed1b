"""The no-allocation ATM energy entry point.

Some callers cannot allocate device memory: plug-ins that are handed only a
stream and their tensors by a host framework whose caching allocator owns
the GPU's memory, or latency-critical loops that must avoid cudaMalloc and
cudaFree because those can synchronise the device.
``simplex_atm_energy_noalloc`` serves them from a fixed scratch array inside
the library.  These tests call it through the C ABI (ctypes, raw pointers)
and compare it with ``simplex_atm_energy`` (caller-provided workspace) on
two calls in a row, within the 1e-6 relative tolerance of the energy tests.
This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
E_TOL = 1e-6
ESCRATCH = 7


def call_noalloc(L, x, e, mp, nu=1.0, eps=1e-4):
    n, d = x.shape
    return L.simplex_atm_energy_noalloc(n, d, ctypes.c_void_p(x.data_ptr()), nu, eps,
                                        ctypes.c_void_p(e.data_ptr()), mp,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_workspace_entry_twice(gpu):
    L = gpu.lib()
    cases = [(synth.make_points("atm_n1024"), 0), (synth.uniform_cube(333, 3, 5.0, seed=77), 1)]
    for pts, mp in cases:   # two calls in a row, different sizes and maps
        x = torch.from_numpy(pts).cuda()
        got = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        assert call_noalloc(L, x, got, mp) == 0
        ref = gpu.atm_energy_raw(x, 1.0, 1e-4, ["lambda", "bbox", "linear"][mp])
        torch.cuda.synchronize()
        assert got.item() == pytest.approx(ref.item(), rel=E_TOL)


def test_noalloc_rejects_sizes_beyond_its_scratch(gpu):
    L = gpu.lib()
    x = torch.zeros((8192, 3), dtype=torch.float32, device="cuda")
    e = torch.zeros((), dtype=torch.float64, device="cuda")
    assert call_noalloc(L, x, e, 0) == ESCRATCH
    assert L.simplex_strerror(ESCRATCH)
    assert e.item() == 0.0
