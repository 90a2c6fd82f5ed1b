"""Small helpers shared by the GPU parity tests."""
import numpy as np
import torch


def rel_err(got, ref, floor=0.0):
    """Elementwise |got - ref| / max(|ref|, floor), in FP64."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref) / np.maximum(np.abs(ref), floor)


def packed_index(i, j):
    """Packed row-major lower index of (i, j), j <= i."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    return i * (i + 1) // 2 + j


def to_gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gather(t: torch.Tensor, idx) -> np.ndarray:
    """t[idx] computed on the device, returned as NumPy."""
    return t[torch.from_numpy(np.asarray(idx, dtype=np.int64)).to(t.device)].cpu().numpy()
