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


def stress_moments(x, y):
    """Stress loss and its full gradient in FP64 from moment matrices,
    O(n d^2): with S = x + y, Delta = x - y, a_i = S_i . Delta_i, the residual
    r_ij = a_i + a_j - S_i.Delta_j - Delta_i.S_j = U_i . V_j for
    U = [a, 1, S, Delta], V = [1, a, -Delta, -S], so
    L = (1/2) sum_ij (U_i . V_j)^2 = (1/2) <U^T U, V^T V>, and
    dL/dx_i = 4 (x_i sum_j r_ij - sum_j r_ij x_j) with both sums linear in the
    moments.  Pinned against the oracle's pairwise loops in test_oracle.py."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = len(x)
    S, De = x + y, x - y
    a = (S * De).sum(1)
    U = np.hstack([a[:, None], np.ones((n, 1)), S, De])
    V = np.hstack([np.ones((n, 1)), a[:, None], -De, -S])
    L = 0.5 * np.sum((U.T @ U) * (V.T @ V))
    rs = n * a + a.sum() - S @ De.sum(0) - De @ S.sum(0)
    rx = np.outer(a, x.sum(0)) + a @ x - S @ (De.T @ x) - De @ (S.T @ x)
    return L, 4 * (x * rs[:, None] - rx)


def _pool_map(fn, items):
    """Runs fn over items on host threads (the oracle's ctypes calls release
    the GIL, so the FP64 loops run on all host cores)."""
    import concurrent.futures as cf
    import os
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return list(ex.map(fn, items))


def grad_all_threads(oracle, x, nu=1.0, eps=1e-4, slices=256):
    """(energy, gradient) of the oracle over all atoms, as slices of its
    outer loop i with about equal work (the triples of row i number about
    (n - i)^2 / 2) run on host threads; the slices partition both sums."""
    n = len(x)
    w = np.cumsum((n - np.arange(n, dtype=np.float64)) ** 2)
    w /= w[-1]
    cuts = sorted(set([0, n] + [min(n, int(np.searchsorted(w, (s + 1) / slices)) + 1) for s in range(slices - 1)]))
    res = _pool_map(lambda k: oracle.atm_energy_grad_slice(x, cuts[k], cuts[k + 1], nu, eps), range(len(cuts) - 1))
    return sum(r[0] for r in res), sum(r[1] for r in res)


def fd_grad_atoms(oracle, x, atoms, h=1e-4, nu=1.0, eps=1e-4):
    """FP64 central differences (x_a +- h e_t) of the oracle's partial energy
    E_a (the triples holding atom a, O(n^2)), which has the same gradient in
    x_a as the total energy.  Rows follow `atoms`."""
    xd = np.asarray(x, dtype=np.float64)

    def one(task):
        a, t = task
        xp, xm = xd.copy(), xd.copy()
        xp[a, t] += h
        xm[a, t] -= h
        return (oracle.atm_atom_energy(xp, a, nu, eps) - oracle.atm_atom_energy(xm, a, nu, eps)) / (2 * h)

    tasks = [(int(a), t) for a in atoms for t in range(3)]
    return np.array(_pool_map(one, tasks)).reshape(len(atoms), 3)


def grad_atoms_threads(oracle, x, atoms, nu=1.0, eps=1e-4):
    """The oracle's analytic gradient rows of `atoms`, one atom per thread."""
    rows = _pool_map(lambda a: oracle.atm_grad_atoms(x, [int(a)], nu, eps)[0], list(atoms))
    return np.array(rows)
