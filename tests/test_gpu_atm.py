"""GPU parity of the Axilrod-Teller-Muto energy and forces over the 3-simplex
{i < j < k} against the FP64 oracle.  Energy within 1e-6 relative; forces
(-dE/dx, adjoint kernel) within 1e-4 relative per atom, against the oracle's
analytic gradient and FP64 central differences; properties that hold at any
size (map agreement, force balance, Euler's theorem) at the full sizes."""
import numpy as np
import pytest
import torch

import synth
from helpers import fd_grad_atoms, grad_all_threads, grad_atoms_threads, rel_err, to_gpu

pytestmark = pytest.mark.gpu
E_TOL = 1e-6
F_TOL = 1e-4
# An FP32 side derivative takes about 16 roundings (the table's r^3 and
# edge terms, their products, the cosine terms), and each atom's force sums
# 32 partners per tile and 32 values of k per coefficient in FP32: about
# 16 + 2 sqrt(32) ~ 27 unit roundoffs of kappa for independent roundings.
KAPPA_C = 32


def energy(gpu, x, mp="lambda", nu=1.0, eps=1e-4):
    return gpu.atm_energy_raw(to_gpu(x), nu, eps, mp).item()


def atom_err(F, G):
    """Per-atom |F - (-G)| / |G| for forces F and gradient G."""
    return np.linalg.norm(F + G, axis=1) / np.linalg.norm(G, axis=1)


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear"])
@pytest.mark.parametrize("n", [3, 4, 31, 32, 33, 65, 100, 250])
def test_energy_small(gpu, oracle, mp, n):
    x = synth.uniform_cube(n, 3, 4.0, seed=200 + n)
    assert energy(gpu, x, mp) == pytest.approx(oracle.atm_energy(x), rel=E_TOL)


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear"])
@pytest.mark.parametrize("n", [3, 5, 33, 64, 97])
def test_forces_small(gpu, oracle, mp, n):
    x = synth.uniform_cube(n, 3, 3.0, seed=300 + n)
    F, E = gpu.atm_forces(to_gpu(x), 1.0, 1e-4, mp)
    G = oracle.atm_grad(x)
    assert atom_err(F.cpu().numpy(), G).max() <= F_TOL
    assert E.item() == pytest.approx(oracle.atm_energy(x), rel=E_TOL)


def test_parameters_nu_eps(gpu, oracle):
    x = synth.uniform_cube(70, 3, 2.0, seed=7)
    for nu, eps in ((0.5, 0.0), (2.0, 1e-2)):
        assert energy(gpu, x, "lambda", nu, eps) == pytest.approx(oracle.atm_energy(x, nu, eps), rel=E_TOL)


def near_coincident(n, side, seed, sep, pairs=10):
    """A uniform cloud in which atoms n/2 .. n/2 + pairs - 1 sit at distances
    sep .. 1.9 sep from atoms 0 .. pairs - 1 (seeded directions)."""
    x = synth.uniform_cube(n, 3, side, seed).astype(np.float64)
    d = synth.normal(pairs, 3, seed + 1).astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    h = n // 2
    x[h:h + pairs] = x[:pairs] + sep * d * (1 + np.arange(pairs)[:, None] / pairs)
    return x.astype(np.float32)


U32 = 2.0 ** -24


@pytest.mark.parametrize("mp", ["lambda", "bbox"])
@pytest.mark.parametrize("side,sep,eps", [(6.0, 1e-3, 1e-4), (6.0, 1e-3, 1e-8), (20.0, 3e-3, 1e-4),
                                          (20.0, 1e-2, 1e-4), (6.0, 3e-3, 1e-6)])
def test_near_coincident_pairs(gpu, oracle, mp, side, sep, eps):
    """Pairs 1e-3 .. 1e-2 apart in clouds of several units, the triples
    that dominate E.  Energy against the oracle within 1e-6.  Forces: the
    parts 2 (de/ds)(x_k - x_q) that a third atom k gets from a close pair
    (i, j) are large and nearly opposite, so an FP32 evaluation of the side
    derivatives errs at k by a few FP32 roundings of their magnitudes, not
    of the small net force: every atom's error is checked against
    C U32 kappa_k, kappa_k the oracle's sum of those magnitudes."""
    x = near_coincident(200, side, 40, sep)
    F, E = gpu.atm_forces(to_gpu(x), 1.0, eps, mp)
    G = oracle.atm_grad(x, 1.0, eps)
    kappa = oracle.atm_grad_abs(x, 1.0, eps)
    err = np.linalg.norm(F.cpu().numpy() + G, axis=1)
    e_ref = oracle.atm_energy(x, 1.0, eps)
    print(f"near-coincident {mp} side {side} sep {sep} eps {eps}: force rel max "
          f"{(err / np.linalg.norm(G, axis=1)).max():.2e}, err / (u kappa) max {(err / (U32 * kappa)).max():.2f}, "
          f"energy rel {abs(E.item() / e_ref - 1):.2e}")
    assert (err <= KAPPA_C * U32 * kappa).all()
    assert E.item() == pytest.approx(e_ref, rel=E_TOL)
    assert energy(gpu, x, mp, 1.0, eps) == pytest.approx(e_ref, rel=E_TOL)


def test_closed_form_triangles(gpu):
    """Equilateral (11/(8 L^9) at eps = 0) and collinear (-1/(4 a^9))."""
    L = 1.25
    x = np.array([[0, 0, 0], [L, 0, 0], [L / 2, L * np.sqrt(3) / 2, 0]], np.float32)
    xd = x.astype(np.float64)
    Lr = np.linalg.norm(xd[0] - xd[1])
    assert energy(gpu, x, "lambda", 1.0, 0.0) == pytest.approx(11 / (8 * Lr ** 9), rel=1e-5)
    a = 0.75
    y = np.array([[0, 0, 0], [0, a, 0], [0, 2 * a, 0]], np.float32)
    assert energy(gpu, y, "lambda", 1.0, 0.0) == pytest.approx(-1 / (4 * a ** 9), rel=1e-5)


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear"])
def test_energy_config_n1024(gpu, oracle, mp):
    """3-simplex plain: n = 1024 uniform in a cube of side 10, seed 1,
    178,433,024 triples, nu = 1, eps = 1e-4."""
    x = synth.make_points("atm_n1024")
    assert energy(gpu, x, mp) == pytest.approx(oracle.atm_energy(x), rel=E_TOL)


def test_differentiation_config_n4096(gpu, oracle):
    """n = 4096 in a cube of side 20, seed 3: autograd backward (adjoint
    kernel) on 64 sampled atoms against the oracle's analytic gradient and
    against FP64 central differences (h = 1e-4) of the oracle's partial
    energy, all 64 atoms both ways, max relative error <= 1e-4."""
    x = synth.make_points("atm_n4096")
    xt = to_gpu(x).requires_grad_(True)
    E = gpu.atm_energy(xt)
    E.backward()
    g = xt.grad.double().cpu().numpy()
    atoms = synth.sample_indices(64, 4096, seed=3 + 10 ** 6)
    G = grad_atoms_threads(oracle, x, atoms)
    err = np.linalg.norm(g[atoms] - G, axis=1) / np.linalg.norm(G, axis=1)
    fd = fd_grad_atoms(oracle, x, atoms, h=1e-4)
    err_fd = np.linalg.norm(g[atoms] - fd, axis=1) / np.linalg.norm(fd, axis=1)
    print(f"n=4096 forces, 64 atoms: max rel err {err.max():.3e} (analytic), {err_fd.max():.3e} (FD)")
    assert err.max() <= F_TOL
    assert err_fd.max() <= F_TOL
    # the three maps give the same energy (no oracle run of 1.1e10 triples)
    e = [energy(gpu, x, mp) for mp in ("lambda", "bbox", "linear")]
    assert e[1] == pytest.approx(e[0], rel=1e-9) and e[2] == pytest.approx(e[0], rel=1e-9)


def test_differentiation_config_all_atoms(gpu, oracle):
    """n = 4096 (U[0,20)^3, seed 3): every atom's force against the oracle's
    FP64 gradient (its outer loop split into slices on the host cores), and
    the energy of the same call."""
    w = synth.WORKLOADS["atm_n4096"]
    x = synth.make_points("atm_n4096")
    F, E = gpu.atm_forces(to_gpu(x), 1.0, 1e-4, "lambda")
    e_ref, G = grad_all_threads(oracle, x)
    err = atom_err(F.cpu().numpy(), G)
    print(f"n={w['n']} all atoms: force max {err.max():.2e}, median {np.median(err):.2e}; "
          f"energy {abs(E.item() / e_ref - 1):.2e}")
    assert err.max() <= F_TOL
    assert E.item() == pytest.approx(e_ref, rel=E_TOL)


def test_properties_full_size(gpu):
    """n = 4096: sum of forces ~ 0, total torque ~ 0, and at eps = 0 Euler's
    theorem for the degree -9 homogeneous energy, sum_i x_i . F_i = 9 E.
    With every force within F_TOL relative and E within E_TOL, the identity
    holds to F_TOL sum_i |x_i| |F_i| + 9 E_TOL |E| (the sum cancels: close
    pairs carry large opposite forces at nearly equal x)."""
    x = synth.make_points("atm_n4096")
    F, E = gpu.atm_forces(to_gpu(x), 1.0, 0.0, "lambda")
    F = F.cpu().numpy()
    E = E.item()
    xd = x.astype(np.float64) - x.astype(np.float64).mean(axis=0)
    scale = np.abs(F).sum()
    assert np.abs(F.sum(axis=0)).max() <= 1e-6 * scale
    assert np.abs(np.cross(xd, F).sum(axis=0)).max() <= 1e-6 * scale * 20
    bound = F_TOL * (np.linalg.norm(xd, axis=1) * np.linalg.norm(F, axis=1)).sum() + 9 * E_TOL * abs(E)
    assert abs((xd * F).sum() - 9 * E) <= bound


def test_scale_config_n16384(gpu, oracle):
    """n = 16384 (7.33e11 triples), seed 6: forces on 8 sampled atoms against
    the oracle's analytic gradient and on 4 of them against FP64 central
    differences (h = 1e-4) of the partial energy; energy equal across lambda
    and bounding box."""
    x = synth.make_points("atm_n16384")
    F, E = gpu.atm_forces(to_gpu(x), 1.0, 1e-4, "lambda")
    F = F.cpu().numpy()
    atoms = synth.sample_indices(8, 16384, seed=6 + 10 ** 6)
    G = grad_atoms_threads(oracle, x, atoms)
    err = atom_err(F[atoms], G)
    fd = fd_grad_atoms(oracle, x, atoms[:4], h=1e-4)
    err_fd = atom_err(F[atoms[:4]], fd)
    print(f"n=16384 forces: max rel err {err.max():.3e} (analytic, 8 atoms), {err_fd.max():.3e} (FD, 4 atoms)")
    assert err.max() <= F_TOL
    assert err_fd.max() <= F_TOL
    e_bb = energy(gpu, x, "bbox")
    assert e_bb == pytest.approx(E.item(), rel=1e-6)


def test_forces_per_tile_tables(gpu, oracle):
    """Past 16 GB of force tables (n >= 21,825: 683 blocks of 32) the forces
    kernel builds each tile's tables from the points instead of copying
    them: n = 21,856, forces of 4 seeded atoms against the oracle's analytic
    gradient, and the energy equal across the lambda and linear maps."""
    n = 21856
    nb = -(-n // 32)
    assert nb * (nb + 1) // 2 * 73728 > 16 << 30
    assert gpu.simplex_workspace_bytes("atm_forces", n, 3, "lambda") < 4 << 30   # no tables
    x = synth.uniform_cube(n, 3, 20.0, seed=21)
    F, E = gpu.atm_forces(to_gpu(x), 1.0, 1e-4, "lambda")
    atoms = synth.sample_indices(4, n, seed=22)
    G = grad_atoms_threads(oracle, x, atoms)
    err = atom_err(F.cpu().numpy()[atoms], G)
    print(f"n={n} per-tile force tables: max rel err {err.max():.3e} (4 atoms)")
    assert err.max() <= F_TOL
    _, E_lin = gpu.atm_forces(to_gpu(x), 1.0, 1e-4, "linear", with_energy=True)
    assert E_lin.item() == pytest.approx(E.item(), rel=1e-9)
