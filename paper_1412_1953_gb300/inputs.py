"""Seeded synthetic inputs for the 2D driven Schrodinger problem (H - E)u = f.

This module only *evaluates given functions at node coordinates*: the
Temkin-Poet and exponential-model potentials of Sec. 5.2 / Sec. 6 and the
impact-ionisation style source term.  It holds none of the solver's
arithmetic (no stencil, no smoother, no transfer operator, no eigen-solve), so
both the CPU oracle and the CUDA path consume the same arrays from here.

Node coordinates follow exterior complex scaling (Sec. 2.5): the real grid
x_i = i*L/n (i = 0..n) is kept for x_i <= R0 and bent into the complex plane
beyond, z(x) = R0 + (x - R0) e^{i theta}.  Potentials and the source are
evaluated at these complex nodes (analytic continuation, as the paper does for
the incoming wave of Sec. 3.1).

Array layout everywhere: interior nodes only, row-major [j][i] with x (index i)
fastest; v1 has nx-1 entries, v2 has ny-1, v12 and f have (ny-1)*(nx-1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Problem:
    """One driven-Schrodinger problem instance on a uniform ECS grid."""
    nx: int
    ny: int
    Lx: float
    Ly: float
    R0x: float
    R0y: float
    theta: float
    E: float
    v1: np.ndarray      # (nx-1,)  complex128, V1 at interior x nodes
    v2: np.ndarray      # (ny-1,)  complex128, V2 at interior y nodes
    v12: np.ndarray     # (ny-1, nx-1) complex128, V12 at interior nodes
    f: np.ndarray       # (ny-1, nx-1) complex128, right-hand side
    name: str = ""

    @property
    def n_unknowns(self) -> int:
        return (self.nx - 1) * (self.ny - 1)


def node_coordinates(n: int, L: float, R0: float, theta: float):
    """Real parameters x_i = i L / n and their ECS images z_i, i = 0..n."""
    x = np.arange(n + 1, dtype=np.float64) * (L / n)
    z = x.astype(np.complex128)
    bent = x > R0
    z[bent] = R0 + (x[bent] - R0) * np.exp(1j * theta)
    return x, z


def _pairwise_max_coordinate(xx, zx, yy, zy):
    """Complex image of max(x, y): the node coordinate of whichever axis is larger."""
    X, Y = np.meshgrid(xx, yy)            # [j][i]
    ZX, ZY = np.meshgrid(zx, zy)
    return np.where(X >= Y, ZX, ZY)


def noise(shape, amplitude: float, seed: int) -> np.ndarray:
    """Complex Gaussian noise: Re then Im, each i.i.d. N(0, amplitude^2)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return amplitude * (re + 1j * im)


def temkin_poet(n: int, L: float = 30.0, R0: float = 20.0, theta: float = math.pi / 6,
                E: float = 0.5, Z: float = 1.0, noise_amplitude: float = 1e-3,
                seed: int = 0, ny: int | None = None) -> Problem:
    """Temkin-Poet potentials V1 = -Z/x, V2 = -Z/y, V12 = 1/max(x, y) (Sec. 5.2, Sec. 6.2)
    with source f = 2x e^{-x} (1/max(x,y) - 1/y) sin(sqrt(2E) y) + complex noise.

    2x e^{-x} is the normalised hydrogenic ground state, so f is the potential
    (V2 + V12) acting on an incoming wave phi_1(x) sin(k y), the impact-ionisation
    form of Sec. 3.1 with k = sqrt(2E) as the workload fixes it.
    """
    ny = n if ny is None else ny
    x, zx = node_coordinates(n, L, R0, theta)
    y, zy = node_coordinates(ny, L, R0, theta)
    xi, zxi = x[1:-1], zx[1:-1]
    yj, zyj = y[1:-1], zy[1:-1]
    v1 = -Z / zxi
    v2 = -Z / zyj
    zmax = _pairwise_max_coordinate(xi, zxi, yj, zyj)
    v12 = 1.0 / zmax
    ZX, ZY = np.meshgrid(zxi, zyj)
    k = math.sqrt(2.0 * E) if E > 0 else 0.0
    f = 2.0 * ZX * np.exp(-ZX) * (1.0 / zmax - 1.0 / ZY) * np.sin(k * ZY)
    if noise_amplitude:
        f = f + noise(f.shape, noise_amplitude, seed)
    return Problem(n, ny, L, L, R0, R0, theta, E, v1.astype(np.complex128),
                   v2.astype(np.complex128), np.ascontiguousarray(v12, dtype=np.complex128),
                   np.ascontiguousarray(f, dtype=np.complex128), name=f"tp{n}")


def exponential_model(n: int, L: float = 20.0, R0: float = 15.0, theta: float = math.pi / 7,
                      E: float = 1.0, a1: float = 4.5, a12: float = 2.0, b12: float = 0.1,
                      noise_amplitude: float = 0.0, seed: int = 0) -> Problem:
    """Exponential model of Sec. 6.1: V1 = -a1 e^{-x^2}, V2 = -a1 e^{-y^2},
    V12 = a12 e^{-b12 (x+y)^2}, f = e^{-3 (x+y)^2}."""
    x, z = node_coordinates(n, L, R0, theta)
    zi = z[1:-1]
    v1 = -a1 * np.exp(-zi ** 2)
    ZX, ZY = np.meshgrid(zi, zi)
    v12 = a12 * np.exp(-b12 * (ZX + ZY) ** 2)
    f = np.exp(-3.0 * (ZX + ZY) ** 2)
    if noise_amplitude:
        f = f + noise(f.shape, noise_amplitude, seed)
    return Problem(n, n, L, L, R0, R0, theta, E, v1.astype(np.complex128), v1.astype(np.complex128).copy(),
                   np.ascontiguousarray(v12, dtype=np.complex128),
                   np.ascontiguousarray(f, dtype=np.complex128), name=f"exp{n}")


def free_problem(n: int, L: float, R0: float, theta: float, E: float, f: np.ndarray) -> Problem:
    """Zero potentials with a caller-given right-hand side (used by special-case checks)."""
    z0 = np.zeros(n - 1, dtype=np.complex128)
    return Problem(n, n, L, L, R0, R0, theta, E, z0, z0.copy(),
                   np.zeros((n - 1, n - 1), dtype=np.complex128),
                   np.ascontiguousarray(f, dtype=np.complex128), name=f"free{n}")


def tp_charge_derivative(n: int, L: float = 30.0, R0: float = 20.0, theta: float = math.pi / 6,
                         ny: int | None = None) -> np.ndarray:
    """d(V1 + V2)/dZ = -1/x - 1/y at the interior complex nodes, [j][i] (Temkin-Poet)."""
    ny = n if ny is None else ny
    _, zx = node_coordinates(n, L, R0, theta)
    _, zy = node_coordinates(ny, L, R0, theta)
    ZX, ZY = np.meshgrid(zx[1:-1], zy[1:-1])
    return np.ascontiguousarray(-(1.0 / ZX + 1.0 / ZY), dtype=np.complex128)


def gaussian_window(n: int, L: float, cx: float, cy: float, sigma: float, ny: int | None = None) -> np.ndarray:
    """g(x, y) = exp(-((x-cx)^2 + (y-cy)^2) / (2 sigma^2)) at the interior real nodes, [j][i]."""
    ny = n if ny is None else ny
    x = np.arange(1, n) * (L / n)
    y = np.arange(1, ny) * (L / ny)
    X, Y = np.meshgrid(x, y)
    return np.ascontiguousarray(np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * sigma ** 2)), dtype=np.complex128)


BATCH_SIZES = (256, 384, 512, 768, 1024)


def batching_problems(count: int = 64, E_min: float = 0.1, E_max: float = 2.0, size_seed: int = 1,
                      sizes=BATCH_SIZES, theta: float = math.pi / 6) -> list[Problem]:
    """Many-energy workload: E_k evenly spaced in [E_min, E_max]; problem k on its own
    n_k x n_k grid drawn from `sizes` by default_rng(size_seed); L = 30 n / 512 (the same
    spacing h = 30/512 on every grid), ECS beyond R0 = 2L/3; source noise seed k."""
    n_k = np.random.default_rng(size_seed).choice(np.asarray(sizes), size=count)
    E_k = np.linspace(E_min, E_max, count)
    out = []
    for k in range(count):
        n = int(n_k[k])
        L = 30.0 * n / 512
        p = temkin_poet(n, L=L, R0=2.0 * L / 3.0, theta=theta, E=float(E_k[k]), seed=k)
        p.name = f"tp{n}_E{E_k[k]:.4f}"
        out.append(p)
    return out
