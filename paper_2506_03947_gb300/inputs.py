"""Seeded synthetic inputs for the all-at-once diffusion system.

This module only draws numbers: grid shapes, lognormal face diffusivities and
right-hand sides.  It holds none of the method's arithmetic, so both the CPU
oracle (tests) and the CUDA path (tests, bench) can be fed from it.

Recipe (stated once, used everywhere):

* RNG: ``numpy.random.default_rng(seed)`` (PCG64).
* Cell ordering: x fastest, ``c = i + n0*(j + n1*k)``; arrays are returned in
  C order with shape ``(n2, n1, n0)`` (1D: ``(1, 1, n0)``).
* Gaussian field ``g``: white N(0,1) per cell, filtered with a Gaussian kernel
  of standard deviation ``Lc/sqrt(2)`` per axis (periodic wrap), so that the
  field's correlation is ``exp(-d^2/(2 Lc^2))``; then standardised to sample
  mean 0 and standard deviation 1.
* Face diffusivity between neighbouring cells L, R:
  ``kappa_f = kappa0 * exp(sigma * (g_L + g_R) / 2)`` with
  ``kappa0 = (L/h)^2 / (2 ell)`` and ``L = 10 h``, i.e. ``kappa0 = 50/ell``.
  ``sigma = 0`` gives the constant-diffusivity case.
* Right-hand side: ``b_1 ~ N(0,1)`` per cell, ``b_2 .. b_ell = 0`` (the
  structure of b in Eq. 1 and Section 5 of the paper).

The paper's own experiments use a 2D Dirichlet finite-difference operator
(Eq. 17); these inputs stand in for the ocean data-assimilation operators that
motivate it (Section 1), which are not available.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np


def kappa0_for(ell: int, length_cells: float = 10.0) -> float:
    """Diffusivity scale (L/h)^2/(2 ell) with L = length_cells * h."""
    return length_cells * length_cells / (2.0 * ell)


def gaussian_field(shape: Tuple[int, int, int], corr: Sequence[float], seed: int) -> np.ndarray:
    """Standardised, Gaussian-correlated random field on a (n2, n1, n0) grid.

    ``corr`` gives the correlation length per axis in (x, y, z) order.
    """
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape)
    # numpy axes are (z, y, x); corr is (x, y, z)
    cx, cy, cz = (list(corr) + [0.0, 0.0, 0.0])[:3]
    sig = [cz / np.sqrt(2.0), cy / np.sqrt(2.0), cx / np.sqrt(2.0)]
    sig = [s if n > 1 else 0.0 for s, n in zip(sig, shape)]
    g = gaussian_filter(w, sigma=sig, mode="wrap")
    g = g - g.mean()
    sd = g.std()
    if sd > 0:
        g = g / sd
    return g


def face_diffusivities(g: np.ndarray, kappa0: float, sigma: float):
    """Face arrays (kx, ky, kz) from a cell field: kappa0*exp(sigma*(gL+gR)/2).

    kx has shape (n2, n1, n0-1), ky (n2, n1-1, n0), kz (n2-1, n1, n0); an axis
    of length 1 gives an empty array.
    """
    kx = kappa0 * np.exp(sigma * 0.5 * (g[:, :, :-1] + g[:, :, 1:]))
    ky = kappa0 * np.exp(sigma * 0.5 * (g[:, :-1, :] + g[:, 1:, :]))
    kz = kappa0 * np.exp(sigma * 0.5 * (g[:-1, :, :] + g[1:, :, :]))
    return (np.ascontiguousarray(kx, dtype=np.float64),
            np.ascontiguousarray(ky, dtype=np.float64),
            np.ascontiguousarray(kz, dtype=np.float64))


def rhs(n_cells: int, ell: int, seed: int) -> np.ndarray:
    """Block right-hand side b of shape (ell, N): b_1 ~ N(0,1), the rest zero."""
    rng = np.random.default_rng(seed)
    b = np.zeros((ell, n_cells), dtype=np.float64)
    b[0] = rng.standard_normal(n_cells)
    return b


@dataclasses.dataclass
class Problem:
    """One all-at-once instance: grid, faces, ell, alpha, inner budget, rhs."""
    name: str
    dim: int
    n: Tuple[int, int, int]           # (n0, n1, n2), x fastest
    ell: int
    alpha: float
    inner_its: int
    kx: np.ndarray
    ky: np.ndarray
    kz: np.ndarray
    b: np.ndarray                     # (ell, N) or (nrhs, ell, N)
    tol: float = 1e-8

    @property
    def N(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def shape(self) -> Tuple[int, int, int]:
        return (self.n[2], self.n[1], self.n[0])


def make_problem(name: str, dim: int, n: Sequence[int], ell: int, alpha: float,
                 inner_its: int, sigma: float, corr: Sequence[float], seed_field: int,
                 seed_b, tol: float = 1e-8, kappa0: Optional[float] = None) -> Problem:
    n3 = tuple(int(v) for v in (list(n) + [1, 1, 1])[:3])
    shape = (n3[2], n3[1], n3[0])
    k0 = kappa0_for(ell) if kappa0 is None else kappa0
    if sigma == 0.0:
        g = np.zeros(shape)
    else:
        g = gaussian_field(shape, corr, seed_field)
    kx, ky, kz = face_diffusivities(g, k0, sigma)
    N = n3[0] * n3[1] * n3[2]
    if isinstance(seed_b, (list, tuple)):
        b = np.stack([rhs(N, ell, s) for s in seed_b])
    else:
        b = rhs(N, ell, seed_b)
    return Problem(name, dim, n3, ell, alpha, inner_its, kx, ky, kz, b, tol)


# ---------------------------------------------------------------------------
# The five workloads (sizes, seeds and budgets fixed here once).
# ---------------------------------------------------------------------------

def config_1d(n: int = 256, ell: int = 10, alpha: float = 1e-2, seed_b: int = 1,
              inner_its: int = 20) -> Problem:
    """1D constant diffusivity, kappa = 50/ell, outer tolerance 1e-10."""
    return make_problem("1d_const_n256", 1, (n,), ell, alpha, inner_its, 0.0, (0.0,),
                        0, seed_b, tol=1e-10)


def config_2d(n: int = 256, ell: int = 10, alpha: float = 1e-2, inner_its: int = 20,
              seed_field: int = 11, seed_b: int = 12, sigma: float = 0.5,
              corr: float = 16.0) -> Problem:
    """2D lognormal diffusivity (sigma 0.5, correlation 16 cells) on n x n."""
    return make_problem(f"2d_lognormal_{n}x{n}", 2, (n, n), ell, alpha, inner_its,
                        sigma, (corr, corr), seed_field, seed_b)


def config_2d_large(inner_its: int = 40, alpha: float = 1e-2) -> Problem:
    """2D 1024 x 1024 (N = 1,048,576), seeds 21/22."""
    return config_2d(n=1024, alpha=alpha, inner_its=inner_its, seed_field=21, seed_b=22)


def config_3d(n: int = 128, nrhs: int = 8, ell: int = 10, alpha: float = 1e-2,
              inner_its: int = 15) -> Problem:
    """3D anisotropic lognormal (sigma 0.7, corr 8/8/4), several right-hand sides."""
    return make_problem(f"3d_lognormal_{n}^3_x{nrhs}rhs", 3, (n, n, n), ell, alpha, inner_its,
                        0.7, (8.0, 8.0, 4.0), 31, [32 + i for i in range(nrhs)])


def batch_specs(count: int = 64, master_seed: int = 42):
    """Draw (n, ell, alpha, sigma) for the batched workload, one per instance."""
    rng = np.random.default_rng(master_seed)
    sizes = [128, 192, 256, 384, 512]
    ells = [6, 8, 10, 12]
    alphas = [1e-1, 1e-2]
    specs = []
    for i in range(count):
        n = int(rng.choice(sizes))
        ell = int(rng.choice(ells))
        alpha = float(rng.choice(alphas))
        sigma = float(rng.uniform(0.2, 1.0))
        specs.append((n, ell, alpha, sigma))
    return specs


def config_batch(count: int = 64, master_seed: int = 42, inner_its: int = 20) -> List[Problem]:
    probs = []
    for i, (n, ell, alpha, sigma) in enumerate(batch_specs(count, master_seed)):
        probs.append(make_problem(f"batch{i}_{n}x{n}_l{ell}", 2, (n, n), ell, alpha,
                                  inner_its, sigma, (16.0, 16.0), 1000 + i, 2000 + i))
    return probs
