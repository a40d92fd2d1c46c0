"""The spatial block A of the all-at-once system (oracle; test infrastructure).

Two operators:

* Neumann finite-volume diffusion, ``A = I + K`` with
  ``(K x)_c = sum over faces f of c of kappa_f (x_c - x_neighbour(f))``.
  No boundary faces (homogeneous Neumann).  This is the SPD implicit-diffusion
  block the all-at-once system (Eq. 1) is built from; K annihilates the
  constant vector, so the smallest eigenvalue of A is exactly 1.
* The paper's test operator, ``A = I - (nu/h^2) L`` with L the 5-point
  Dirichlet Laplacian on the unit square, ``nu = D^2/(2 ell - 4)``,
  ``h = 1/(n_x+1)`` (Eq. 17), with eigenvalues given in Appendix A.

Grid arrays have shape (n2, n1, n0) (x fastest).  Face arrays: kx
(n2, n1, n0-1), ky (n2, n1-1, n0), kz (n2-1, n1, n0).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def fv_apply(x: np.ndarray, kx: np.ndarray, ky: np.ndarray, kz: np.ndarray) -> np.ndarray:
    """y = (I + K) x for a grid array x of shape (n2, n1, n0), real or complex."""
    y = x.copy()
    # x-faces: flux kappa*(x_{i+1} - x_i); cell i gains kappa*(x_i - x_{i+1})
    if kx.size:
        f = kx * (x[:, :, 1:] - x[:, :, :-1])
        y[:, :, :-1] -= f
        y[:, :, 1:] += f
    if ky.size:
        f = ky * (x[:, 1:, :] - x[:, :-1, :])
        y[:, :-1, :] -= f
        y[:, 1:, :] += f
    if kz.size:
        f = kz * (x[1:, :, :] - x[:-1, :, :])
        y[:-1, :, :] -= f
        y[1:, :, :] += f
    return y


def fv_dense(kx: np.ndarray, ky: np.ndarray, kz: np.ndarray, shape) -> np.ndarray:
    """Dense N x N matrix of I + K assembled face by face (small N only)."""
    n2, n1, n0 = shape
    N = n0 * n1 * n2
    A = np.eye(N)

    def idx(k, j, i):
        return i + n0 * (j + n1 * k)

    def add_face(c, d, kap):
        A[c, c] += kap
        A[d, d] += kap
        A[c, d] -= kap
        A[d, c] -= kap

    for k in range(n2):
        for j in range(n1):
            for i in range(n0 - 1):
                add_face(idx(k, j, i), idx(k, j, i + 1), kx[k, j, i])
    for k in range(n2):
        for j in range(n1 - 1):
            for i in range(n0):
                add_face(idx(k, j, i), idx(k, j + 1, i), ky[k, j, i])
    for k in range(n2 - 1):
        for j in range(n1):
            for i in range(n0):
                add_face(idx(k, j, i), idx(k + 1, j, i), kz[k, j, i])
    return A


def fv_sparse(kx, ky, kz, shape) -> sp.csr_matrix:
    """Sparse I + K (same assembly as fv_dense, vectorised over faces)."""
    n2, n1, n0 = shape
    N = n0 * n1 * n2
    c = np.arange(N).reshape(shape)
    rows, cols, vals = [], [], []
    diag = np.ones(N)
    for kap, a, b in ((kx, c[:, :, :-1], c[:, :, 1:]),
                      (ky, c[:, :-1, :], c[:, 1:, :]),
                      (kz, c[:-1, :, :], c[1:, :, :])):
        if kap.size == 0:
            continue
        a = a.ravel(); b = b.ravel(); k = kap.ravel()
        np.add.at(diag, a, k)
        np.add.at(diag, b, k)
        rows += [a, b]; cols += [b, a]; vals += [-k, -k]
    rows.append(np.arange(N)); cols.append(np.arange(N)); vals.append(diag)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


def gershgorin_mu_max(kx, ky, kz, shape) -> float:
    """Upper bound on the largest eigenvalue of I + K: max_c (1 + 2 sum_{f of c} kappa_f).

    Row c of I + K has diagonal 1 + S_c and off-diagonal magnitudes summing to
    S_c, S_c = sum of the face diffusivities of cell c (Gershgorin's theorem).
    """
    S = np.zeros(shape)
    if kx.size:
        S[:, :, :-1] += kx; S[:, :, 1:] += kx
    if ky.size:
        S[:, :-1, :] += ky; S[:, 1:, :] += ky
    if kz.size:
        S[:-1, :, :] += kz; S[1:, :, :] += kz
    return float(1.0 + 2.0 * S.max())


MU_MIN_NEUMANN = 1.0  # K @ ones = 0 and K is PSD, so lambda_min(I + K) = 1 exactly


# --- the paper's operator (Eq. 17) ------------------------------------------

def dirichlet_params(nx: int, ell: int, D: float = 0.2):
    """nu = D^2/(2 ell - 4), h = 1/(n_x + 1) (Section 5, Eq. 17)."""
    return D * D / (2.0 * ell - 4.0), 1.0 / (nx + 1)


def dirichlet_sparse(nx: int, ell: int, D: float = 0.2) -> sp.csr_matrix:
    """A = I - (nu/h^2) L, L the 5-point Dirichlet Laplacian on n_x^2 points (Eq. 17)."""
    nu, h = dirichlet_params(nx, ell, D)
    e = np.ones(nx)
    T = sp.diags([e[:-1], -2.0 * e, e[:-1]], [-1, 0, 1])   # 1D second difference
    I = sp.identity(nx)
    L = sp.kron(I, T) + sp.kron(T, I)
    return (sp.identity(nx * nx) - (nu / (h * h)) * L).tocsr()


def dirichlet_mu_bounds(nx: int, ell: int, D: float = 0.2):
    """mu_min and mu_max of Eq. 17's A, from the closed form of Appendix A."""
    nu, h = dirichlet_params(nx, ell, D)
    c = 8.0 * nu / (h * h)
    mu_min = 1.0 + c * np.sin(np.pi / (2.0 * (nx + 1))) ** 2
    mu_max = 1.0 + c * np.sin(nx * np.pi / (2.0 * (nx + 1))) ** 2
    return mu_min, mu_max
