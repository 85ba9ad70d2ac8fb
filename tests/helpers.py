"""Independent reference constructions used by the tests (not the oracle, not the product)."""
import numpy as np
import scipy.sparse as sp


def kron_laplacian(nx: int, ny: int) -> sp.csr_matrix:
    """The 5-point Dirichlet Laplacian as the Kronecker sum I (x) T_nx + T_ny (x) I,
    T = tridiag(-1, 2, -1); unknown (i, j) has index j*nx + i."""
    tx = sp.diags([-np.ones(nx - 1), 2 * np.ones(nx), -np.ones(nx - 1)], [-1, 0, 1], format="csr")
    ty = sp.diags([-np.ones(ny - 1), 2 * np.ones(ny), -np.ones(ny - 1)], [-1, 0, 1], format="csr")
    return (sp.kron(sp.identity(ny, format="csr"), tx) + sp.kron(ty, sp.identity(nx, format="csr"))).tocsr()


def interior(a: np.ndarray, nx: int) -> np.ndarray:
    return np.ascontiguousarray(a[:, :nx])


def flat(a: np.ndarray, nx: int) -> np.ndarray:
    return interior(a, nx).reshape(-1)


def unflat(v: np.ndarray, nx: int, ny: int, ld: int = None) -> np.ndarray:
    ld = nx if ld is None else ld
    out = np.zeros((ny, ld), dtype=v.dtype)
    out[:, :nx] = v.reshape(ny, nx)
    return out


def rel_err(a: np.ndarray, b: np.ndarray) -> float:
    """Relative difference of a from b, the larger of the norm-wise
    ||a - b||_2 / ||b||_2 and the element-wise max|a - b| / max|b|: a defect in
    a few points (a halo, a strip edge) that a norm would average away still
    shows in the second."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = a - b
    nb = np.linalg.norm(b)
    mb = np.max(np.abs(b)) if b.size else 0.0
    norm = np.linalg.norm(d) / (nb if nb > 0 else 1.0)
    elem = (np.max(np.abs(d)) if d.size else 0.0) / (mb if mb > 0 else 1.0)
    return float(max(norm, elem))
