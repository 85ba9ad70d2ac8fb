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
