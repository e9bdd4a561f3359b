"""Column-sampled evaluation of the same definitions (oracle side).

For sizes where a dense inverse is too slow, column j of (H - z S)^{-1} is
the solution of (H - z S) x = e_j. A sparse LU factorisation (scipy's
SuperLU, a library primitive used as one step) followed by solves for a
few sampled columns gives the selected elements of those columns exactly,
which is what Sec. II.A says selected inversion returns.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _csc(n, colptr, rowind, vals):
    return sp.csc_matrix((vals, rowind, colptr), shape=(n, n))


def factor_shifted(n, colptr, rowind, H, S, z):
    """Sparse LU of A = H - z S (complex symmetric)."""
    A = _csc(n, colptr, rowind, np.asarray(H, complex) - z * np.asarray(S, float))
    return spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A")


def selected_columns(n, colptr, rowind, H, S, z, cols, lu=None):
    """Selected elements of (H - z S)^{-1} in the given columns.

    Returns a dict col -> complex values at the pattern rows of that column
    (CSC order within the column).
    """
    if lu is None:
        lu = factor_shifted(n, colptr, rowind, H, S, z)
    cols = np.asarray(cols, dtype=np.int64)
    E = np.zeros((n, cols.shape[0]), dtype=complex)
    E[cols, np.arange(cols.shape[0])] = 1.0
    X = lu.solve(E)
    out = {}
    for k, j in enumerate(cols.tolist()):
        rows = rowind[colptr[j]:colptr[j + 1]]
        out[j] = X[rows, k]
    return out


def dm_columns(n, colptr, rowind, H, S, table, cols, poles_idx=None):
    """DM / EDM / FDM restricted to the given columns, pole by pole.

    ``poles_idx`` limits the sum to a subset of the table's poles (the same
    subset must then be used on the other side of a comparison).
    """
    if poles_idx is None:
        poles_idx = range(len(table["z"]))
    acc = {j: [0.0, 0.0, 0.0] for j in np.asarray(cols).tolist()}
    for l in poles_idx:
        sel = selected_columns(n, colptr, rowind, H, S, table["z"][l], cols)
        for j, v in sel.items():
            acc[j][0] = acc[j][0] + np.imag(table["w_rho"][l] * v)
            acc[j][1] = acc[j][1] + np.imag(table["w_E"][l] * v)
            acc[j][2] = acc[j][2] + np.imag(table["w_F"][l] * v)
    return acc


def factor_shifted_dense(n, colptr, rowind, H, S, z):
    """Dense LU with partial pivoting of A = H - z S (scipy's LAPACK getrf,
    a library primitive used as one step); for the near-dense 3D systems where
    a sparse LU fills in completely anyway."""
    import scipy.linalg as sla
    from .dense import dense_from_csc
    A = dense_from_csc(n, colptr, rowind, np.asarray(H, complex))
    A -= z * dense_from_csc(n, colptr, rowind, np.asarray(S, float))
    return sla.lu_factor(A, overwrite_a=True, check_finite=False)


def selected_columns_dense(n, colptr, rowind, H, S, z, cols, lu=None):
    """As selected_columns, with the dense LU of factor_shifted_dense."""
    import scipy.linalg as sla
    if lu is None:
        lu = factor_shifted_dense(n, colptr, rowind, H, S, z)
    cols = np.asarray(cols, dtype=np.int64)
    E = np.zeros((n, cols.shape[0]), dtype=complex)
    E[cols, np.arange(cols.shape[0])] = 1.0
    X = sla.lu_solve(lu, E, check_finite=False)
    return {j: X[rowind[colptr[j]:colptr[j + 1]], k] for k, j in enumerate(cols.tolist())}
