"""Dense definitions of what the PEXSI hot path computes (oracle side).

Sec. II.A states that selected inversion returns the selected elements of
(H - z S)^{-1} *exactly* (up to roundoff), as if the full inverse had been
formed and then restricted. So the oracle for the factorisation + selected
inversion + pole sum is that definition written out with a dense inverse:

    Gamma^{rho,E,F} = Im sum_l w^{rho,E,F}_l (H - z_l S)^{-1}  on pattern(H)

(Eq. gammapole, Eq. gammaF; z_l here already includes mu). The inertia
count (Sec. II.C) is, by Sylvester's law of inertia, the number of
generalised eigenvalues of (H, S) below the shift.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import poles


def dense_from_csc(n, colptr, rowind, vals):
    A = np.zeros((n, n), dtype=np.asarray(vals).dtype)
    cols = np.repeat(np.arange(n), np.diff(colptr))
    A[rowind, cols] = vals
    return A


def pattern_coords(n, colptr, rowind):
    """(row, col) of every stored entry, CSC order."""
    return np.asarray(rowind, dtype=np.int64), np.repeat(np.arange(n), np.diff(colptr))


def shifted_inverse(Hd, Sd, z):
    """(H - z S)^{-1} for a complex shift z: the matrix whose selected
    elements one pole of Eq. gammapole needs (complex symmetric, so the
    transpose, not the conjugate, appears)."""
    A = Hd.astype(complex) - z * Sd
    return np.linalg.inv(A)


def selected_inverse(n, colptr, rowind, H, S, z):
    """Selected elements of (H - z S)^{-1} on the pattern, CSC order."""
    Hd = dense_from_csc(n, colptr, rowind, H)
    Sd = dense_from_csc(n, colptr, rowind, S)
    r, c = pattern_coords(n, colptr, rowind)
    return shifted_inverse(Hd, Sd, z)[r, c]


def density_matrices(n, colptr, rowind, H, S, mu, beta, n_poles, delta_e, table=None):
    """DM, EDM, FDM on the pattern (Eq. gammapole and Eq. gammaF).

    Returns (dm, edm, fdm, table) with each matrix as nnz float64 values in
    CSC order, and the pole table used.
    """
    if table is None:
        table = poles.pole_table(beta, delta_e, n_poles, mu)
    Hd = dense_from_csc(n, colptr, rowind, H)
    Sd = dense_from_csc(n, colptr, rowind, S)
    r, c = pattern_coords(n, colptr, rowind)
    dm = np.zeros(r.shape[0]); edm = np.zeros_like(dm); fdm = np.zeros_like(dm)
    for l, z in enumerate(table["z"]):
        sel = shifted_inverse(Hd, Sd, z)[r, c]
        dm += np.imag(table["w_rho"][l] * sel)
        edm += np.imag(table["w_E"][l] * sel)
        fdm += np.imag(table["w_F"][l] * sel)
    return dm, edm, fdm, table


def trace_with_s(vals, S):
    """Tr[Gamma S] = sum_ij Gamma_ij S_ji over the stored pattern (Eq. Nmu).

    Both matrices are symmetric and stored on the same full pattern, so
    the trace of the product is the entrywise dot product.
    """
    return float(np.dot(np.asarray(vals, float), np.asarray(S, float)))


def inertia_counts(n, colptr, rowind, H, S, shifts):
    """#{generalised eigenvalues of (H, S) < sigma} for each shift (Sec. II.C).

    This is N_infinity(sigma) per spin; Sylvester's law says it equals the
    number of negative entries of D in H - sigma S = L D L^T.
    """
    Hd = dense_from_csc(n, colptr, rowind, H)
    Sd = dense_from_csc(n, colptr, rowind, S)
    ev = sla.eigh(Hd, Sd, eigvals_only=True)
    return np.array([int(np.sum(ev < s)) for s in np.atleast_1d(shifts)], dtype=np.int64)


def eig_pencil(n, colptr, rowind, H, S):
    """Generalised eigenpairs H C = S C Lambda with C^T S C = I (LAPACK sygvd
    through scipy, a library primitive)."""
    Hd = dense_from_csc(n, colptr, rowind, H)
    Sd = dense_from_csc(n, colptr, rowind, S)
    return sla.eigh(Hd, Sd, overwrite_a=True, overwrite_b=True, check_finite=False)


def dm_columns_eig(lam, C, colptr, rowind, table, cols, poles_idx):
    """DM / EDM / FDM in the given columns, summed over the poles in
    poles_idx, from the closed form (H - z S)^{-1} = C (Lambda - z)^{-1} C^T.

    Returns {j: (dm_col, edm_col, fdm_col)} at the pattern rows of column j.
    """
    out = {}
    for j in np.asarray(cols).tolist():
        rows = rowind[colptr[j]:colptr[j + 1]]
        Cr = C[rows, :]
        cj = C[j, :]
        acc = [np.zeros(rows.shape[0]) for _ in range(3)]
        for l in poles_idx:
            col = Cr @ (cj / (lam - table["z"][l]))
            for q, key in enumerate(("w_rho", "w_E", "w_F")):
                acc[q] += np.imag(table[key][l] * col)
        out[j] = tuple(acc)
    return out


def trace_eig(lam, table, poles_idx):
    """Tr[Gamma S] for the poles in poles_idx from the eigenvalues:
    sum_i Im sum_l w_l / (lam_i - z_l) (DM, EDM, FDM)."""
    z = table["z"][list(poles_idx)]
    out = []
    for key in ("w_rho", "w_E", "w_F"):
        w = table[key][list(poles_idx)]
        out.append(float(np.sum(np.imag(w[None, :] / (lam[:, None] - z[None, :])))))
    return out


def electron_count_poles(lam, beta, delta_e, n_poles, mu):
    """N_P(mu) = sum_i Im sum_l w_l / (lam_i - z_l): the electron count the
    P-pole expansion at mu gives for generalised eigenvalues lam (Eq. Nmu)."""
    tab = poles.pole_table(beta, delta_e, n_poles, mu)
    return float(np.sum(poles.rational_approx(lam, tab)))


def chemical_potential(lam, beta, delta_e, n_poles, n_e, lo, hi):
    """The mu in [lo, hi] with N_P(mu) = n_e (Sec. II.C), by bisection on the
    non-decreasing N_P (Eq. Nmu)."""
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if electron_count_poles(lam, beta, delta_e, n_poles, mid) < n_e:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
