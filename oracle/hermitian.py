"""Complex Hermitian H and S (k-points, spin-orbit coupling: the variant the
paper names as future work, Sec. IV) -- TEST INFRASTRUCTURE ONLY, under the
same rules as the rest of this package.

For Hermitian H and S, (H - conj(z) S)^{-1} = ((H - z S)^{-1})^H, so the pole
pairs z, conj(z) of the expansion (Sec. II.A) fold into the shifts Im z > 0
of the real symmetric case with the conjugate transpose in place of the
transpose. With the folded weights w_l of Eq. gammapole / Eq. gammaF:

    Gamma = sum_l ( w_l G_l - conj(w_l) G_l^H ) / (2 i),   G_l = (H - z_l S)^{-1}

restricted to the pattern. For real symmetric H and S, G_l is complex
symmetric, conj(w G)^T = conj(w G), and the expression reduces to
Im(w_l G_l) of oracle.dense. Gamma is Hermitian; Tr[Gamma S] is real.
"""
from __future__ import annotations

import numpy as np

from . import dense, poles


def density_matrices_hermitian(n, colptr, rowind, H, S, mu, beta, n_poles, delta_e, table=None):
    """DM, EDM, FDM (complex Hermitian, nnz values in CSC order) for complex
    Hermitian H and S on the pattern, and the pole table used."""
    if table is None:
        table = poles.pole_table(beta, delta_e, n_poles, mu)
    Hd = dense.dense_from_csc(n, colptr, rowind, np.asarray(H, dtype=complex))
    Sd = dense.dense_from_csc(n, colptr, rowind, np.asarray(S, dtype=complex))
    r, c = dense.pattern_coords(n, colptr, rowind)
    out = [np.zeros(r.shape[0], dtype=complex) for _ in range(3)]
    for l, z in enumerate(table["z"]):
        G = dense.shifted_inverse(Hd, Sd, z)
        g, gh = G[r, c], np.conj(G[c, r])  # (G)_rc and (G^H)_rc
        for q, key in enumerate(("w_rho", "w_E", "w_F")):
            w = table[key][l]
            out[q] += (w * g - np.conj(w) * gh) / 2j
    return out[0], out[1], out[2], table


def trace_with_s_hermitian(vals, S):
    """Tr[Gamma S] = sum_ij Gamma_ij S_ji = sum_ij Gamma_ij conj(S_ij) for
    Hermitian S on a symmetric pattern; real for Hermitian Gamma."""
    return complex(np.dot(np.asarray(vals, complex), np.conj(np.asarray(S, complex))))


def dm_columns_hermitian(n, colptr, rowind, H, S, table, cols, poles_idx=None):
    """DM / EDM / FDM of the Hermitian variant in the given columns, for sizes
    where a dense inverse is too slow: per pole, a sparse LU of A = H - z S
    (scipy's SuperLU, one library step) gives column j of G = A^{-1} by a
    solve with A and row j of G by a solve with A^T, so that
    Gamma[r, j] = sum_l (w_l G[r, j] - conj(w_l) conj(G[j, r])) / 2i
    at the pattern rows r of column j. Returns {j: (dm, edm, fdm)}, complex."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    if poles_idx is None:
        poles_idx = range(len(table["z"]))
    cols = np.asarray(cols, dtype=np.int64)
    Hc, Sc = np.asarray(H, complex), np.asarray(S, complex)
    E = np.zeros((n, cols.shape[0]), dtype=complex)
    E[cols, np.arange(cols.shape[0])] = 1.0
    acc = {int(j): [0j, 0j, 0j] for j in cols}
    for l in poles_idx:
        z = table["z"][l]
        lu = spla.splu(sp.csc_matrix((Hc - z * Sc, rowind, colptr), shape=(n, n)).tocsc(),
                       permc_spec="MMD_AT_PLUS_A")
        Xc = lu.solve(E)               # columns j of G
        Xr = lu.solve(E, trans="T")    # columns j of G^T = rows j of G
        for k, j in enumerate(cols.tolist()):
            rows = rowind[colptr[j]:colptr[j + 1]]
            g, gh = Xc[rows, k], np.conj(Xr[rows, k])  # G[r, j] and (G^H)[r, j] = conj(G[j, r])
            for q, key in enumerate(("w_rho", "w_E", "w_F")):
                w = table[key][l]
                acc[j][q] = acc[j][q] + (w * g - np.conj(w) * gh) / 2j
    return {j: tuple(v) for j, v in acc.items()}
