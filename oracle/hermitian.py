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
