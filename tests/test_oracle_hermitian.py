"""Pins of the complex Hermitian oracle (oracle/hermitian.py, the k-point /
spin-orbit variant named as future work in Sec. IV): closed form from the
generalised eigen-decomposition of the Hermitian pencil, the reduction to the
real symmetric oracle, Hermiticity and the trace invariant (Eq. Nmu), and the
inertia count against a Hermitian LDL^H (Sylvester's law, Sec. II.C)."""
import numpy as np
import pytest
import scipy.linalg as sla

import nao_synth as ns
from oracle import dense, hermitian, poles


@pytest.fixture(scope="module")
def herm_chain():
    s = ns.make_chain(natoms=16, seed=3)
    H, S = ns.hermitian_from(s, seed=5)
    mu, dE = ns.mu_and_delta_e(s)
    return s, H, S, mu, dE


def _dense(s, vals):
    return dense.dense_from_csc(s.n, s.colptr, s.rowind, vals)


def test_generator_hermitian_and_positive_definite(herm_chain):
    s, H, S, _, _ = herm_chain
    Hd, Sd = _dense(s, H), _dense(s, S)
    assert np.max(np.abs(Hd - Hd.conj().T)) == 0.0
    assert np.max(np.abs(Sd - Sd.conj().T)) == 0.0
    assert np.max(np.abs(H.imag)) > 0.05 and np.max(np.abs(S.imag)) > 1e-3
    assert np.min(np.linalg.eigvalsh(Sd)) > 0.0


@pytest.mark.parametrize("key,idx", [("w_rho", 0), ("w_E", 1), ("w_F", 2)])
def test_hermitian_closed_form(herm_chain, key, idx):
    """Gamma = C f_P(Lambda) C^H with H C = S C Lambda, C^H S C = I, where
    f_P is the scalar rational pole approximation (pinned in test_oracle_pins)."""
    s, H, S, mu, dE = herm_chain
    out = hermitian.density_matrices_hermitian(s.n, s.colptr, s.rowind, H, S, mu, s.beta, 40, dE)
    tab = out[3]
    lam, C = sla.eigh(_dense(s, H), _dense(s, S))
    G = (C * poles.rational_approx(lam, tab, key)[None, :]) @ C.conj().T
    r, c = dense.pattern_coords(s.n, s.colptr, s.rowind)
    ref = G[r, c]
    assert np.max(np.abs(out[idx] - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))


def test_plain_im_formula_fails_for_hermitian_data(herm_chain):
    """The mistake the closed form is there to catch: Im(w G) of the real
    symmetric case (transpose instead of conjugate transpose) is wrong here."""
    s, H, S, mu, dE = herm_chain
    dm = hermitian.density_matrices_hermitian(s.n, s.colptr, s.rowind, H, S, mu, s.beta, 40, dE)[0]
    tab = poles.pole_table(s.beta, dE, 40, mu)
    Hd, Sd = _dense(s, H), _dense(s, S)
    r, c = dense.pattern_coords(s.n, s.colptr, s.rowind)
    wrong = sum(np.imag(tab["w_rho"][l] * dense.shifted_inverse(Hd, Sd, z)[r, c]) for l, z in enumerate(tab["z"]))
    assert np.max(np.abs(wrong - dm)) > 1e-3


def test_reduces_to_real_symmetric_oracle():
    s = ns.make_chain(natoms=16, seed=3)
    mu, dE = ns.mu_and_delta_e(s)
    got = hermitian.density_matrices_hermitian(s.n, s.colptr, s.rowind, s.H.astype(complex), s.S.astype(complex),
                                               mu, s.beta, 40, dE)
    ref = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, 40, dE)
    for q in range(3):
        assert np.max(np.abs(got[q].imag)) <= 1e-12 * max(1.0, np.max(np.abs(ref[q])))
        assert np.max(np.abs(got[q].real - ref[q])) <= 1e-12 * max(1.0, np.max(np.abs(ref[q])))


def test_hermitian_dm_is_hermitian_and_trace_is_electron_count(herm_chain):
    s, H, S, mu, dE = herm_chain
    dm = hermitian.density_matrices_hermitian(s.n, s.colptr, s.rowind, H, S, mu, s.beta, 40, dE)[0]
    D = _dense(s, dm)
    assert np.max(np.abs(D - D.conj().T)) <= 1e-12 * np.max(np.abs(D))
    tr = hermitian.trace_with_s_hermitian(dm, S)
    lam = sla.eigh(_dense(s, H), _dense(s, S), eigvals_only=True)
    n_p = dense.electron_count_poles(lam, s.beta, dE, 40, mu)
    assert abs(tr.imag) <= 1e-10 * abs(n_p)
    assert abs(tr.real - n_p) <= 1e-10 * abs(n_p)


def test_hermitian_inertia_sylvester(herm_chain):
    """#{eig(H, S) < sigma} (dense.inertia_counts on the Hermitian pencil)
    equals the negative inertia of D in H - sigma S = L D L^H (Bunch-Kaufman,
    LAPACK hetrf via scipy.linalg.ldl)."""
    s, H, S, mu, _ = herm_chain
    shifts = mu + np.linspace(-0.5, 0.5, 7)
    counts = dense.inertia_counts(s.n, s.colptr, s.rowind, H, S, shifts)
    Hd, Sd = _dense(s, H), _dense(s, S)
    for sigma, want in zip(shifts, counts):
        _, Dm, _ = sla.ldl(Hd - sigma * Sd, hermitian=True)
        assert int(np.sum(np.linalg.eigvalsh(Dm) < 0)) == want


def test_sampled_columns_match_dense(herm_chain):
    """The sparse-LU column evaluation equals the dense definition."""
    s, H, S, mu, dE = herm_chain
    full = hermitian.density_matrices_hermitian(s.n, s.colptr, s.rowind, H, S, mu, s.beta, 40, dE)
    tab = full[3]
    cols = [0, 7, s.n // 2, s.n - 1]
    got = hermitian.dm_columns_hermitian(s.n, s.colptr, s.rowind, H, S, tab, cols)
    for j in cols:
        lo, hi = s.colptr[j], s.colptr[j + 1]
        for q in range(3):
            ref = full[q][lo:hi]
            assert np.max(np.abs(got[j][q] - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))
