"""Pins of the CPU oracle against facts that do not come from the oracle.

* Jacobi elliptic functions of complex argument: algebraic identities,
  the derivative sn' = cn dn, and tabulated special values (A&S 16.5).
* Pole expansion (Eq. polerho, Eq. gammaF): the contour integrates the
  constant function to 1 inside and 0 outside; the error against the exact
  Fermi-Dirac, band-energy and grand-potential functions falls at the
  trapezoidal-rule rate exp(-pi K' P / (4K)) of the strip it lives in.
* DM / EDM / FDM (Eq. gammapole, Eq. gammaF): equal to C g_P(Lambda) C^T from
  the generalised eigen-decomposition (H C = S C Lambda, C^T S C = I), and
  to C g(Lambda) C^T with the exact functions within the pole error.
* Tr[Gamma S] = sum_i f_P(eps_i) and N(mu) is non-decreasing (Eq. Nmu).
* Inertia (Sec. II.C): equal to the count from a Bunch-Kaufman LDL^T
  (Sylvester's law), and exact on a pencil with a known spectrum.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.special import ellipk

import nao_synth as ns
from oracle import dense, poles, sampled


# ---------------------------------------------------------------- elliptic
@pytest.mark.parametrize("m", [0.3, 0.9, 1.0 - 1e-3])
def test_jacobi_complex_identities(m):
    rng = np.random.default_rng(1)
    K = ellipk(m); Kp = ellipk(1 - m)
    u = rng.uniform(-2 * K, 2 * K, 50) + 1j * rng.uniform(-0.9 * Kp, 0.9 * Kp, 50)
    sn, cn, dn = poles.jacobi_sncndn(u, m)
    assert np.max(np.abs(sn**2 + cn**2 - 1)) < 1e-11
    assert np.max(np.abs(dn**2 + m * sn**2 - 1)) < 1e-11
    h = 1e-6
    for step in (h, 1j * h):
        d = (poles.jacobi_sncndn(u + step, m)[0] - poles.jacobi_sncndn(u - step, m)[0]) / (2 * step)
        assert np.max(np.abs(d - cn * dn) / (1 + np.abs(cn * dn))) < 1e-6


@pytest.mark.parametrize("m", [0.2, 0.7])
def test_jacobi_special_values(m):
    k = math.sqrt(m)
    K = ellipk(m); Kp = ellipk(1 - m)
    sn, cn, dn = poles.jacobi_sncndn(np.array([K + 0j, 0.5j * Kp]), m)
    # A&S 16.5: sn K = 1, cn K = 0, dn K = k'; sn(iK'/2) = i k^{-1/2},
    # cn(iK'/2) = (1+k)^{1/2} k^{-1/2}, dn(iK'/2) = (1+k)^{1/2}
    assert abs(sn[0] - 1) < 1e-13 and abs(cn[0]) < 1e-13 and abs(dn[0] - math.sqrt(1 - m)) < 1e-13
    assert abs(sn[1] - 1j / math.sqrt(k)) < 1e-12
    assert abs(cn[1] - math.sqrt(1 + k) / math.sqrt(k)) < 1e-12
    assert abs(dn[1] - math.sqrt(1 + k)) < 1e-12


# ---------------------------------------------------------------- poles
def test_contour_encloses_spectrum():
    beta, dE = 1000.0, 2.0
    x, c, _ = poles.contour_nodes(beta, dE, 80)
    def one(e):
        e = np.asarray(e, float)[:, None]
        return np.sum(-c / (e - x) + c / (e + x), axis=1)
    inside = np.linspace(-dE, dE, 2001)
    assert np.max(np.abs(one(inside) - 1)) < 1e-9
    outside = np.array([-50 * dE, -10 * dE, 10 * dE, 50 * dE])
    assert np.max(np.abs(one(outside))) < 1e-9


@pytest.mark.parametrize("beta,dE,mu", [(1000.0, 2.0, 0.1), (2000.0, 5.0, -0.3), (300.0, 1.0, 0.0)])
def test_pole_expansion_converges_at_trapezoid_rate(beta, dE, mu):
    xs = np.linspace(-dE, dE, 8001)
    exact = {
        "w_rho": poles.fermi_dirac(xs, beta).real,
        "w_E": poles.energy_fn(xs, beta, mu).real,
        "w_F": poles.free_energy_fn(xs, beta).real,
        "w_d": poles.dfermi_dmu(xs, beta).real,
    }
    errs = {k: [] for k in exact}
    Ps = [20, 40, 60, 80]
    for P in Ps:
        tab = poles.pole_table(beta, dE, P, mu)
        assert tab["z"].shape == (P,) and np.all(tab["z"].imag > 0)
        for k in exact:
            scale = max(1.0, np.max(np.abs(exact[k])))
            errs[k].append(np.max(np.abs(poles.rational_approx(xs + mu, tab, k) - exact[k])) / scale)
    _, _, (k_, K, Kp) = poles.contour_nodes(beta, dE, 20)
    rate20 = math.exp(-math.pi * Kp * 20 / (4 * K))  # error ratio per 20 poles
    for k in exact:
        e = np.array(errs[k])
        assert np.all(np.diff(np.log(e[e > 1e-13])) < 0)
        for a, b in zip(e[:-1], e[1:]):
            if b > 1e-12 and a < 1e-2:  # asymptotic regime of the trapezoid rule
                assert 0.3 * rate20 < b / a < 3.0 * rate20
    assert errs["w_rho"][-1] < 1e-6


def test_pole_table_real_axis_symmetry():
    """Im sum w/(x - z) with the conjugate poles added back is a real rational
    function: the full 2P-term sum has no imaginary part on the real axis."""
    tab = poles.pole_table(1000.0, 2.0, 40, 0.0)
    xs = np.linspace(-2, 2, 101)[:, None]
    full = np.sum(tab["w_rho"] / (2j * (xs - tab["z"])) + np.conj(tab["w_rho"]) / (-2j * (xs - np.conj(tab["z"]))), axis=1)
    assert np.max(np.abs(full.imag)) < 1e-12
    assert np.max(np.abs(full.real - poles.rational_approx(xs[:, 0], tab))) < 1e-12


# ---------------------------------------------------------------- matrices
def _eig(sys_):
    Hd = dense.dense_from_csc(sys_.n, sys_.colptr, sys_.rowind, sys_.H)
    Sd = dense.dense_from_csc(sys_.n, sys_.colptr, sys_.rowind, sys_.S)
    lam, C = sla.eigh(Hd, Sd)
    return lam, C


@pytest.fixture(scope="module")
def chain():
    s = ns.make_chain(natoms=40, seed=3)
    mu, dE = ns.mu_and_delta_e(s)
    return s, mu, dE, _eig(s)


@pytest.fixture(scope="module")
def small_fluid():
    s = ns.make_fluid(nmol=24, seed=1)
    mu, dE = ns.mu_and_delta_e(s)
    return s, mu, dE, _eig(s)


@pytest.mark.parametrize("which", ["chain", "small_fluid"])
def test_density_matrices_closed_form(which, request):
    s, mu, dE, (lam, C) = request.getfixturevalue(which)
    dm, edm, fdm, tab = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, 40, dE)
    r, c = dense.pattern_coords(s.n, s.colptr, s.rowind)
    for vals, key in ((dm, "w_rho"), (edm, "w_E"), (fdm, "w_F")):
        g = poles.rational_approx(lam, tab, key)
        ref = ((C * g) @ C.T)[r, c]
        assert np.max(np.abs(vals - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))


def test_selected_inverse_closed_form(chain):
    s, mu, dE, (lam, C) = chain
    z = mu + 0.3 + 0.01j
    sel = dense.selected_inverse(s.n, s.colptr, s.rowind, s.H, s.S, z)
    r, c = dense.pattern_coords(s.n, s.colptr, s.rowind)
    ref = ((C / (lam - z)) @ C.T)[r, c]
    assert np.max(np.abs(sel - ref)) < 1e-10 * np.max(np.abs(ref))
    # complex symmetric, not Hermitian: the transpose appears, the conjugate does not
    assert np.max(np.abs(sel.imag)) > 1e-3


def test_dm_pole_error_falls_with_P(chain):
    s, mu, dE, (lam, C) = chain
    r, c = dense.pattern_coords(s.n, s.colptr, s.rowind)
    ref = ((C * poles.fermi_dirac(lam - mu, s.beta).real) @ C.T)[r, c]
    errs = []
    for P in (20, 40, 60):
        dm, *_ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, P, dE)
        errs.append(np.max(np.abs(dm - ref)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5


def test_trace_equals_electron_count(chain):
    s, mu, dE, (lam, C) = chain
    dm, edm, fdm, tab = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, 40, dE)
    assert abs(dense.trace_with_s(dm, s.S) - poles.rational_approx(lam, tab).sum()) < 1e-10
    assert abs(dense.trace_with_s(edm, s.S) - poles.rational_approx(lam, tab, "w_E").sum()) < 1e-9
    assert abs(dense.trace_with_s(fdm, s.S) - poles.rational_approx(lam, tab, "w_F").sum()) < 1e-9
    # and the electron count of the exact Fermi function, within the pole error
    assert abs(dense.trace_with_s(dm, s.S) - poles.fermi_dirac(lam - mu, s.beta).real.sum()) < 1e-2


def test_electron_count_non_decreasing_in_mu(chain):
    s, mu, dE, _ = chain
    Ns = []
    for m_ in np.linspace(mu - 0.5, mu + 0.5, 9):
        dm, *_ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, m_, s.beta, 40, dE + 0.5)
        Ns.append(dense.trace_with_s(dm, s.S))
    assert np.all(np.diff(Ns) >= -1e-8)


def test_inertia_sylvester(chain):
    s, mu, dE, _ = chain
    Hd = dense.dense_from_csc(s.n, s.colptr, s.rowind, s.H)
    Sd = dense.dense_from_csc(s.n, s.colptr, s.rowind, s.S)
    shifts = np.linspace(mu - 1.0, mu + 1.0, 7) + 1e-3
    counts = dense.inertia_counts(s.n, s.colptr, s.rowind, s.H, s.S, shifts)
    for sig, cnt in zip(shifts, counts):
        _, D, _ = sla.ldl(Hd - sig * Sd)
        assert int(np.sum(np.linalg.eigvalsh(D) < 0)) == cnt


def test_inertia_known_spectrum():
    n = 30
    rng = np.random.default_rng(7)
    lam = np.sort(rng.uniform(-3, 3, n))
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Hd = (Q * lam) @ Q.T
    Hd = 0.5 * (Hd + Hd.T)
    Sd = np.eye(n)
    colptr = np.arange(0, n * n + 1, n, dtype=np.int64)
    rowind = np.tile(np.arange(n, dtype=np.int32), n)
    H = Hd.T.ravel(); S = Sd.T.ravel()
    sig = np.array([-4.0, 0.05, 4.0])
    assert dense.inertia_counts(n, colptr, rowind, H, S, sig).tolist() == [0, int(np.sum(lam < 0.05)), n]


def test_sampled_columns_match_dense(small_fluid):
    s, mu, dE, _ = small_fluid
    tab = poles.pole_table(s.beta, dE, 20, mu)
    dm, edm, fdm, _ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, 20, dE, table=tab)
    cols = [0, s.n // 3, s.n - 1]
    acc = sampled.dm_columns(s.n, s.colptr, s.rowind, s.H, s.S, tab, cols)
    for j in cols:
        sl = slice(s.colptr[j], s.colptr[j + 1])
        assert np.max(np.abs(acc[j][0] - dm[sl])) < 1e-11
        assert np.max(np.abs(acc[j][1] - edm[sl])) < 1e-10
        assert np.max(np.abs(acc[j][2] - fdm[sl])) < 1e-10


def test_sampled_dense_lu_matches_dense(small_fluid):
    s, mu, dE, (lam, C) = small_fluid
    z = mu + 0.21 + 0.003j
    cols = [1, s.n // 2, s.n - 2]
    got = sampled.selected_columns_dense(s.n, s.colptr, s.rowind, s.H, s.S, z, cols)
    ref = ((C / (lam - z)) @ C.T)
    for j in cols:
        rows = s.rowind[s.colptr[j]:s.colptr[j + 1]]
        assert np.max(np.abs(got[j] - ref[rows, j])) < 1e-10 * np.max(np.abs(ref))


def test_eig_closed_form_columns_match_definition(small_fluid):
    s, mu, dE, (lam, C) = small_fluid
    tab = poles.pole_table(s.beta, dE, 20, mu)
    dm, edm, fdm, _ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, 20, dE, table=tab)
    lam2, C2 = dense.eig_pencil(s.n, s.colptr, s.rowind, s.H, s.S)
    sub = range(3, 11)
    dm_s, edm_s, fdm_s, _ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, 20, dE,
                                                   table={k: v[3:11] for k, v in tab.items()})
    cols = [0, 7, s.n - 1]
    got = dense.dm_columns_eig(lam2, C2, s.colptr, s.rowind, tab, cols, sub)
    for j in cols:
        sl = slice(s.colptr[j], s.colptr[j + 1])
        assert np.max(np.abs(got[j][0] - dm_s[sl])) < 1e-11
        assert np.max(np.abs(got[j][1] - edm_s[sl])) < 1e-11
        assert np.max(np.abs(got[j][2] - fdm_s[sl])) < 1e-11
    tr = dense.trace_eig(lam2, tab, sub)
    assert abs(tr[0] - dense.trace_with_s(dm_s, s.S)) < 1e-9
    assert abs(tr[2] - dense.trace_with_s(fdm_s, s.S)) < 1e-9


def test_dfermi_is_mu_derivative():
    """w_d targets the mu-derivative of the Fermi function: a central
    difference of f(x - mu) in mu matches (beta/2) f (2 - f)."""
    beta, h = 1000.0, 1e-7
    xs = np.linspace(-0.02, 0.02, 41)
    fd = (poles.fermi_dirac(xs + h, beta).real - poles.fermi_dirac(xs - h, beta).real) / (2 * h)
    assert np.max(np.abs(-fd - poles.dfermi_dmu(xs, beta).real)) < 1e-4 * beta


def test_electron_count_derivative_closed_form(chain):
    """N'(mu) = Tr[Gamma^d S] equals sum_i (beta/2) f (2-f) (eps_i - mu) from
    the eigenvalues, with the P-pole rational function."""
    s, mu, dE, (lam, C) = chain
    tab = poles.pole_table(s.beta, dE, 80, mu)
    r, c = dense.pattern_coords(s.n, s.colptr, s.rowind)
    g = poles.rational_approx(lam, tab, "w_d")
    Gd = ((C * g) @ C.T)[r, c]
    assert abs(dense.trace_with_s(Gd, s.S) - g.sum()) < 1e-8 * max(1.0, abs(g.sum()))
    # and it is the slope of N(mu): compare with a finite difference of the exact count
    N = lambda m: poles.fermi_dirac(lam - m, s.beta).real.sum()
    h = 1e-6
    assert abs(g.sum() - (N(mu + h) - N(mu - h)) / (2 * h)) < 1e-3 * max(1.0, abs(g.sum()))


def test_chemical_potential_single_level_closed_form():
    """One level at eps0 holding n_e electrons (spin included): the Fermi
    function gives mu = eps0 - ln(2/n_e - 1)/beta in closed form (Eq.
    fermidirac, Eq. Nmu). The search converges to it as the pole error
    falls with P, from a bracket placed off-centre on either side (a
    bisection that moves the wrong end ends at a bracket edge)."""
    beta, eps0 = 1000.0, 0.2
    lam = np.array([eps0])
    errs = []
    for ne in (0.5, 1.0, 1.7):
        exact = eps0 - math.log(2.0 / ne - 1.0) / beta
        for P in (40, 60, 80):
            mu = dense.chemical_potential(lam, beta, 1.0, P, ne, -0.5, 0.9)
            errs.append((ne, P, abs(mu - exact)))
        assert abs(dense.chemical_potential(lam, beta, 1.0, 80, ne, exact - 0.01, exact + 0.6) - exact) < 1e-11
        assert abs(dense.chemical_potential(lam, beta, 1.0, 80, ne, exact - 0.6, exact + 0.01) - exact) < 1e-11
    for ne in (0.5, 1.0, 1.7):
        e = [err for (n_, P, err) in errs if n_ == ne]
        assert e[2] < 1e-11 and e[0] >= e[2]


def test_chemical_potential_lands_in_a_gap():
    """Four levels, n_e = 4 (two filled levels with spin): N_P(mu) = 4 holds
    across the whole gap (-0.1, 0.05) to the pole error, so any root found
    must lie in the gap and give N_P(mu) = 4."""
    beta = 1000.0
    lam = np.array([-0.3, -0.1, 0.05, 0.3])
    mu = dense.chemical_potential(lam, beta, 1.0, 60, 4.0, -0.29, 0.29)
    assert -0.1 < mu < 0.05
    assert abs(dense.electron_count_poles(lam, beta, 1.0, 60, mu) - 4.0) < 1e-9
