"""Fermi-Dirac pole expansion (oracle side).

The paper (Sec. II.A, Eq. polerho) states that

    f_beta(eps - mu) ~= Im sum_{l=1}^{P} w^rho_l / (eps - (z_l + mu)),

with shifts z_l and weights w_l depending only on beta, Delta E and P, and
(Eq. gammaF) that the energy- and free-energy-density matrices use the
same shifts with other weights. It refers the construction to the pole
expansion of Lin, Lu, Ying and E (2009); the paper itself prints no formula.
This module rebuilds that construction from the mathematics:

1.  f(x) = 2 / (1 + exp(beta x)) (Eq. fermidirac, spin factor 2) is analytic
    except at the Matsubara points x = i pi (2j+1) / beta on the imaginary
    axis, |Im x| >= pi / beta.
2.  xi = x^2 + m with m = (pi/beta)^2 maps those points onto (-inf, 0] and
    the spectrum x in [-dE, dE] onto [m, M], M = dE^2 + m.
3.  The doubly connected region C \\ ((-inf, 0] U [m, M]) is the conformal
    image of a rectangle under xi(t) = sqrt(mM) (1/k + sn t)/(1/k - sn t)
    (Hale, Higham and Trefethen 2008), k = (sqrt(M/m) - 1)/(sqrt(M/m) + 1),
    sn = Jacobi sn with parameter k^2. The line Im t = K'/2, Re t in
    [-K, 3K) maps to a closed contour around [m, M].
4.  Each point xi on that contour has two square roots x = +-sqrt(xi - m);
    together they trace a closed "dumbbell" around [-dE, dE] that passes
    between the Matsubara points +- i pi / beta. The trapezoidal rule in t
    (N points, step 4K/N) applied to (1/2 pi i) \\oint F(x) / (x - eps) dx
    gives 2N simple poles. They come in conjugate pairs; keeping the N with
    Im z > 0 and weight w = 2 i r (r the residue) gives the Im-form above,
    so P = N (even).

Jacobi functions with complex argument are built from scipy's real-argument
``ellipj`` by the addition theorem with Jacobi's imaginary transformation
(Abramowitz and Stegun 16.21.1-16.21.4).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import ellipj, ellipk, ellipkm1


def fermi_dirac(x, beta):
    """f_beta(x) = 2 / (1 + exp(beta x)) (Eq. fermidirac), stable for complex x."""
    x = np.asarray(x, dtype=complex)
    bx = beta * x
    out = np.empty_like(bx)
    pos = bx.real >= 0
    e = np.exp(-bx[pos])
    out[pos] = 2.0 * e / (1.0 + e)
    out[~pos] = 2.0 / (1.0 + np.exp(bx[~pos]))
    return out


def energy_fn(x, beta, mu):
    """(x + mu) f_beta(x): absolute band energy weight for Gamma^E (Eq. gammaF)."""
    return (np.asarray(x, dtype=complex) + mu) * fermi_dirac(x, beta)


def free_energy_fn(x, beta):
    """-(2/beta) ln(1 + exp(-beta x)): grand-potential weight for Gamma^F.

    Tr[Gamma^F S] then equals the grand potential sum_i -(2/beta)
    ln(1 + exp(-beta (eps_i - mu))), which with mu N_e added gives the band
    part of F_tot in Eq. Helmholtzpole. The two-sided form keeps the
    logarithm on its principal branch on both half-planes.
    """
    x = np.asarray(x, dtype=complex)
    bx = beta * x
    out = np.empty_like(bx)
    pos = bx.real >= 0
    out[pos] = np.log1p(np.exp(-bx[pos]))
    out[~pos] = -bx[~pos] + np.log1p(np.exp(bx[~pos]))
    return -(2.0 / beta) * out


def dfermi_dmu(x, beta):
    """d/dmu f_beta(eps - mu) at x = eps - mu: (beta/2) f (2 - f) = -f'(x).

    Weights for this function give Gamma^d, whose trace with S is N'(mu)
    (Sec. II.C, the Newton step on the chemical potential)."""
    f = fermi_dirac(x, beta)
    return 0.5 * beta * f * (2.0 - f)


def jacobi_sncndn(u, m):
    """sn, cn, dn(u | m) for complex u and real parameter 0 < m < 1.

    A&S 16.21.2-16.21.4: with s, c, d = sn, cn, dn(x | m) and s1, c1, d1 =
    sn, cn, dn(y | 1 - m), u = x + i y,
        sn = (s d1 + i c d s1 c1) / den
        cn = (c c1 - i s d s1 d1) / den
        dn = (d c1 d1 - i m s c s1) / den,   den = c1^2 + m s^2 s1^2.
    """
    u = np.asarray(u, dtype=complex)
    s, c, d, _ = ellipj(u.real, m)
    s1, c1, d1, _ = ellipj(u.imag, 1.0 - m)
    den = c1 * c1 + m * s * s * s1 * s1
    sn = (s * d1 + 1j * c * d * s1 * c1) / den
    cn = (c * c1 - 1j * s * d * s1 * d1) / den
    dn = (d * c1 * d1 - 1j * m * s * c * s1) / den
    return sn, cn, dn


def contour_nodes(beta, delta_e, n_poles):
    """Trapezoidal nodes of the contour: x_j (right-lobe root) and c_j.

    Returns (x, c) with the 2N poles of the rational approximation being
    y = +x_j with residue -c_j F(x_j) and y = -x_j with residue +c_j F(-x_j).
    Also returns (k, K, K') for the convergence-rate pin.
    """
    if n_poles < 2 or n_poles % 2:
        raise ValueError("n_poles must be even and >= 2")
    N = n_poles
    m = (math.pi / beta) ** 2
    M = delta_e * delta_e + m
    q = math.sqrt(M / m)
    k = (q - 1.0) / (q + 1.0)
    ksq = k * k
    m1 = 4.0 * q / (q + 1.0) ** 2  # 1 - k^2 without cancellation
    K = float(ellipkm1(m1))  # K(k^2)
    Kp = float(ellipk(m1))  # K'(k^2) = K(1 - k^2)
    h = 4.0 * K / N
    t = -K + 0.5j * Kp + (np.arange(1, N + 1) - 0.5) * h
    sn, cn, dn = jacobi_sncndn(t, ksq)
    root = math.sqrt(m * M)
    xi = root * (1.0 / k + sn) / (1.0 / k - sn)
    dxi_dt = root * (2.0 / k) * cn * dn / (1.0 / k - sn) ** 2
    x = np.sqrt(xi - m)
    # Increasing t runs the xi-contour clockwise (t = -K is the crossing in
    # (0, m), t = 0 lies above the real axis, t = K is the crossing beyond
    # M), so the counter-clockwise Cauchy integral takes a minus sign.
    c = -h * dxi_dt / (4j * math.pi * x)
    return x, c, (k, K, Kp)


def pole_table(beta, delta_e, n_poles, mu=0.0):
    """Shifts and weights for DM, EDM and FDM (Eq. polerho, Eq. gammaF).

    Returns a dict with complex arrays of length n_poles:
      ``z``     -- z_l + mu (the shifts that enter H - (z_l + mu) S), Im > 0,
      ``w_rho`` -- weights for f_beta,
      ``w_E``   -- weights for (x + mu) f_beta(x),
      ``w_F``   -- weights for -(2/beta) ln(1 + exp(-beta x)),
      ``w_d``   -- weights for d f / d mu = (beta/2) f (2 - f),
    such that  F(eps - mu) ~= Im sum_l w_l / (eps - z[l]).
    """
    x, c, _ = contour_nodes(beta, delta_e, n_poles)
    shifts = np.concatenate([x, -x])
    fns = {
        "w_rho": lambda y: fermi_dirac(y, beta),
        "w_E": lambda y: energy_fn(y, beta, mu),
        "w_F": lambda y: free_energy_fn(y, beta),
        "w_d": lambda y: dfermi_dmu(y, beta),
    }
    upper = shifts.imag > 0
    out = {"z": shifts[upper] + mu}
    for name, F in fns.items():
        res = np.concatenate([-c * F(x), c * F(-x)])
        out[name] = 2j * res[upper]
    if out["z"].shape[0] != n_poles:
        raise AssertionError("pole count mismatch")
    return out


def rational_approx(eps, table, which="w_rho"):
    """Scalar f_P(eps) = Im sum_l w_l / (eps - z_l) for real eps (array)."""
    eps = np.asarray(eps, dtype=float)[..., None]
    return np.imag(np.sum(table[which] / (eps - table["z"]), axis=-1))
