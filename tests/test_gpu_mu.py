"""Chemical-potential search (Sec. II.C) through the C ABI against the oracle:
the mu found gives Tr[DM S] = N_e within the tolerance, agrees with the root
of the oracle's P-pole electron count, and N'(mu) = Tr[Gamma^d S] matches the
closed form from the eigenvalues."""
import numpy as np
import pytest

import nao_synth as ns
from oracle import dense, poles

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1405_0194_gb300 as px  # noqa: E402


@pytest.fixture(scope="module")
def fluid():
    from paper_1405_0194_gb300 import build
    build.build()
    s = ns.make_fluid(nmol=24, seed=1)
    lam, C = dense.eig_pencil(s.n, s.colptr, s.rowind, s.H, s.S)
    return s, lam


@pytest.mark.parametrize("fill", [0.3, 0.5, 0.71])
def test_mu_search_hits_electron_count(fluid, fill):
    s, lam = fluid
    P = 40
    Ne = 2.0 * round(fill * s.n) + 0.37          # a fractional count: metallic-like filling
    dE = 1.2 * (lam[-1] - lam[0])
    lo, hi = lam[0] - 0.1, lam[-1] + 0.1
    mu_ref = dense.chemical_potential(lam, s.beta, dE, P, Ne, lo, hi)
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind)
    opts = px.pexsi_mu_opts_default(mu_lo=float(np.median(lam)) - 0.3, mu_hi=float(np.median(lam)) + 0.3,
                                    n_electrons=Ne, tol_ne=1e-6)
    dm, edm, fdm, info = px.pexsi_mu_solve(plan, s.H, s.S, s.beta, P, dE, opts)
    px.pexsi_plan_destroy(plan)
    assert info["converged"] == 1
    assert abs(info["n_e"] - Ne) <= 1e-6
    # the oracle's count at the mu found, and the oracle's root
    assert abs(dense.electron_count_poles(lam, s.beta, dE, P, info["mu"]) - Ne) <= 1e-6 + 1e-8
    tab = poles.pole_table(s.beta, dE, P, info["mu"])
    nprime = float(np.sum(poles.rational_approx(lam, tab, "w_d")))
    assert abs(info["dn_dmu"] - nprime) <= 1e-6 * max(1.0, abs(nprime))
    assert abs(info["mu"] - mu_ref) <= 1e-6 / max(nprime, 1e-3) + 1e-9
    assert abs(dense.trace_with_s(dm, s.S) - info["n_e"]) <= 1e-8


def test_mu_search_gap_rule(fluid):
    """An even count with mu inside the gap between two eigenvalues: the
    search settles in that gap and the count matches."""
    s, lam = fluid
    k = int(0.5 * s.n)
    gaps = np.diff(lam)
    k = int(np.argmax(gaps[k - 20:k + 20])) + k - 20 + 1   # a wide gap near half filling
    Ne = 2.0 * k
    dE = 1.2 * (lam[-1] - lam[0])
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind)
    opts = px.pexsi_mu_opts_default(mu_lo=float(lam[0]), mu_hi=float(lam[-1]), n_electrons=Ne, tol_ne=1e-4)
    _, _, _, info = px.pexsi_mu_solve(plan, s.H, s.S, s.beta, 40, dE, opts, want=())
    px.pexsi_plan_destroy(plan)
    assert info["converged"] == 1 and abs(info["n_e"] - Ne) <= 1e-4
    assert lam[k - 1] - 5.0 / s.beta < info["mu"] < lam[k] + 5.0 / s.beta
