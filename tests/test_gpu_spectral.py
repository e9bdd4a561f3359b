"""DOS and LDOS (Sec. II.D) through the C ABI against the oracle."""
import numpy as np
import pytest

import nao_synth as ns
from oracle import dense

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1405_0194_gb300 as px  # noqa: E402


@pytest.fixture(scope="module")
def sheet():
    from paper_1405_0194_gb300 import build
    build.build()
    s = ns.make_sheet(ncell=8, seed=4)
    lam, C = dense.eig_pencil(s.n, s.colptr, s.rowind, s.H, s.S)
    return s, lam, C


def test_cdos_and_dos(sheet):
    s, lam, _ = sheet
    lo, hi = float(lam[0]) - 0.3, float(lam[-1]) + 0.3
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind)
    eps, cdos, dos = px.pexsi_dos(plan, s.H, s.S, lo + 1.234e-4, hi, 41)
    px.pexsi_plan_destroy(plan)
    ref = 2.0 * np.array([np.sum(lam < e) for e in eps])     # Eq. cdos with spin 2
    assert cdos.tolist() == ref.tolist()
    assert cdos[0] == 0 and cdos[-1] == 2 * s.n
    d = np.empty_like(ref)
    d[1:-1] = (ref[2:] - ref[:-2]) / (eps[2:] - eps[:-2])
    d[0] = (ref[1] - ref[0]) / (eps[1] - eps[0])
    d[-1] = (ref[-1] - ref[-2]) / (eps[-1] - eps[-2])
    assert np.max(np.abs(dos - d)) <= 1e-9 * max(1.0, np.max(np.abs(d)))
    # the DOS integrates to 2n (both spins) over the spectrum
    assert abs(np.trapezoid(d, eps) - 2 * s.n) <= 2 * s.n * 0.05


def test_ldos_matrix(sheet):
    s, lam, C = sheet
    e0, eta = float(np.median(lam)) + 0.011, 0.02
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind)
    got = px.pexsi_ldos(plan, s.H, s.S, e0, eta)
    px.pexsi_plan_destroy(plan)
    sel = dense.selected_inverse(s.n, s.colptr, s.rowind, s.H, s.S, e0 + 1j * eta)
    ref = (2.0 / np.pi) * sel.imag
    assert np.max(np.abs(got - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))
    # Tr[L S] is the eta-broadened DOS: (2/pi) sum_i eta / ((lam_i - e)^2 + eta^2)
    lor = (2.0 / np.pi) * np.sum(eta / ((lam - e0) ** 2 + eta ** 2))
    assert abs(dense.trace_with_s(got, s.S) - lor) <= 1e-8 * max(1.0, lor)
