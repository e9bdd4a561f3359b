"""GPU parity of the complex Hermitian variant (Sec. IV: k-points, spin-orbit
coupling) through the C ABI: LDU fronts, the two-sided Takahashi recursion
and the Hermitian pole sum (w G - conj(w) G^H) / 2i, against the CPU oracle
(oracle/hermitian.py, pinned on the CPU by tests/test_oracle_hermitian.py).

Tolerances as the FP64 path of the real case: 1e-10 on DM entries (absolute,
entries of order one), Tr[DM S] to 1e-8, inertia counts exact."""
import numpy as np
import pytest
import scipy.linalg as sla

import nao_synth as ns
from oracle import dense, hermitian, poles

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1405_0194_gb300 as px  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module")
def systems():
    from paper_1405_0194_gb300 import build
    build.build()
    out = {}
    for name, s, seed in (("chain37_ragged", ns.make_chain(natoms=37, seed=5, norb=5), 7),
                          ("fluid24", ns.make_fluid(nmol=24, seed=1), 8),
                          ("sheet8", ns.make_sheet(ncell=8, seed=2), 9)):
        H, S = ns.hermitian_from(s, seed=seed)
        mu, dE = ns.mu_and_delta_e(s)
        lam = sla.eigh(dense.dense_from_csc(s.n, s.colptr, s.rowind, H),
                       dense.dense_from_csc(s.n, s.colptr, s.rowind, S), eigvals_only=True)
        # the Hermitian spectrum: widen Delta E so that it covers it around mu
        dE = max(dE, 1.1 * max(lam[-1] - mu, mu - lam[0]))
        out[name] = (s, H, S, mu, dE, lam)
    return out


def _transpose_index(s):
    """CSC index of the transposed entry (c, r) of every entry (r, c)."""
    cols = np.repeat(np.arange(s.n), np.diff(s.colptr))
    key = {(int(r), int(c)): e for e, (r, c) in enumerate(zip(s.rowind, cols))}
    return np.array([key[(int(c), int(r))] for r, c in zip(s.rowind, cols)])


@pytest.mark.parametrize("panel,amalg", [(64, 1), (32, 1), (16, 0), (48, 0)])
def test_selinv_hermitian_matches_dense_inverse(systems, panel, amalg):
    s, H, S, mu, dE, _ = systems["fluid24"]
    z = mu + 0.21 + 0.003j
    Hd = dense.dense_from_csc(s.n, s.colptr, s.rowind, H)
    Sd = dense.dense_from_csc(s.n, s.colptr, s.rowind, S)
    r, c = dense.pattern_coords(s.n, s.colptr, s.rowind)
    ref = np.linalg.inv(Hd - z * Sd)[r, c]
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind,
                          opts=px.pexsi_opts_default(panel=panel, amalgamate=amalg, leaf_cols=40))
    got = px.pexsi_selinv_hermitian(plan, H, S, z)
    px.pexsi_plan_destroy(plan)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    print(f"panel {panel} amalg {amalg}: max rel err {err:.3e}")
    assert err <= 1e-10
    # not complex symmetric: the two triangles differ
    t = _transpose_index(s)
    assert np.max(np.abs(got - got[t])) > 1e-3 * np.max(np.abs(got))


@pytest.mark.parametrize("name", ["chain37_ragged", "fluid24", "sheet8"])
def test_dm_hermitian_matches_oracle(systems, name):
    s, H, S, mu, dE, lam = systems[name]
    P = 20
    dm0, edm0, fdm0, tab = hermitian.density_matrices_hermitian(s.n, s.colptr, s.rowind, H, S, mu, s.beta, P, dE)
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind)
    dm, edm, fdm, info = px.pexsi_dm_hermitian(plan, H, S, mu, s.beta, P, dE)
    px.pexsi_plan_destroy(plan)
    err = np.max(np.abs(dm - dm0))
    tr0 = hermitian.trace_with_s_hermitian(dm0, S)
    print(f"{name}: max|dDM| = {err:.3e}, |dTr| = {abs(info['trace_dm_s'] - tr0.real):.3e}")
    assert err <= TOL
    assert np.max(np.abs(edm - edm0)) <= TOL * max(1.0, np.max(np.abs(edm0)))
    assert np.max(np.abs(fdm - fdm0)) <= TOL * max(1.0, np.max(np.abs(fdm0)))
    assert abs(info["trace_dm_s"] - tr0.real) <= 1e-8
    # Tr[DM S] = N_P(mu) from the Hermitian spectrum (Eq. Nmu)
    assert abs(info["trace_dm_s"] - float(np.sum(poles.rational_approx(lam, tab)))) <= 1e-8
    # Hermitian output
    t = _transpose_index(s)
    assert np.max(np.abs(dm - np.conj(dm[t]))) <= 1e-12 * max(1.0, np.max(np.abs(dm)))


def test_real_input_reduces_to_the_symmetric_path(systems):
    s, _, _, mu, dE, _ = systems["chain37_ragged"]
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind)
    dm_r, edm_r, fdm_r, info_r = px.pexsi_dm(plan, s.H, s.S, mu, s.beta, 16, dE)
    dm_c, edm_c, fdm_c, info_c = px.pexsi_dm_hermitian(plan, s.H.astype(complex), s.S.astype(complex), mu, s.beta,
                                                       16, dE)
    px.pexsi_plan_destroy(plan)
    assert np.max(np.abs(dm_c - dm_r)) <= 1e-12
    assert np.max(np.abs(fdm_c - fdm_r)) <= 1e-12 * max(1.0, np.max(np.abs(fdm_r)))
    assert abs(info_c["trace_dm_s"] - info_r["trace_dm_s"]) <= 1e-10


def test_identity_overlap_and_subranges(systems):
    s, H, _, mu, dE, _ = systems["fluid24"]
    S_id = np.where(s.rowind == np.repeat(np.arange(s.n), np.diff(s.colptr)), 1.0 + 0j, 0.0j)
    P = 12
    Hd = dense.dense_from_csc(s.n, s.colptr, s.rowind, H)
    span = np.linalg.eigvalsh(Hd)
    dE2 = 1.1 * max(span[-1] - mu, mu - span[0])
    dm0, *_ = hermitian.density_matrices_hermitian(s.n, s.colptr, s.rowind, H, S_id, mu, s.beta, P, dE2)
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(max_batch=4))
    dm, *_ = px.pexsi_dm_hermitian(plan, H, None, mu, s.beta, P, dE2, want=("dm",))
    assert np.max(np.abs(dm - dm0)) <= TOL
    # device form over pole subranges, accumulated
    dH = torch.from_numpy(H).cuda()
    out = torch.zeros(3, s.nnz, dtype=torch.complex128, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    for lo, hi, acc in [(0, 5, 0), (5, 9, 1), (9, 12, 1)]:
        px.pexsi_dm_hermitian_device(plan, dH.data_ptr(), 0, mu, s.beta, P, dE2, lo, hi, acc, out[0].data_ptr(),
                                     out[1].data_ptr(), out[2].data_ptr(), st, want_info=(hi == 12))
    torch.cuda.synchronize()
    px.pexsi_plan_destroy(plan)
    assert np.max(np.abs(out[0].cpu().numpy() - dm)) <= 1e-12


@pytest.mark.parametrize("name", ["chain37_ragged", "fluid24", "sheet8"])
def test_inertia_hermitian_exact(systems, name):
    s, H, S, mu, dE, lam = systems[name]
    shifts = []
    for x in mu + np.linspace(-0.8, 0.8, 9):
        while np.min(np.abs(lam - x)) < 1e-7:
            x += 3.3e-7
        shifts.append(x)
    shifts = np.array(shifts)
    want = [int(np.sum(lam < x)) for x in shifts]
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(panel=32))
    got = px.pexsi_inertia_hermitian(plan, H, S, shifts)
    px.pexsi_plan_destroy(plan)
    assert got.tolist() == want
    lo, hi = lam[0] - 1.0, lam[-1] + 1.0
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind)
    ext = px.pexsi_inertia_hermitian(plan, H, S, [lo, hi])
    px.pexsi_plan_destroy(plan)
    assert ext.tolist() == [0, s.n]


def test_dm_hermitian_sampled_columns_fluid64():
    """A larger case (fluid64, n = 1,472) against the column-sampled oracle
    (sparse LU, solves with A and A^T), on the 10 poles of a 40-pole table
    that carry the most weight."""
    s = ns.make_fluid(nmol=64, seed=3)
    H, S = ns.hermitian_from(s, seed=4)
    mu, dE = ns.mu_and_delta_e(s)
    dE *= 1.3
    P = 40
    tab = poles.pole_table(s.beta, dE, P, mu)
    heavy = np.argsort(-np.abs(tab["w_rho"]))[:10]
    lo, hi = int(np.min(heavy)), int(np.max(heavy)) + 1
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind)
    dH = torch.from_numpy(H).cuda(); dS = torch.from_numpy(S).cuda()
    out = torch.zeros(3, s.nnz, dtype=torch.complex128, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    px.pexsi_dm_hermitian_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, lo, hi, 0,
                                 out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), st, want_info=True)
    px.pexsi_plan_destroy(plan)
    got = out.cpu().numpy()
    cols = np.sort(np.random.default_rng(0).choice(s.n, 6, replace=False))
    ref = hermitian.dm_columns_hermitian(s.n, s.colptr, s.rowind, H, S, tab, cols, range(lo, hi))
    worst = 0.0
    for j in cols:
        sl = slice(s.colptr[j], s.colptr[j + 1])
        for q in range(3):
            worst = max(worst, float(np.max(np.abs(got[q, sl] - ref[j][q]))))
    print(f"fluid64 hermitian poles {lo}-{hi - 1}: max sampled |d| = {worst:.3e}")
    assert worst <= TOL * max(1.0, float(np.max(np.abs(got))))
