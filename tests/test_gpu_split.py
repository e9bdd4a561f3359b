"""Split-precision path (bf16 Ozaki slices on the tcgen05 tensor cores for the
Schur update and the Takahashi GEMM) against the FP64 oracle: max |Delta DM|
<= 1e-7, the stated tolerance of the split path; errors printed per slice
count. Inertia counts through the split real Schur update must equal the
oracle's eigenvalue counts exactly."""
import numpy as np
import pytest

import nao_synth as ns
from oracle import dense

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1405_0194_gb300 as px  # noqa: E402

TOL_SPLIT = 1e-7
TOL_TRACE = 1e-8  # |Tr[DM S] - N_P| for both paths (Eq. Nmu)


@pytest.fixture(scope="module")
def cases():
    from paper_1405_0194_gb300 import build
    build.build()
    out = {}
    for name, s in (("chain64", ns.make_chain()), ("fluid24", ns.make_fluid(nmol=24, seed=1)),
                    ("sheet8", ns.make_sheet(ncell=8, seed=2))):
        mu, dE = ns.mu_and_delta_e(s)
        out[name] = (s, mu, dE)
    return out


@pytest.mark.parametrize("name", ["chain64", "fluid24", "sheet8"])
def test_split_dm_within_tolerance(cases, name):
    s, mu, dE = cases[name]
    P = s.n_poles if name == "chain64" else 16
    dm0, edm0, fdm0, _ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, P, dE)
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(split_slices=6))
    dm, edm, fdm, info = px.pexsi_dm(plan, s.H, s.S, mu, s.beta, P, dE)
    px.pexsi_plan_destroy(plan)
    err = np.max(np.abs(dm - dm0))
    tr0 = dense.trace_with_s(dm0, s.S)
    dtr = abs(info["trace_dm_s"] - tr0)
    print(f"{name}: split(6) max|dDM| = {err:.3e}, |dTr| = {dtr:.3e}")
    assert err <= TOL_SPLIT
    assert dtr <= TOL_TRACE
    assert np.max(np.abs(edm - edm0)) <= TOL_SPLIT * max(1.0, np.max(np.abs(edm0)))
    assert np.max(np.abs(fdm - fdm0)) <= TOL_SPLIT * max(1.0, np.max(np.abs(fdm0)))


@pytest.mark.parametrize("name", ["chain64", "fluid24", "sheet8"])
def test_split_inertia_counts_exact(cases, name):
    """Sylvester's law through the split real LDL^T: counts equal the number of
    generalised eigenvalues below each shift (shifts kept 1e-6 away from every
    eigenvalue, so that the count is well defined at the split path's error)."""
    s, mu, dE = cases[name]
    lam = dense.eig_pencil(s.n, s.colptr, s.rowind, s.H, s.S)[0]
    shifts = []
    for x in mu + np.linspace(-0.6, 0.6, 13):
        while np.min(np.abs(lam - x)) < 1e-6:
            x += 3.7e-6
        shifts.append(x)
    want = np.array([np.count_nonzero(lam < x) for x in shifts])
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(split_slices=6))
    got = px.pexsi_inertia(plan, s.H, s.S, np.array(shifts))
    px.pexsi_plan_destroy(plan)
    np.testing.assert_array_equal(got, want)


def test_split_selinv_error_falls_with_slices(cases):
    s, mu, dE = cases["sheet8"]
    z = mu + 0.13 + 0.002j
    ref = dense.selected_inverse(s.n, s.colptr, s.rowind, s.H, s.S, z)
    errs = []
    for slices in (2, 3, 4, 5, 6):
        plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(split_slices=slices))
        got = px.pexsi_selinv(plan, s.H, s.S, z)
        px.pexsi_plan_destroy(plan)
        errs.append(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        print(f"sheet8 selinv split({slices}) max rel err {errs[-1]:.3e}")
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[-1] <= 1e-7


def test_split_matches_fp64_gpu_path_at_full_size():
    """fluid512 (n = 11,776) in the split path's benchmark launch
    configuration (a 20-pole batch): split-precision DM against the FP64 GPU
    path on poles 40-59, which carry the density matrix."""
    s = ns.make_fluid(nmol=512, seed=0)
    mu, dE = ns.mu_and_delta_e(s)
    dH = torch.from_numpy(s.H).cuda(); dS = torch.from_numpy(s.S).cuda()
    outs = []
    for k in (0, 6):
        plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(max_batch=20, split_slices=k))
        out = torch.zeros(3, s.nnz, dtype=torch.float64, device="cuda")
        st = torch.cuda.current_stream().cuda_stream
        info = px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, 60, dE, 40, 60, 0,
                                  out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), st, want_info=True)
        px.pexsi_plan_destroy(plan)
        outs.append((out.cpu().numpy(), info))
    (a, ia), (b, ib) = outs
    err = np.max(np.abs(a[0] - b[0]))
    print(f"fluid512 poles 40-59 split(6) vs FP64: max|dDM| = {err:.3e} ({err / np.max(np.abs(a[0])):.2e} of the "
          f"largest entry), dTr = {abs(ia['trace_dm_s'] - ib['trace_dm_s']):.3e}, "
          f"ms {ia['ms_total']:.0f} -> {ib['ms_total']:.0f}")
    assert err <= TOL_SPLIT
    assert abs(ia["trace_dm_s"] - ib["trace_dm_s"]) <= 2 * TOL_TRACE


def test_split_inertia_matches_fp64_gpu_path_at_full_size():
    """fluid512: the split real LDL^T, whose 5005-wide root supernode runs
    many 4-panel blocks of the blocked Schur update, gives the same inertia
    counts as the FP64 GPU path at shifts around mu (a count can differ only
    if an eigenvalue lies within the split path's error, ~1e-10, of a shift)."""
    s = ns.make_fluid(nmol=512, seed=0)
    mu, _ = ns.mu_and_delta_e(s)
    shifts = mu + np.array([-0.37, -0.11, -0.023, 0.0071, 0.041, 0.29])
    counts = []
    for k in (0, 6):
        plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(max_batch=8, split_slices=k))
        counts.append(px.pexsi_inertia(plan, s.H, s.S, shifts))
        px.pexsi_plan_destroy(plan)
    print(f"fluid512 inertia counts: FP64 {counts[0].tolist()}, split(6) {counts[1].tolist()}")
    assert np.all(np.diff(counts[0]) >= 0)
    np.testing.assert_array_equal(counts[1], counts[0])
