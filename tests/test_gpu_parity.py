"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: max |Delta DM| <= 1e-10 for the FP64 path (absolute, on entries of
order one), inertia counts exact, |Tr[DM S]| matching the oracle to 1e-8.
"""
import numpy as np
import pytest

import nao_synth as ns
from oracle import dense, poles, sampled

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1405_0194_gb300 as px  # noqa: E402

TOL_DM = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1405_0194_gb300 import build
    build.build()


def _plan(s, **kw):
    return px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(**kw))


SYSTEMS = {
    "chain64": lambda: ns.make_chain(),                      # the tiny plain-method case, n = 256
    "chain37_ragged": lambda: ns.make_chain(natoms=37, seed=5, norb=5),
    "fluid24": lambda: ns.make_fluid(nmol=24, seed=1),
    "sheet8": lambda: ns.make_sheet(ncell=8, seed=2),
}


@pytest.fixture(scope="module")
def cases():
    out = {}
    for k, f in SYSTEMS.items():
        s = f()
        mu, dE = ns.mu_and_delta_e(s)
        out[k] = (s, mu, dE)
    return out


@pytest.mark.parametrize("name", ["chain64", "chain37_ragged", "fluid24"])
def test_dm_edm_fdm_match_oracle(cases, name):
    s, mu, dE = cases[name]
    P = s.n_poles if name == "chain64" else 20
    dm0, edm0, fdm0, _ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, P, dE)
    plan = _plan(s)
    dm, edm, fdm, info = px.pexsi_dm(plan, s.H, s.S, mu, s.beta, P, dE)
    px.pexsi_plan_destroy(plan)
    assert np.max(np.abs(dm - dm0)) <= TOL_DM
    assert np.max(np.abs(edm - edm0)) <= TOL_DM * max(1.0, np.max(np.abs(edm0)))
    assert np.max(np.abs(fdm - fdm0)) <= TOL_DM * max(1.0, np.max(np.abs(fdm0)))
    assert abs(info["trace_dm_s"] - dense.trace_with_s(dm0, s.S)) <= 1e-8
    assert abs(info["trace_edm_s"] - dense.trace_with_s(edm0, s.S)) <= 1e-8 * max(1, abs(info["trace_edm_s"]))
    assert info["breakdown_front"] == -1 and info["n_poles"] == P


@pytest.mark.parametrize("panel,amalg", [(64, 1), (32, 1), (16, 0), (48, 0)])
def test_selinv_one_shift_matches_dense_inverse(cases, panel, amalg):
    s, mu, dE = cases["fluid24"]
    z = mu + 0.37 + 0.004j
    ref = dense.selected_inverse(s.n, s.colptr, s.rowind, s.H, s.S, z)
    plan = _plan(s, panel=panel, amalgamate=amalg, leaf_cols=40)
    got = px.pexsi_selinv(plan, s.H, s.S, z)
    px.pexsi_plan_destroy(plan)
    assert np.max(np.abs(got - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))


def test_sheet_dm_matches_oracle(cases):
    s, mu, dE = cases["sheet8"]
    P = 10
    tab = poles.pole_table(s.beta, dE, P, mu)
    dm0, edm0, fdm0, _ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, P, dE, table=tab)
    plan = _plan(s)
    dm, edm, fdm, info = px.pexsi_dm(plan, s.H, s.S, mu, s.beta, P, dE)
    px.pexsi_plan_destroy(plan)
    assert np.max(np.abs(dm - dm0)) <= TOL_DM


def test_identity_overlap(cases):
    s, mu, dE = cases["chain37_ragged"]
    S_id = np.where(s.rowind == np.repeat(np.arange(s.n), np.diff(s.colptr)), 1.0, 0.0)
    dm0, *_ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, S_id, mu, s.beta, 16, dE + 2.0)
    plan = _plan(s)
    dm, _, _, info = px.pexsi_dm(plan, s.H, None, mu, s.beta, 16, dE + 2.0, want=("dm",))
    px.pexsi_plan_destroy(plan)
    assert np.max(np.abs(dm - dm0)) <= TOL_DM


def test_pole_subranges_accumulate(cases):
    s, mu, dE = cases["chain37_ragged"]
    plan = _plan(s, max_batch=3)
    dm_full, *_ = px.pexsi_dm(plan, s.H, s.S, mu, s.beta, 20, dE)
    dH = torch.from_numpy(s.H).cuda(); dS = torch.from_numpy(s.S).cuda()
    out = torch.zeros(3, s.nnz, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    for lo, hi, acc in [(0, 7, 0), (7, 13, 1), (13, 20, 1)]:
        px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, 20, dE, lo, hi, acc,
                           out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), st)
    torch.cuda.synchronize()
    px.pexsi_plan_destroy(plan)
    assert np.max(np.abs(out[0].cpu().numpy() - dm_full)) <= 1e-12


def test_deterministic_repeat(cases):
    s, mu, dE = cases["fluid24"]
    plan = _plan(s)
    a, *_ = px.pexsi_dm(plan, s.H, s.S, mu, s.beta, 12, dE)
    b, *_ = px.pexsi_dm(plan, s.H, s.S, mu, s.beta, 12, dE)
    px.pexsi_plan_destroy(plan)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["chain64", "fluid24", "sheet8"])
def test_inertia_counts_exact(cases, name):
    s, mu, dE = cases[name]
    shifts = mu + np.linspace(-0.8, 0.8, 9) + 1.234e-4
    ref = dense.inertia_counts(s.n, s.colptr, s.rowind, s.H, s.S, shifts)
    plan = _plan(s, panel=32)
    got = px.pexsi_inertia(plan, s.H, s.S, shifts)
    px.pexsi_plan_destroy(plan)
    assert got.tolist() == ref.tolist()


def test_inertia_extremes_and_monotone(cases):
    s, mu, dE = cases["chain37_ragged"]
    lo, hi = ns.spectral_interval(s)
    shifts = np.concatenate([[lo - 1.0], np.linspace(lo + 0.01, hi - 0.01, 13), [hi + 1.0]])
    plan = _plan(s)
    got = px.pexsi_inertia(plan, s.H, s.S, shifts)
    px.pexsi_plan_destroy(plan)
    assert got[0] == 0 and got[-1] == s.n
    assert np.all(np.diff(got) >= 0)


def test_tiny_systems():
    # n = 1 and a purely diagonal pattern (every column its own front)
    for n in (1, 7):
        cp = np.arange(n + 1, dtype=np.int64); ri = np.arange(n, dtype=np.int32)
        H = np.linspace(-1, 1, n); S = np.full(n, 1.5)
        plan = px.pexsi_setup(n, cp, ri)
        z = 0.1 + 0.02j
        got = px.pexsi_selinv(plan, H, S, z)
        cnt = px.pexsi_inertia(plan, H, S, [0.05])
        px.pexsi_plan_destroy(plan)
        assert np.max(np.abs(got - 1.0 / (H - z * S))) < 1e-14
        assert cnt[0] == int(np.sum(H / 1.5 < 0.05))


@pytest.fixture(scope="module")
def full_fluid():
    """The benchmark workload at full size (n = 11,776) with its generalised
    eigen-decomposition (one dense sygvd on the host, about a minute)."""
    s = ns.make_fluid(nmol=512, seed=0)
    mu, dE = ns.mu_and_delta_e(s)
    lam, C = dense.eig_pencil(s.n, s.colptr, s.rowind, s.H, s.S)
    return s, mu, dE, lam, C


def _full_size_all_poles(full_fluid, split, tol):
    """All 60 poles of the table, in the launch configuration the benchmark
    times (20-pole batches, each batch its own call), with the 5 inertia
    shifts of a step. Per batch, 8 sampled DM/EDM/FDM columns against the
    eigen closed form (absolute, and relative to the batch's largest entry);
    the 60-pole sum's traces against the closed form, |Tr[DM S] - N_P| <=
    1e-8 (Eq. Nmu); inertia exact. Poles 30-59 carry the density matrix
    (|w^rho| up to ~2, Im z down to ~3e-3 on the occupied side); poles 0-19
    lie on the empty side, where |w^rho| <= 4e-4."""
    s, mu, dE, lam, C = full_fluid
    B, P = 20, 60
    tab = poles.pole_table(s.beta, dE, P, mu)
    plan = _plan(s, max_batch=B, split_slices=split)
    dH = torch.from_numpy(s.H).cuda(); dS = torch.from_numpy(s.S).cuda()
    out = torch.zeros(3, s.nnz, dtype=torch.float64, device="cuda")
    tot = torch.zeros(3, s.nnz, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(0)
    cols = np.sort(rng.choice(s.n, 8, replace=False))
    report = []
    for b0 in range(0, P, B):
        px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, b0, b0 + B, 0,
                           out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), st, want_info=True)
        tot += out
        got = out.cpu().numpy()
        ref = dense.dm_columns_eig(lam, C, s.colptr, s.rowind, tab, cols, range(b0, b0 + B))
        for q, name in enumerate(("dm", "edm", "fdm")):
            err = max(float(np.max(np.abs(got[q, s.colptr[j]:s.colptr[j + 1]] - ref[j][q]))) for j in cols)
            big = max(float(np.max(np.abs(ref[j][q]))) for j in cols)
            report.append((b0, name, err, big))
    shifts = (mu + np.linspace(-0.5, 0.5, 16) + 1.0e-4)[:5]
    cnt = px.pexsi_inertia_device(plan, dH.data_ptr(), dS.data_ptr(), shifts, st)
    full = px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, 0, P, 0,
                              out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), st, want_info=True)
    px.pexsi_plan_destroy(plan)
    for b0, name, err, big in report:
        print(f"fluid512 split={split} poles {b0}-{b0 + B - 1} {name}: max|d| = {err:.3e} "
              f"({err / big:.2e} of the largest sampled entry {big:.3e})")
    tr = dense.trace_eig(lam, tab, range(P))
    dtr = abs(full["trace_dm_s"] - tr[0])
    print(f"fluid512 split={split} 60 poles: Tr[DM S] = {full['trace_dm_s']:.12f}, |dTr| = {dtr:.3e}, "
          f"|dTr[FDM S]| = {abs(full['trace_fdm_s'] - tr[2]):.3e}")
    for b0, name, err, big in report:
        assert err <= tol * max(1.0, big), (b0, name, err)
    # the batched chain and the single 60-pole call agree
    assert float(torch.max(torch.abs(tot - out))) <= tol
    assert abs(full["trace_fdm_s"] - tr[2]) <= 1e-8 * max(1.0, abs(tr[2]))
    assert cnt.tolist() == [int(np.sum(lam < x)) for x in shifts]
    # the trace invariant Tr[DM S] = N_P (Eq. Nmu) to 1e-8 on both paths:
    # 8.5e-13 relative to N = 11,709; the split path's six slices give each
    # product about 2^-43 of its row maximum over 5.7e6 weighted entries
    assert dtr <= 1e-8


@pytest.mark.slow
def test_full_size_fluid_all_poles(full_fluid):
    """The FP64 path (the benchmark's headline path) on all 60 poles: entries
    within 1e-10."""
    _full_size_all_poles(full_fluid, 0, TOL_DM)


@pytest.mark.slow
def test_full_size_fluid_all_poles_split(full_fluid):
    """The split-precision path (S = 6) on all 60 poles: entries within the
    split tolerance 1e-7, |Tr[DM S] - N_P| within 1e-8."""
    _full_size_all_poles(full_fluid, 6, 1e-7)


@pytest.mark.slow
def test_full_size_sheet_two_poles():
    """The 2D sheet at full size (sheet32x32, n = 26,624, 60-pole table): two
    poles of the occupied side (one next to the real axis, one further out),
    FP64 and split paths, against the oracle's dense LU with 4 sampled column
    solves (about two minutes of host LAPACK per pole)."""
    s = ns.make_sheet(ncell=32, seed=0)
    mu, dE = ns.mu_and_delta_e(s)
    P = 60
    tab = poles.pole_table(s.beta, dE, P, mu)
    dH = torch.from_numpy(s.H).cuda(); dS = torch.from_numpy(s.S).cuda()
    st = torch.cuda.current_stream().cuda_stream
    cols = np.sort(np.random.default_rng(5).choice(s.n, 4, replace=False))
    for l in (59, 45):
        ref = {}
        lu = sampled.factor_shifted_dense(s.n, s.colptr, s.rowind, s.H, s.S, tab["z"][l])
        sel = sampled.selected_columns_dense(s.n, s.colptr, s.rowind, s.H, s.S, tab["z"][l], cols, lu=lu)
        del lu
        for j, v in sel.items():
            ref[j] = [np.imag(tab[k][l] * v) for k in ("w_rho", "w_E", "w_F")]
        for split, tol in ((0, TOL_DM), (6, 1e-7)):
            plan = _plan(s, max_batch=1, split_slices=split)
            out = torch.zeros(3, s.nnz, dtype=torch.float64, device="cuda")
            px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, l, l + 1, 0,
                               out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), st, want_info=True)
            px.pexsi_plan_destroy(plan)
            got = out.cpu().numpy()
            worst = max(float(np.max(np.abs(got[q, s.colptr[j]:s.colptr[j + 1]] - ref[j][q])))
                        for j in cols for q in range(3))
            big = max(float(np.max(np.abs(ref[j][0]))) for j in cols)
            print(f"sheet32x32 pole {l} split={split}: max sampled |d| = {worst:.3e} (largest sampled DM entry "
                  f"{big:.3e})")
            assert worst <= tol * max(1.0, big)
