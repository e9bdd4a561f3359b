"""Groups of systems (batching across systems and poles; Sec. II.B's
independence of poles and the elimination-tree concurrency of Eq. parent):
the fronts of several systems of uneven size share every launch of the level
schedule. Each system's result must equal the one its own plan gives (same
wave size: bit for bit) and the oracle's (1e-10 FP64, 1e-7 split, traces
1e-8); the schedule tuner must choose a valid schedule and find it again in
its cache file."""
import numpy as np
import pytest

import nao_synth as ns
from oracle import dense, poles, sampled

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1405_0194_gb300 as px  # noqa: E402

SMALL = [("chain37", lambda: ns.make_chain(natoms=37, seed=5, norb=5)),
         ("fluid24", lambda: ns.make_fluid(nmol=24, seed=1)),
         ("sheet8", lambda: ns.make_sheet(ncell=8, seed=2)),
         ("chain64", lambda: ns.make_chain())]


@pytest.fixture(scope="module")
def small():
    from paper_1405_0194_gb300 import build
    build.build()
    out = []
    for name, f in SMALL:
        s = f()
        mu, dE = ns.mu_and_delta_e(s)
        out.append((name, s, mu, dE))
    return out


def _group(systems, **kw):
    plans = [px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(device=-1)) for _, s, _, _ in systems]
    g = px.pexsi_group_create(plans, opts=px.pexsi_opts_default(**kw))
    for p in plans:
        px.pexsi_plan_destroy(p)
    return g


def _device_inputs(systems):
    dH = [torch.from_numpy(s.H).cuda() for _, s, _, _ in systems]
    dS = [torch.from_numpy(s.S).cuda() for _, s, _, _ in systems]
    outs = [torch.zeros(3, s.nnz, dtype=torch.float64, device="cuda") for _, s, _, _ in systems]
    return dH, dS, outs


@pytest.mark.parametrize("split", [0, 6])
def test_group_equals_each_system_alone(small, split):
    P, W = 16, 4
    g = _group(small, max_batch=W, split_slices=split)
    dH, dS, outs = _device_inputs(small)
    st = torch.cuda.current_stream().cuda_stream
    infos = px.pexsi_group_dm_device(g, [h.data_ptr() for h in dH], [x.data_ptr() for x in dS],
                                     [m for _, _, m, _ in small], [s.beta for _, s, _, _ in small], P,
                                     [d for _, _, _, d in small], 0, P, 0, [o[0].data_ptr() for o in outs],
                                     [o[1].data_ptr() for o in outs], [o[2].data_ptr() for o in outs], st,
                                     want_info=True)
    assert px.pexsi_group_get_schedule(g)["wave"] == W
    px.pexsi_group_destroy(g)
    tol = 1e-10 if split == 0 else 1e-7
    for q, (name, s, mu, dE) in enumerate(small):
        got = outs[q].cpu().numpy()
        plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(max_batch=W, split_slices=split))
        alone, e_alone, f_alone, info = px.pexsi_dm(plan, s.H, s.S, mu, s.beta, P, dE)
        px.pexsi_plan_destroy(plan)
        # the same launches' arithmetic per front, the same pole grouping: identical
        assert np.array_equal(got[0], alone), name
        assert np.array_equal(got[2], f_alone), name
        assert infos[q]["trace_dm_s"] == info["trace_dm_s"]
        dm0, edm0, fdm0, _ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, P, dE)
        err = float(np.max(np.abs(got[0] - dm0)))
        print(f"group split={split} {name}: max|dDM| = {err:.3e}, "
              f"|dTr| = {abs(infos[q]['trace_dm_s'] - dense.trace_with_s(dm0, s.S)):.3e}")
        assert err <= tol
        assert np.max(np.abs(got[1] - edm0)) <= tol * max(1.0, np.max(np.abs(edm0)))
        assert abs(infos[q]["trace_dm_s"] - dense.trace_with_s(dm0, s.S)) <= 1e-8


def test_group_host_form_and_identity_overlap(small):
    P = 8
    g = _group(small[:2], max_batch=8)
    H = [s.H for _, s, _, _ in small[:2]]
    dm, edm, fdm, infos = px.pexsi_group_dm(g, H, [None, small[1][1].S], [m for _, _, m, _ in small[:2]],
                                            [s.beta for _, s, _, _ in small[:2]], P,
                                            [d + 2.0 for _, _, _, d in small[:2]])
    px.pexsi_group_destroy(g)
    _, s0, mu0, dE0 = small[0]
    S_id = np.where(s0.rowind == np.repeat(np.arange(s0.n), np.diff(s0.colptr)), 1.0, 0.0)
    ref0, *_ = dense.density_matrices(s0.n, s0.colptr, s0.rowind, s0.H, S_id, mu0, s0.beta, P, dE0 + 2.0)
    _, s1, mu1, dE1 = small[1]
    ref1, *_ = dense.density_matrices(s1.n, s1.colptr, s1.rowind, s1.H, s1.S, mu1, s1.beta, P, dE1 + 2.0)
    assert np.max(np.abs(dm[0] - ref0)) <= 1e-10
    assert np.max(np.abs(dm[1] - ref1)) <= 1e-10


def test_schedule_tuner_and_cache(small, tmp_path):
    P = 16
    g = _group(small, max_batch=8, split_slices=6)
    dH, dS, outs = _device_inputs(small)
    args = ([h.data_ptr() for h in dH], [x.data_ptr() for x in dS], [m for _, _, m, _ in small],
            [s.beta for _, s, _, _ in small], P, [d for _, _, _, d in small])
    cache = tmp_path / "schedules.txt"
    first = px.pexsi_group_tune(g, *args, cache_path=cache)
    assert first["from_cache"] == 0 and first["candidates"] >= 3 and first["ms_per_pole"] > 0
    assert 1 <= first["wave"] <= 8 and first["oz_block"] in (1, 2, 4)
    again = px.pexsi_group_tune(g, *args, cache_path=cache)
    assert again["from_cache"] == 1 and (again["wave"], again["oz_block"]) == (first["wave"], first["oz_block"])
    assert px.pexsi_group_get_schedule(g)["wave"] == first["wave"]
    # the tuned schedule still gives the oracle's result
    st = torch.cuda.current_stream().cuda_stream
    px.pexsi_group_dm_device(g, *args[:5], args[5], 0, P, 0, [o[0].data_ptr() for o in outs],
                             [o[1].data_ptr() for o in outs], [o[2].data_ptr() for o in outs], st, want_info=True)
    with pytest.raises(px.PexsiError):  # beyond the batch capacity
        px.pexsi_group_set_schedule(g, wave=1000, oz_block=4)
    px.pexsi_group_destroy(g)
    _, s, mu, dE = small[2]
    dm0, *_ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, P, dE)
    assert np.max(np.abs(outs[2][0].cpu().numpy() - dm0)) <= 1e-7


# The batched split-precision workload: six systems of uneven size drawn as
# the chain, sheet and bulk recipes, n from 2,000 to 30,000, 64 poles each.
CONFIG3 = [("chain500", lambda: ns.make_chain(natoms=500, seed=21)),
           ("fluid96", lambda: ns.make_fluid(nmol=96, seed=22)),
           ("sheet14", lambda: ns.make_sheet(ncell=14, seed=23)),
           ("fluid384", lambda: ns.make_fluid(nmol=384, seed=24)),
           ("sheet23", lambda: ns.make_sheet(ncell=23, seed=25)),
           ("chain7500", lambda: ns.make_chain(natoms=7500, seed=26))]


def _oracle_columns(s, tab, cols, poles_idx):
    """The oracle's DM / EDM / FDM columns by the cheapest exact route for
    the system: sparse LU (chains, small systems) or dense LU (2D / 3D
    systems above 3,000 columns, where the sparse factor fills in)."""
    if s.n <= 3000 or s.name.startswith("chain"):
        return sampled.dm_columns(s.n, s.colptr, s.rowind, s.H, s.S, tab, cols, poles_idx)
    acc = {int(j): [0.0, 0.0, 0.0] for j in cols}
    for l in poles_idx:
        lu = sampled.factor_shifted_dense(s.n, s.colptr, s.rowind, s.H, s.S, tab["z"][l])
        sel = sampled.selected_columns_dense(s.n, s.colptr, s.rowind, s.H, s.S, tab["z"][l], cols, lu=lu)
        for j, v in sel.items():
            for k, key in enumerate(("w_rho", "w_E", "w_F")):
                acc[j][k] = acc[j][k] + np.imag(tab[key][l] * v)
    return acc


@pytest.mark.slow
def test_batched_split_six_systems_against_the_oracle():
    """The six systems of the batched workload in one group, split
    precision, 64 poles each: the full table once (every system's trace
    finite, no breakdown), then poles 60-63 (occupied side, next to the real
    axis) against the oracle in 4 sampled columns of every system, within
    1e-7; one system also alone, bit-identical."""
    systems = []
    for name, f in CONFIG3:
        s = f()
        mu, dE = ns.mu_and_delta_e(s)
        systems.append((name, s, mu, dE))
    P, lo, hi = 64, 60, 64
    g = _group(systems, split_slices=6, max_batch=16)
    dH, dS, outs = _device_inputs(systems)
    st = torch.cuda.current_stream().cuda_stream
    common = ([h.data_ptr() for h in dH], [x.data_ptr() for x in dS], [m for _, _, m, _ in systems],
              [s.beta for _, s, _, _ in systems], P, [d for _, _, _, d in systems])
    ptrs = ([o[0].data_ptr() for o in outs], [o[1].data_ptr() for o in outs], [o[2].data_ptr() for o in outs])
    full = px.pexsi_group_dm_device(g, *common, 0, P, 0, *ptrs, st, want_info=True)
    for (name, s, _, _), inf in zip(systems, full):
        print(f"config-3 {name} n={s.n}: Tr[DM S] = {inf['trace_dm_s']:.6f} ({inf['ms_total']:.0f} ms for the group)")
        assert np.isfinite(inf["trace_dm_s"]) and inf["breakdown_front"] == -1
    px.pexsi_group_dm_device(g, *common, lo, hi, 0, *ptrs, st, want_info=True)
    wave = px.pexsi_group_get_schedule(g)["wave"]
    px.pexsi_group_destroy(g)
    rng = np.random.default_rng(3)
    for q, (name, s, mu, dE) in enumerate(systems):
        got = outs[q].cpu().numpy()
        tab = poles.pole_table(s.beta, dE, P, mu)
        cols = np.sort(rng.choice(s.n, 4, replace=False))
        ref = _oracle_columns(s, tab, cols, range(lo, hi))
        worst = big = 0.0
        for j in cols:
            sl = slice(s.colptr[j], s.colptr[j + 1])
            for k in range(3):
                worst = max(worst, float(np.max(np.abs(got[k, sl] - ref[j][k]))))
            big = max(big, float(np.max(np.abs(ref[j][0]))))
        print(f"config-3 group (wave {wave}) {name} n={s.n}: poles {lo}-{hi - 1}, max sampled |d| = {worst:.3e} "
              f"(largest sampled DM entry {big:.3e})")
        assert worst <= 1e-7
    name, s, mu, dE = systems[3]
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(max_batch=wave, split_slices=6))
    o = torch.zeros(3, s.nnz, dtype=torch.float64, device="cuda")
    px.pexsi_dm_device(plan, dH[3].data_ptr(), dS[3].data_ptr(), mu, s.beta, P, dE, lo, hi, 0, o[0].data_ptr(),
                       o[1].data_ptr(), o[2].data_ptr(), st, want_info=True)
    px.pexsi_plan_destroy(plan)
    assert torch.equal(o, outs[3])
