"""Host-side checks of the library (no GPU needed): exports, pole table,
CSC validation and the symbolic analysis (Sec. II.B steps 1-2)."""
import os
import re

import numpy as np
import pytest

import nao_synth as ns
from oracle import poles

px = pytest.importorskip("paper_1405_0194_gb300")

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "pexsi_gb300.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1405_0194_gb300 import build
    build.build()


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(pexsi_\w+)\s*\(", txt, flags=re.M)))


def test_library_exports_every_declared_symbol():
    from paper_1405_0194_gb300 import capi
    L = capi.lib()
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    bound = {s[0] for s in capi.SIGNATURES}
    assert set(names) <= bound


def test_pole_table_matches_oracle():
    for beta, dE, P, mu in [(1000.0, 2.0, 40, 0.1), (2000.0, 6.0, 60, -0.4), (300.0, 1.5, 20, 0.0)]:
        a = px.pexsi_pole_table(beta, dE, P, mu)
        b = poles.pole_table(beta, dE, P, mu)
        for k in ("z", "w_rho", "w_E", "w_F"):
            assert np.max(np.abs(a[k] - b[k])) < 1e-12 * max(1.0, np.max(np.abs(b[k]))), k


def test_pole_table_rejects_bad_args():
    for args in [(1000.0, 2.0, 39, 0.0), (1000.0, 2.0, 0, 0.0), (-1.0, 2.0, 40, 0.0), (1000.0, 0.0, 40, 0.0)]:
        with pytest.raises(px.PexsiError) as e:
            px.pexsi_pole_table(*args)
        assert e.value.code == -1


def host_opts(**kw):
    return px.pexsi_opts_default(device=-1, **kw)


def test_setup_rejects_bad_patterns():
    # missing diagonal
    with pytest.raises(px.PexsiError) as e:
        px.pexsi_setup(2, [0, 1, 2], [1, 0], opts=host_opts())
    assert e.value.code == -1
    # asymmetric
    with pytest.raises(px.PexsiError) as e:
        px.pexsi_setup(2, [0, 2, 3], [0, 1, 1], opts=host_opts())
    assert e.value.code == -2
    # unsorted rows
    with pytest.raises(px.PexsiError) as e:
        px.pexsi_setup(2, [0, 2, 4], [1, 0, 0, 1], opts=host_opts())
    assert e.value.code == -1
    # bad permutation
    with pytest.raises(px.PexsiError) as e:
        px.pexsi_setup(2, [0, 2, 4], [0, 1, 0, 1], perm=[0, 0], opts=host_opts())
    assert e.value.code == -1


def test_setup_rejects_bad_split_options():
    s = ns.make_chain(natoms=8)
    for split, panel in ((1, 64), (7, 64), (-1, 64), (6, 32), (2, 48)):
        with pytest.raises(px.PexsiError) as e:
            px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(device=-1, split_slices=split,
                                                                                panel=panel))
        assert e.value.code == -1
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(device=-1, split_slices=6))
    px.pexsi_plan_destroy(plan)


def test_host_only_plan_refuses_numeric_calls():
    s = ns.make_chain(natoms=8)
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=host_opts())
    with pytest.raises(px.PexsiError) as e:
        px.pexsi_dm(plan, s.H, s.S, 0.0, 100.0, 10, 2.0)
    assert e.value.code == -1
    px.pexsi_plan_destroy(plan)


def brute_force_fill(n, colptr, rowind, perm):
    """Boolean Gaussian elimination of P A P^T: pattern of L (column lists)."""
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    A = np.zeros((n, n), dtype=bool)
    cols = np.repeat(np.arange(n), np.diff(colptr))
    A[iperm[rowind], iperm[cols]] = True
    for k in range(n):
        nz = np.nonzero(A[k + 1:, k])[0] + k + 1
        if nz.size:
            A[np.ix_(nz, nz)] = True
    return [np.nonzero(A[j + 1:, j])[0] + j + 1 for j in range(n)]


def random_pattern(n, p, seed):
    rng = np.random.default_rng(seed)
    M = rng.random((n, n)) < p
    M = M | M.T
    np.fill_diagonal(M, True)
    colptr = np.concatenate([[0], np.cumsum(M.sum(axis=0))]).astype(np.int64)
    rowind = np.concatenate([np.nonzero(M[:, j])[0] for j in range(n)]).astype(np.int32)
    return colptr, rowind


@pytest.mark.parametrize("case", ["chain", "fluid", "random1", "random2", "diag"])
@pytest.mark.parametrize("amalg", [0, 1])
def test_symbolic_contains_true_fill(case, amalg):
    if case == "chain":
        s = ns.make_chain(natoms=30, seed=2); n, cp, ri = s.n, s.colptr, s.rowind
    elif case == "fluid":
        s = ns.make_fluid(nmol=12, seed=4, cutoff=6.0); n, cp, ri = s.n, s.colptr, s.rowind
    elif case == "diag":
        n = 40; cp = np.arange(n + 1, dtype=np.int64); ri = np.arange(n, dtype=np.int32)
    else:
        n = 150 if case == "random1" else 211
        cp, ri = random_pattern(n, 0.02 if case == "random1" else 0.05, seed=len(case))
    plan = px.pexsi_setup(n, cp, ri, opts=host_opts(amalgamate=amalg, leaf_cols=16))
    perm = px.pexsi_plan_get_perm(plan)
    assert sorted(perm.tolist()) == list(range(n))
    first, rptr, rows, parent = px.pexsi_plan_get_supernodes(plan)
    st = px.pexsi_plan_get_stats(plan)
    px.pexsi_plan_destroy(plan)
    fill = brute_force_fill(n, cp, ri, perm)
    ns_ = first.shape[0] - 1
    assert first[0] == 0 and first[-1] == n and np.all(np.diff(first) > 0)
    col2sn = np.repeat(np.arange(ns_), np.diff(first))
    nnzL = 0
    for K in range(ns_):
        own = set(range(first[K], first[K + 1]))
        struct = rows[rptr[K]:rptr[K + 1]]
        assert np.all(np.diff(struct) > 0) and (struct.size == 0 or struct[0] >= first[K + 1])
        front = own | set(struct.tolist())
        for j in range(first[K], first[K + 1]):
            assert set(fill[j].tolist()) <= front, (K, j)
        sK = first[K + 1] - first[K]
        nnzL += sK * (sK + 1) // 2 + sK * struct.size
        if struct.size:
            P = parent[K]
            assert P == col2sn[struct[0]] and P > K       # Eq. parent
            pf = set(range(first[P], first[P + 1])) | set(rows[rptr[P]:rptr[P + 1]].tolist())
            assert set(struct.tolist()) <= pf               # multifrontal containment
        else:
            assert parent[K] == -1
    assert st["nnz_L"] == nnzL
    true_nnz = sum(len(f) + 1 for f in fill)
    assert nnzL >= true_nnz
    if not amalg:
        assert nnzL == true_nnz   # fundamental supernodes add no zeros


def test_setup_accepts_caller_permutation():
    s = ns.make_chain(natoms=20, seed=1)
    perm = np.arange(s.n)[::-1].copy()
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, perm=perm, opts=host_opts(amalgamate=0))
    p2 = px.pexsi_plan_get_perm(plan)
    px.pexsi_plan_destroy(plan)
    assert sorted(p2.tolist()) == list(range(s.n))
