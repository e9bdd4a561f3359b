"""Failure paths, made to happen without faulting the GPU.

- A bounded device-side wait that runs out: with pexsi_opts.inject = 1, CTA 0
  of each short-K split GEMM launch issues no operand copy, so its MMA
  issuer's wait (bounded by pexsi_opts.wait_ns, 2 ms here) runs out; every
  role of the CTA returns, TMEM is freed, the later launches of the call
  return at once, and the call returns PEXSI_ERR_TIMEOUT. The context stays
  usable: a plan without injection then gives the oracle's result.
- A device budget below one pole's workspace: the call returns
  PEXSI_ERR_NOMEM before it allocates anything; a budget that fits a few
  poles gives a smaller batch and the oracle's result.
- A breakdown in an early pole batch of a chain: with inject = 2 the host
  records a breakdown of front 0 after the first batch of a call with
  accumulate = 0. Calls that accumulate keep the status, so the call that
  reads it (info), and the server's request, report BREAKDOWN although the
  last batch itself is clean.
"""
import numpy as np
import pytest

import nao_synth as ns
from oracle import dense

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1405_0194_gb300 as px  # noqa: E402

WAIT_NS = 2_000_000  # 2 ms


@pytest.fixture(scope="module")
def chain():
    from paper_1405_0194_gb300 import build
    build.build()
    s = ns.make_chain()
    mu, dE = ns.mu_and_delta_e(s)
    return s, mu, dE


def test_timed_out_wait_returns_timeout_and_context_survives(chain):
    s, mu, dE = chain
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind,
                          opts=px.pexsi_opts_default(split_slices=6, inject=1, wait_ns=WAIT_NS))
    try:
        with pytest.raises(px.PexsiError) as e:
            px.pexsi_dm(plan, s.H, s.S, mu, s.beta, 8, dE)
        assert e.value.code == px.capi.PEXSI_ERR_TIMEOUT
        assert "wait ran out" in str(e.value)
        # the real split GEMMs of the inertia LDL^T take the same path
        with pytest.raises(px.PexsiError) as e:
            px.pexsi_inertia(plan, s.H, s.S, [mu])
        assert e.value.code == px.capi.PEXSI_ERR_TIMEOUT
    finally:
        px.pexsi_plan_destroy(plan)
    torch.cuda.synchronize()  # no sticky error: the launches returned normally
    dm0, *_ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, 8, dE)
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(split_slices=6))
    dm, *_ = px.pexsi_dm(plan, s.H, s.S, mu, s.beta, 8, dE)
    px.pexsi_plan_destroy(plan)
    assert np.max(np.abs(dm - dm0)) <= 1e-7


def test_breakdown_in_an_early_batch_is_reported_at_the_end_of_the_chain(chain):
    s, mu, dE = chain
    P = 12
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(max_batch=4, inject=2))
    dH = torch.from_numpy(s.H).cuda(); dS = torch.from_numpy(s.S).cuda()
    out = torch.zeros(3, s.nnz, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    ptrs = [out[k].data_ptr() for k in range(3)]
    try:
        # one call over three batches: the first batch's breakdown survives
        with pytest.raises(px.PexsiError) as e:
            px.pexsi_dm(plan, s.H, s.S, mu, s.beta, P, dE)
        assert e.value.code == px.capi.PEXSI_ERR_BREAKDOWN
        # a chain of calls: clean accumulating calls keep the status
        px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, 0, 4, 0, *ptrs, st)
        px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, 4, 8, 1, *ptrs, st)
        with pytest.raises(px.PexsiError) as e:
            px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, 8, 12, 1, *ptrs, st,
                               want_info=True)
        assert e.value.code == px.capi.PEXSI_ERR_BREAKDOWN
        # inertia keeps status words of its own: the chain's breakdown does
        # not leak into it
        cnt = px.pexsi_inertia(plan, s.H, s.S, [mu])
        assert cnt[0] == int(np.sum(dense.eig_pencil(s.n, s.colptr, s.rowind, s.H, s.S)[0] < mu))
    finally:
        px.pexsi_plan_destroy(plan)
    # without injection the same chain is clean
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(max_batch=4))
    px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, 0, 4, 0, *ptrs, st)
    info = px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, 4, 12, 1, *ptrs, st,
                              want_info=True)
    px.pexsi_plan_destroy(plan)
    assert info["breakdown_front"] == -1


def test_server_reports_a_breakdown_of_an_early_batch(chain):
    s, mu, dE = chain
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(inject=2))
    clean = px.pexsi_setup(s.n, s.colptr, s.rowind)
    server = px.pexsi_server_create(px.pexsi_server_opts_default(slots=2, batch=4))
    try:
        bad = px.ServerRequest(plan, s.H, s.S, mu=mu, beta=s.beta, n_poles=16, delta_e=dE)
        good = px.ServerRequest(clean, s.H, s.S, mu=mu, beta=s.beta, n_poles=16, delta_e=dE)
        px.pexsi_server_submit(server, bad)
        px.pexsi_server_submit(server, good)
        rb = px.pexsi_server_wait(server, bad.ticket)
        rg = px.pexsi_server_wait(server, good.ticket)
    finally:
        px.pexsi_server_destroy(server)
        px.pexsi_plan_destroy(plan)
        px.pexsi_plan_destroy(clean)
    # four batches of 4 poles; the breakdown happened in the first
    assert rb["status"] == px.capi.PEXSI_ERR_BREAKDOWN and rb["breakdown_front"] == 0
    assert rg["status"] == 0


def test_budget_below_one_pole_returns_nomem(chain):
    s, mu, dE = chain
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(hbm_budget=4096))
    try:
        with pytest.raises(px.PexsiError) as e:
            px.pexsi_dm(plan, s.H, s.S, mu, s.beta, 8, dE)
        assert e.value.code == px.capi.PEXSI_ERR_NOMEM
        assert "exceeds the HBM budget" in str(e.value)
        assert px.pexsi_plan_get_stats(plan)["batch"] == 0  # nothing allocated
    finally:
        px.pexsi_plan_destroy(plan)
    # the workspace of a 2-pole batch as the budget: the plan chooses a
    # batch that fits it and still gives the oracle's result
    probe = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(max_batch=2))
    px.pexsi_inertia(probe, s.H, s.S, [mu])
    two = px.pexsi_plan_get_stats(probe)["workspace_bytes"]
    px.pexsi_plan_destroy(probe)
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(hbm_budget=two))
    try:
        dm, *_ = px.pexsi_dm(plan, s.H, s.S, mu, s.beta, 8, dE)
        st = px.pexsi_plan_get_stats(plan)
    finally:
        px.pexsi_plan_destroy(plan)
    assert 1 <= st["batch"] <= 2 and st["workspace_bytes"] <= two
    dm0, *_ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, 8, dE)
    assert np.max(np.abs(dm - dm0)) <= 1e-10
