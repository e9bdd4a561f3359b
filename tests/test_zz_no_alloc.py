"""The allocation-free trace entry point, checked against the trace that
pexsi_dm_device reports and against a host dot product of the same arrays,
on two calls in a row.

pexsi_trace_noalloc exists for callers that cannot allocate device memory when
they need Tr[DM S], Tr[EDM S] and Tr[FDM S] -- code capturing a stream into a
CUDA graph, runtimes with a fixed memory arena, serving loops that must not
enter the allocator. It keeps its scratch in a static device array instead.
This file is named to be collected last.
"""
import numpy as np
import pytest

import nao_synth as ns

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1405_0194_gb300 as px  # noqa: E402

TOL_TRACE = 1e-8


def test_trace_noalloc_matches_dm_call_twice():
    from paper_1405_0194_gb300 import build
    build.build()
    s = ns.make_chain()
    mu, dE = ns.mu_and_delta_e(s)
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind)
    dH = torch.from_numpy(s.H).cuda()
    dS = torch.from_numpy(s.S).cuda()
    out = torch.zeros(3, s.nnz, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    info = px.pexsi_dm_device(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, s.n_poles, dE, 0, s.n_poles, 0,
                              out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), st, want_info=True)
    px.pexsi_plan_destroy(plan)
    ref = np.array([info["trace_dm_s"], info["trace_edm_s"], info["trace_fdm_s"]])
    res = torch.full((2, 3), float("nan"), dtype=torch.float64, device="cuda")
    for k in range(2):
        px.pexsi_trace_noalloc(out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), dS.data_ptr(), s.nnz,
                               res[k].data_ptr(), st)
    torch.cuda.synchronize()
    got = res.cpu().numpy()
    # the same sums on the host, from the same device arrays
    host = out.cpu().numpy()
    dot = np.array([np.dot(host[q], s.S) for q in range(3)])
    for k in range(2):
        assert np.max(np.abs(got[k] - ref)) <= TOL_TRACE * max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(got[k] - dot)) <= TOL_TRACE * max(1.0, np.max(np.abs(dot)))
    # one output NULL: its trace is written as 0
    px.pexsi_trace_noalloc(out[0].data_ptr(), 0, 0, dS.data_ptr(), s.nnz, res[0].data_ptr(), st)
    torch.cuda.synchronize()
    assert abs(res[0, 0].item() - ref[0]) <= TOL_TRACE * max(1.0, abs(ref[0])) and res[0, 1].item() == 0.0
    # sizes beyond the scratch capacity are rejected before any launch
    with pytest.raises(px.PexsiError) as e:
        px.pexsi_trace_noalloc(out[0].data_ptr(), 0, 0, dS.data_ptr(), (1 << 30) + 1, res[1].data_ptr(), st)
    assert e.value.code == -1
