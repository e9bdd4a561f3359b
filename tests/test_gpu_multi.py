"""The pole-sharded DM and shift-sharded inertia drivers (multi.py) on the
GPU with one rank: the per-rank calls run the CUDA path through the C ABI,
the sum-allreduce and the all-gather run through torch.distributed (NCCL),
and the result must equal the CPU oracle. The sharding arithmetic with more
ranks is covered by the gloo CPU test (tests/test_multi_rank.py)."""
import socket

import numpy as np
import pytest

import nao_synth as ns
from oracle import dense

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import torch.distributed as dist  # noqa: E402

import paper_1405_0194_gb300 as px  # noqa: E402
from paper_1405_0194_gb300 import multi  # noqa: E402


def _port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


@pytest.fixture(scope="module")
def group():
    from paper_1405_0194_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    backend = "nccl" if dist.is_nccl_available() else "gloo"
    dist.init_process_group(backend, init_method=f"tcp://127.0.0.1:{_port()}", rank=0, world_size=1)
    yield backend
    dist.destroy_process_group()


def test_dm_sharded_and_inertia_sharded_one_rank(group):
    s = ns.make_chain(natoms=37, seed=5, norb=5)
    mu, dE = ns.mu_and_delta_e(s)
    P = 16
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(max_batch=4))
    dH = torch.from_numpy(s.H).cuda(); dS = torch.from_numpy(s.S).cuda()
    out = torch.full((3, s.nnz), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    multi.dm_sharded(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, P, dE, out, st, batch=3)
    shifts = mu + np.linspace(-0.6, 0.6, 7) + 1.234e-4
    cnt = multi.inertia_sharded(plan, dH.data_ptr(), dS.data_ptr(), shifts, st, device=torch.device("cuda"))
    px.pexsi_plan_destroy(plan)
    dm0, edm0, fdm0, _ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, P, dE)
    got = out.cpu().numpy()
    print(f"backend {group}: max|dDM| = {np.max(np.abs(got[0] - dm0)):.3e}")
    assert np.max(np.abs(got[0] - dm0)) <= 1e-10
    assert np.max(np.abs(got[1] - edm0)) <= 1e-10 * max(1.0, np.max(np.abs(edm0)))
    assert np.max(np.abs(got[2] - fdm0)) <= 1e-10 * max(1.0, np.max(np.abs(fdm0)))
    ref = dense.inertia_counts(s.n, s.colptr, s.rowind, s.H, s.S, shifts)
    assert cnt.tolist() == ref.tolist()


def test_dm_sharded_raises_on_a_breakdown_in_an_early_batch(group):
    """With a breakdown recorded after the rank's first batch, its last
    batch reads the chain's status and raises before the collective."""
    s = ns.make_chain()
    mu, dE = ns.mu_and_delta_e(s)
    plan = px.pexsi_setup(s.n, s.colptr, s.rowind, opts=px.pexsi_opts_default(max_batch=4, inject=2))
    dH = torch.from_numpy(s.H).cuda(); dS = torch.from_numpy(s.S).cuda()
    out = torch.zeros(3, s.nnz, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    try:
        with pytest.raises(px.PexsiError) as e:
            multi.dm_sharded(plan, dH.data_ptr(), dS.data_ptr(), mu, s.beta, 12, dE, out, st, batch=4)
        assert e.value.code == px.capi.PEXSI_ERR_BREAKDOWN
    finally:
        px.pexsi_plan_destroy(plan)
