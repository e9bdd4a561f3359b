"""Multi-rank host logic of the pole-parallel path, on CPU ranks (gloo,
world size 2): the pole shards cover every pole exactly once, the
sum-allreduce of per-rank partial pole sums reproduces the single-process
DM / EDM / FDM of Eq. gammapole and Eq. gammaF, and the all-gathered inertia
counts come back in shift order. The per-rank compute is the oracle (the
orchestration under test is the same one the GPU ranks run)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1405_0194_gb300.multi import shard  # noqa: E402


def test_shard_partition():
    for count in (0, 1, 5, 40, 60, 61):
        for world in (1, 2, 3, 4, 8):
            spans = [shard(count, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == count
            for (b0, e0), (b1, e1) in zip(spans, spans[1:]):
                assert e0 == b1
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_poles, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put(_rank_work(rank, n_poles))
    except Exception as e:  # reported to the parent instead of leaving it waiting
        q.put((rank, "error", repr(e), None))
    finally:
        dist.destroy_process_group()


def _rank_work(rank, n_poles):
    import torch

    import nao_synth as ns
    from oracle import dense, poles
    import torch.distributed as dist

    from paper_1405_0194_gb300 import multi
    from paper_1405_0194_gb300.multi import dm_allreduce, inertia_allgather

    s = ns.make_chain(natoms=16, seed=3)
    mu, dE = ns.mu_and_delta_e(s)
    tab = poles.pole_table(s.beta, dE, n_poles, mu)
    Hd = dense.dense_from_csc(s.n, s.colptr, s.rowind, s.H)
    Sd = dense.dense_from_csc(s.n, s.colptr, s.rowind, s.S)
    r, c = dense.pattern_coords(s.n, s.colptr, s.rowind)
    out = torch.zeros(3, s.nnz, dtype=torch.float64)
    seen = []

    def compute_range(b, e, acc, last):
        # the status of a rank's chain is read on its final batch alone
        assert last == (e == multi.shard(n_poles, dist.get_world_size(), dist.get_rank())[1])
        seen.extend(range(b, e))
        part = np.zeros((3, s.nnz))
        for l in range(b, e):
            sel = dense.shifted_inverse(Hd, Sd, tab["z"][l])[r, c]
            part[0] += np.imag(tab["w_rho"][l] * sel)
            part[1] += np.imag(tab["w_E"][l] * sel)
            part[2] += np.imag(tab["w_F"][l] * sel)
        if acc:
            out.add_(torch.from_numpy(part))
        else:
            out.copy_(torch.from_numpy(part))

    dm_allreduce(compute_range, out, n_poles, batch=3)
    shifts = mu + np.linspace(-0.4, 0.4, 7)
    counts = inertia_allgather(lambda sh: dense.inertia_counts(s.n, s.colptr, s.rowind, s.H, s.S, sh), shifts)
    return rank, seen, out.numpy().copy(), counts


def _run(world, n_poles):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n_poles, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    errors = [r for r in res if isinstance(r[1], str)]
    assert not errors, errors
    assert all(p.exitcode == 0 for p in procs)
    return sorted(res, key=lambda t: t[0])


@pytest.mark.parametrize("world,n_poles", [(2, 20), (3, 2)])
def test_pole_sharded_dm_and_inertia_gloo(world, n_poles):
    """(3, 2): the third rank owns no pole and contributes zeros."""
    import nao_synth as ns
    from oracle import dense, poles

    res = _run(world, n_poles)
    s = ns.make_chain(natoms=16, seed=3)
    mu, dE = ns.mu_and_delta_e(s)
    tab = poles.pole_table(s.beta, dE, n_poles, mu)
    dm, edm, fdm, _ = dense.density_matrices(s.n, s.colptr, s.rowind, s.H, s.S, mu, s.beta, n_poles, dE, table=tab)
    ref = np.stack([dm, edm, fdm])
    # every pole evaluated exactly once across the ranks
    assert sorted(p for _, seen, _, _ in res for p in seen) == list(range(n_poles))
    for _, _, out, _ in res:  # the reduced sum on every rank
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))
    counts = dense.inertia_counts(s.n, s.colptr, s.rowind, s.H, s.S, mu + np.linspace(-0.4, 0.4, 7))
    for *_, got in res:
        np.testing.assert_array_equal(got, counts)
