"""The continuous-batching request server: each result is the same alone and
in the mix (requests of different sizes admitted concurrently), admission
respects the HBM budget, and cancellation works."""
import numpy as np
import pytest

import nao_synth as ns

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1405_0194_gb300 as px  # noqa: E402

TOL_DM = 1e-10


@pytest.fixture(scope="module")
def systems():
    from paper_1405_0194_gb300 import build
    build.build()
    out = []
    for s in (ns.make_chain(), ns.make_fluid(nmol=24, seed=1), ns.make_sheet(ncell=8, seed=2),
              ns.make_chain(natoms=37, seed=5, norb=5)):
        mu, dE = ns.mu_and_delta_e(s)
        plan = px.pexsi_setup(s.n, s.colptr, s.rowind)
        out.append((s, mu, dE, plan))
    yield out
    for *_, plan in out:
        px.pexsi_plan_destroy(plan)


def _alone(s, mu, dE, plan, P, shifts):
    dm, edm, fdm, info = px.pexsi_dm(plan, s.H, s.S, mu, s.beta, P, dE)
    cnt = px.pexsi_inertia(plan, s.H, s.S, shifts)
    return dm, edm, fdm, cnt, info


def test_results_same_alone_and_in_the_mix(systems):
    rng = np.random.default_rng(3)
    jobs = []
    for k in range(12):
        s, mu, dE, plan = systems[k % len(systems)]
        m = mu + 0.02 * rng.standard_normal()     # mu jitter per request
        shifts = m + np.linspace(-0.4, 0.4, 8) + 1.0e-4
        P = 20
        jobs.append((s, m, dE, plan, P, shifts))
    server = px.pexsi_server_create(px.pexsi_server_opts_default(slots=4, batch=6))
    try:
        reqs = []
        for s, m, dE, plan, P, shifts in jobs:
            r = px.ServerRequest(plan, s.H, s.S, mu=m, beta=s.beta, n_poles=P, delta_e=dE, shifts=shifts)
            px.pexsi_server_submit(server, r)
            reqs.append(r)
        results = [px.pexsi_server_wait(server, r.ticket) for r in reqs]
        stats = px.pexsi_server_get_stats(server)
    finally:
        px.pexsi_server_destroy(server)
    assert stats["completed"] == len(jobs) and stats["failed"] == 0
    assert stats["peak_concurrent"] >= 2            # requests overlapped on the device
    for (s, m, dE, plan, P, shifts), r, res in zip(jobs, reqs, results):
        assert res["status"] == 0
        dm, edm, fdm, cnt, info = _alone(s, m, dE, plan, P, shifts)
        assert np.max(np.abs(r.dm - dm)) <= TOL_DM
        assert np.max(np.abs(r.edm - edm)) <= TOL_DM * max(1.0, np.max(np.abs(edm)))
        assert np.max(np.abs(r.fdm - fdm)) <= TOL_DM * max(1.0, np.max(np.abs(fdm)))
        assert r.counts.tolist() == cnt.tolist()
        assert abs(res["trace_dm_s"] - info["trace_dm_s"]) <= 1e-8
        assert res["latency_ms"] >= res["run_ms"] > 0


def test_admission_by_footprint(systems):
    s, mu, dE, plan = systems[2]
    server = px.pexsi_server_create(px.pexsi_server_opts_default(slots=4, batch=4))
    probe = px.ServerRequest(plan, s.H, s.S, mu=mu, beta=s.beta, n_poles=8, delta_e=dE)
    px.pexsi_server_submit(server, probe)
    fp = px.pexsi_server_wait(server, probe.ticket)["footprint_bytes"]
    px.pexsi_server_destroy(server)
    # a budget that holds one request at a time: no two may run together
    server = px.pexsi_server_create(px.pexsi_server_opts_default(slots=4, batch=4, hbm_budget=int(fp * 1.5)))
    try:
        reqs = [px.ServerRequest(plan, s.H, s.S, mu=mu, beta=s.beta, n_poles=8, delta_e=dE) for _ in range(5)]
        for r in reqs:
            px.pexsi_server_submit(server, r)
        res = [px.pexsi_server_wait(server, r.ticket) for r in reqs]
        st = px.pexsi_server_get_stats(server)
    finally:
        px.pexsi_server_destroy(server)
    assert all(x["status"] == 0 for x in res)
    assert st["peak_concurrent"] == 1 and st["peak_bytes"] <= st["budget"]
    for r in reqs[1:]:
        assert np.array_equal(r.dm, reqs[0].dm)


def test_cancel_and_bad_requests(systems):
    s, mu, dE, plan = systems[1]
    server = px.pexsi_server_create(px.pexsi_server_opts_default(slots=1, batch=2))
    try:
        reqs = [px.ServerRequest(plan, s.H, s.S, mu=mu, beta=s.beta, n_poles=40, delta_e=dE) for _ in range(4)]
        for r in reqs:
            px.pexsi_server_submit(server, r)
        px.pexsi_server_cancel(server, reqs[-1].ticket)       # still queued behind the others
        res = [px.pexsi_server_wait(server, r.ticket) for r in reqs]
        with pytest.raises(px.PexsiError):
            px.pexsi_server_submit(server, px.ServerRequest(plan, s.H, s.S, n_poles=3, beta=1.0, delta_e=1.0))
    finally:
        px.pexsi_server_destroy(server)
    assert res[-1]["status"] == -7
    assert all(x["status"] == 0 for x in res[:-1])


def test_small_request_passes_a_large_one_that_does_not_fit(systems):
    """Under a budget that holds the large request alone or the small ones
    beside the one running, a small request queued behind a large one that
    does not fit yet is admitted first (the large one runs once there is
    room; bypasses are bounded, so it still runs)."""
    small_s, mu_s, dE_s, small_plan = systems[0]   # chain64, n = 256
    big_s, mu_b, dE_b, big_plan = systems[2]        # sheet8, n = 1,664
    server = px.pexsi_server_create(px.pexsi_server_opts_default(slots=4, batch=8))
    probes = [px.ServerRequest(p, s.H, s.S, mu=m, beta=s.beta, n_poles=16, delta_e=d)
              for s, m, d, p in ((small_s, mu_s, dE_s, small_plan), (big_s, mu_b, dE_b, big_plan))]
    fps = []
    for r in probes:
        px.pexsi_server_submit(server, r)
        fps.append(px.pexsi_server_wait(server, r.ticket)["footprint_bytes"])
    px.pexsi_server_destroy(server)
    fs, fb = fps
    assert fb > 2 * fs
    # room for the large one alone, or for a few small ones, not for both
    server = px.pexsi_server_create(px.pexsi_server_opts_default(slots=4, batch=8, hbm_budget=int(fb + 0.5 * fs)))
    try:
        first = px.ServerRequest(small_plan, small_s.H, small_s.S, mu=mu_s, beta=small_s.beta, n_poles=40,
                                 delta_e=dE_s)
        big = px.ServerRequest(big_plan, big_s.H, big_s.S, mu=mu_b, beta=big_s.beta, n_poles=16, delta_e=dE_b)
        late = px.ServerRequest(small_plan, small_s.H, small_s.S, mu=mu_s, beta=small_s.beta, n_poles=8,
                                delta_e=dE_s)
        for r in (first, big, late):
            px.pexsi_server_submit(server, r)
        res = [px.pexsi_server_wait(server, r.ticket) for r in (first, big, late)]
    finally:
        px.pexsi_server_destroy(server)
    assert all(x["status"] == 0 for x in res)
    r_first, r_big, r_late = res
    # the late small request ran beside the first one, before the large one started
    assert r_late["max_concurrent"] == 2
    assert r_big["queue_ms"] > r_late["queue_ms"]
