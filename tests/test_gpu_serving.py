"""Request scheduler (ssqcd_server_*): several eigen-window requests on
different lattices and precisions in flight together.  Each result must be
the same as the request solved alone (bit for bit: a request's arithmetic
and reduction order do not depend on the others), admission must keep the
running requests within the memory budget, and a request larger than the
budget is refused at submission."""
import json
import os

import numpy as np
import pytest

from tests._lib import gpu_module

import bench
import synthetic

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "windows.json")


@pytest.fixture(scope="module")
def setup():
    import torch
    ss = gpu_module()
    stream = torch.cuda.Stream()
    dims4 = (4, 4, 4, 4)
    U4 = synthetic.gauge_field(dims4, "haar", seed=1)
    lat4 = ss.create_lattice(dims4, 0.13, -1, stream=stream)
    ss.upload_gauge(lat4, U4)
    lat4df = ss.create_lattice(dims4, 0.13, -1, precision=ss.DF, stream=stream)
    ss.upload_gauge(lat4df, U4)
    w = bench.CONFIG2
    U8, src8 = bench.make_inputs(0, bench.CONFIG2)
    lat8 = ss.create_lattice(w["dims"], w["kappa"], w["bc_t"], precision=ss.FP64_DFSHIFT, stream=stream)
    ss.upload_gauge(lat8, U8)
    reqs = [
        (lat4, (0.374, 0.3930), 16, 8, synthetic.gaussian_sources(dims4, 3, seed=100), dict(beta=0.3, nprime=14)),
        (lat4, (0.374, 0.3930), 20, 6, synthetic.gaussian_sources(dims4, 2, seed=101), dict(beta=0.4, nprime=16)),
        (lat4df, (0.374, 0.3930), 16, 8, synthetic.gaussian_sources(dims4, 3, seed=102), dict(beta=0.3, nprime=14)),
        (lat8, w["interval"], w["N"], w["M"], src8, dict(beta=w["beta"], nprime=w["nprime"])),
    ]
    alone = []
    for lat, iv, N, M, src, kw in reqs:
        res = ss.ss_solve(lat, iv, N, M, src, **kw)
        assert res.status == ss.OK, res.error
        ev, _, rs, st = ss.ss_eigpairs(res, want_vectors=False)
        alone.append((ev, rs, st["iterations"]))
    return ss, reqs, alone


def _drain(ss, srv, ids, budget=None, est=None):
    seen_running = []
    while True:
        srv.progress(wait=True)
        states = {i: srv.status(i)[0] for i in ids}
        running = [i for i, s in states.items() if s == srv.RUNNING]
        seen_running.append(running)
        if budget is not None and len(running) > 1:
            assert sum(est[i] for i in running) <= budget
        if all(s in (srv.DONE, srv.FAILED) for s in states.values()):
            return seen_running


def test_results_same_alone_and_in_the_mix(setup):
    ss, reqs, alone = setup
    srv = ss.Server()
    ids = [srv.submit(lat, iv, N, M, src, **kw) for lat, iv, N, M, src, kw in reqs]
    assert srv.counts() == (len(ids), 0, 0)
    seen = _drain(ss, srv, ids)
    assert max(len(r) for r in seen) >= 2  # requests overlapped on the device
    for i, (ev0, rs0, it0) in zip(ids, alone):
        state, lat_ms = srv.status(i)
        assert state == srv.DONE and lat_ms > 0
        res = srv.take(i)
        assert res.status == ss.OK, res.error
        ev, _, rs, st = ss.ss_eigpairs(res, want_vectors=False)
        assert st["iterations"] == it0
        assert np.array_equal(ev, ev0) and np.array_equal(rs, rs0)
    assert srv.counts() == (0, 0, 0)
    srv.close()


def test_admission_keeps_running_requests_within_the_budget(setup):
    ss, reqs, alone = setup
    probe = ss.Server(memory_budget=1 << 40)
    est = [probe.request_bytes(probe.submit(lat, iv, N, M, src, **kw)) for lat, iv, N, M, src, kw in reqs]
    probe.close()
    budget = max(est)  # the largest fits alone; it cannot share the device with the others
    srv = ss.Server(memory_budget=budget)
    ids = [srv.submit(lat, iv, N, M, src, **kw) for lat, iv, N, M, src, kw in reqs]
    seen = _drain(ss, srv, ids, budget=budget, est=dict(zip(ids, est)))
    big = ids[int(np.argmax(est))]
    assert all(r == [big] for r in seen if big in r)  # the largest always ran alone
    # admission deferred requests on memory (the first one runs at once, the
    # others queue while it holds the budget), and their results below are
    # still bit-identical to the solo runs
    assert srv.deferred() >= 1
    for i, (ev0, rs0, _) in zip(ids, alone):
        res = srv.take(i)
        ev, _, rs, _ = ss.ss_eigpairs(res, want_vectors=False)
        assert np.array_equal(ev, ev0) and np.array_equal(rs, rs0)
    srv.close()


def test_request_above_the_budget_is_refused(setup):
    ss, reqs, _ = setup
    srv = ss.Server(memory_budget=1 << 20)
    lat, iv, N, M, src, kw = reqs[0]
    with pytest.raises(ss.SsqcdError) as e:
        srv.submit(lat, iv, N, M, src, **kw)
    assert e.value.code == ss.ERR_OOM
    assert srv.counts() == (0, 0, 0)
    srv.close()


def test_window_list_request_with_source_blocks(setup):
    """A request for two windows (one on each side of the gap) whose sources
    run in blocks of one: the scheduler chains the blocks' shifted-CG runs
    and forms the moments block by block; the result is bit-identical to
    ssqcd_ss_solve_windows with the same blocks, alone and next to other
    requests."""
    ss, reqs, alone = setup
    lat4 = reqs[0][0]
    src = synthetic.gaussian_sources((4, 4, 4, 4), 3, seed=103)
    wins = [(-0.3932, -0.3785), (0.374, 0.3930)]
    res = ss.ss_solve_windows(lat4, wins, 16, 8, src, beta=0.3, nprime=14, source_block=1)
    assert res.status == ss.OK, res.error
    ev0, _, rs0, st0 = ss.ss_eigpairs(res, want_vectors=False)
    assert len(ev0) == 16 and np.max(rs0) <= 1e-8
    srv = ss.Server()
    rid = srv.submit_windows(lat4, wins, 16, 8, src, beta=0.3, nprime=14, source_block=1)
    others = [srv.submit(lat, iv, N, M, s, **kw) for lat, iv, N, M, s, kw in reqs[:2]]
    _drain(ss, srv, [rid] + others)
    out = srv.take(rid)
    assert out.status == ss.OK, out.error
    ev, _, rs, st = ss.ss_eigpairs(out, want_vectors=False)
    assert np.array_equal(ev, ev0) and np.array_equal(rs, rs0)
    assert st["iterations"] == st0["iterations"]
    for i in others:
        assert srv.take(i).status == ss.OK
    srv.close()


def test_update_form_requests_with_different_shift_counts_side_by_side(setup):
    """Two requests whose float-float shift vectors are updated by the
    TMA-fed kernel (its shared memory grows with N x L), the one with fewer
    shifts admitted second: the kernel's shared-memory limit is shared by the
    process, so the second request must not lower it below the first one's
    need.  Both finish and equal their solo runs bit for bit."""
    ss, reqs, alone = setup
    lat8 = reqs[3][0]
    w = bench.CONFIG2
    _, src8 = bench.make_inputs(0, bench.CONFIG2)
    items = [(w["N"], src8), (16, src8[:1])]
    solo = []
    for N, src in items:
        res = ss.ss_solve(lat8, w["interval"], N, w["M"], src, beta=w["beta"], nprime=min(w["nprime"], N))
        assert res.status == ss.OK, res.error
        ev, _, rs, _ = ss.ss_eigpairs(res, want_vectors=False)
        solo.append((ev, rs))
    srv = ss.Server()
    ids = [srv.submit(lat8, w["interval"], N, w["M"], src, beta=w["beta"], nprime=min(w["nprime"], N))
           for N, src in items]
    _drain(ss, srv, ids)
    for i, (ev0, rs0) in zip(ids, solo):
        out = srv.take(i)
        assert out.status == ss.OK, out.error
        ev, _, rs, _ = ss.ss_eigpairs(out, want_vectors=False)
        assert np.array_equal(ev, ev0) and np.array_equal(rs, rs0)
    srv.close()


def test_batched_uneven_requests_match_their_solo_runs():
    """The batched workload's first six requests (8^4, 12^4 and 16^4 fields,
    each with its own window, L and N) submitted at once through the
    scheduler, in FP64 and float-float: none fails, each request's
    eigenvalues and residuals equal its solo run bit for bit, and each
    cluster window's converged eigenvalues lie in its interval."""
    ss = gpu_module()
    import torch
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    try:
        out = bench.run_batched_uneven(ss, stream, n_requests=6, solo_checks=6)
    finally:
        torch.cuda.set_stream(torch.cuda.default_stream())
    for arm in ("plain_fp64", "mixed"):
        r = out[arm]
        assert r["failed"] == 0
        assert r["solo_identical"] == "6 of 6"
        assert r["eigenpairs"] >= 12
