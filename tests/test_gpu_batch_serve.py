"""Batched jobs, CUDA-graph replay and the continuous-batching server.

Every job's result must equal the single-job result bit for bit, whether it
runs alone, in a multi-stream batch, in a replayed graph, or on the server
beside other requests (the kernels are deterministic and jobs share nothing).
Jobs mix dimension, N, box size, rank and precision, as batched workloads do.
"""
import numpy as np
import pytest

from paper_2501_05528_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

JOBS = [  # kernel, d, grid, n, k, e, precision, seed
    ("laplace2d", 2, (4, 4), 2600, 8, 3, 0, 1),
    ("laplace3d", 3, (3, 3, 3), 3000, 6, 1, 1, 2),
    ("laplace2d", 2, (8, 4), 5000, 12, 3, 1, 3),
    ("laplace2d", 2, (5, 5), 1500, 4, 0, 0, 4),
    ("laplace3d", 3, (4, 4, 4), 4100, 8, 2, 0, 5),
]


def _tb():
    from paper_2501_05528_gb300 import tblr
    return tblr


def _make(spec):
    tb = _tb()
    kernel, d, grid, n, k, e, prec, seed = spec
    pts = inputs.uniform_points(n, d, seed=seed)
    b = int(np.prod(grid))
    T, G, H = inputs.tagging_draws(b, 3 ** d + 1 + e, n, k + 10, seed=seed + 50)
    prob = tb.make_problem(d, kernel, n, grid, (0.0,) * d, (1.0,) * d, k, 10, e, precision=prec)
    return prob, pts, T, G, H


def _host(o):
    return {name: getattr(o, name).cpu().numpy() for name in ("u", "v", "at", "ranks")} | {
        "bnear": o.bnear.cpu().numpy()[:o.total]}


@pytest.fixture(scope="module")
def singles():
    tb = _tb()
    dev = torch.device("cuda")
    out = []
    for spec in JOBS:
        prob, pts, T, G, H = _make(spec)
        t = lambda a: torch.as_tensor(a, device=dev)
        res = tb.compress(prob, t(pts), t(T), t(G), t(H))
        torch.cuda.synchronize()
        out.append(_host(res))
    assert tb.tblr_device_timeouts() == 0
    return out


def _batch_jobs():
    tb = _tb()
    dev = torch.device("cuda")
    jobs = []
    for spec in JOBS:
        prob, pts, T, G, H = _make(spec)
        t = lambda a: torch.as_tensor(a, device=dev)
        jobs.append(tb.BatchJob(prob, t(pts), t(T), t(G), t(H)))
    tb.tblr_batch_plan(jobs)
    return jobs


def _same(a, b):
    for key in a:
        assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("n_streams", [1, 3])
def test_batch_equals_single_jobs(singles, n_streams):
    tb = _tb()
    jobs = _batch_jobs()
    tb.tblr_batch_run(jobs, n_streams=n_streams)
    torch.cuda.synchronize()
    for j, ref in zip(jobs, singles):
        _same(_host(j.out), ref)


def test_graph_replay_equals_single_jobs(singles):
    tb = _tb()
    jobs = _batch_jobs()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = tb.Graph(jobs, n_streams=4)
        for j in jobs:                      # clear outputs, then replay twice
            j.out.u.zero_()
            j.out.at.zero_()
        g.launch()
        g.launch()
    torch.cuda.synchronize()
    for j, ref in zip(jobs, singles):
        _same(_host(j.out), ref)
    del g


def test_server_result_is_the_same_alone_and_in_the_mix(singles):
    tb = _tb()
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
    reqs = []
    for spec, ref in zip(JOBS, singles):
        prob, pts, T, G, H = _make(spec)
        reqs.append((prob, pin(pts), pin(T), pin(G), pin(H), len(ref["bnear"])))
    # a budget of about two jobs' memory forces queueing and admission control
    srv = tb.Server(mem_budget_bytes=64 << 20, max_inflight=4)
    try:
        prob, p, T, G, H, cap = reqs[2]
        o = tb.host_outputs(prob, cap)
        st, lat = srv.wait(srv.submit(prob, p, T, G, H, o))
        assert st == tb.TBLR_OK
        alone = {k: o[k].numpy().copy() for k in ("u", "v", "at", "ranks")}
        outs = []
        tickets = []
        for prob, p, T, G, H, cap in reqs + reqs:       # every request twice, concurrently
            o = tb.host_outputs(prob, cap)
            outs.append(o)
            tickets.append(srv.submit(prob, p, T, G, H, o))
        for t in tickets:
            st, lat = srv.wait(t)
            assert st == tb.TBLR_OK and lat > 0
        for idx, o in enumerate(outs):
            ref = singles[idx % len(JOBS)]
            for key in ("u", "v", "at", "ranks"):
                assert np.array_equal(o[key].numpy(), ref[key]), key
            assert np.array_equal(o["bnear"].numpy()[:len(ref["bnear"])], ref["bnear"])
        for key in alone:
            assert np.array_equal(alone[key], outs[2][key].numpy())
        stats = srv.stats()
        assert stats["completed"] == 1 + 2 * len(JOBS) and stats["failed"] == 0
        assert 0 < stats["p50_ms"] <= stats["p99_ms"]
        assert stats["mem_in_use"] == 0 and stats["mem_peak"] > 0
    finally:
        srv.close()
    assert tb.tblr_device_timeouts() == 0


def test_server_reports_a_too_small_output_buffer():
    tb = _tb()
    prob, pts, T, G, H = _make(JOBS[0])
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
    srv = tb.Server(mem_budget_bytes=1 << 30, max_inflight=2)
    try:
        o = tb.host_outputs(prob, 10)
        st, _ = srv.wait(srv.submit(prob, pin(pts), pin(T), pin(G), pin(H), o))
        assert st == tb.TBLR_EWORKSPACE
    finally:
        srv.close()
