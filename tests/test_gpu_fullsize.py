"""Parity at the benchmark's full sizes, in the configuration bench.py times.

The whole compression runs through the C ABI at N = 65,536 (2-D, FP64, black-box
sketch: the default benchmark line) and N = 262,144 (3-D, mixed precision,
tag-factored sketch).  The oracle cannot form these problems, so it computes a
sample one block at a time: the sketch rows, samples and bases of a few boxes far
apart and the coupling blocks among them (the same routine as the benchmark's CPU
baseline), and the far-field blocks U_i Atilde_ij V_j^T are compared with the
GPU's.  Index lists are compared bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(workload, precision, sketch, boxes, bound):
    import bench
    from paper_2501_05528_gb300 import tblr as tb
    w = dict(bench.WORKLOADS[workload])
    pts, T, G, H = bench.make_inputs(w, 0)
    d = w["d"]
    prob = tb.make_problem(d, w["kernel"], w["n"], w["grid"], (0.0,) * d, (1.0,) * d, w["k"],
                           w["p"], w["e"], precision=precision, sketch=sketch)
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    out = tb.compress(prob, t(pts), t(T), t(G), t(H))
    torch.cuda.synchronize()
    assert tb.tblr_device_timeouts() == 0
    gpu = dict(u=out.u.cpu().numpy(), v=out.v.cpu().numpy(), at=out.at.cpu().numpy())
    sample_ids = bench.sample_boxes(w["grid"], boxes)
    secs, frac, sample = bench.oracle_sample(w, pts, T, G, H, sample_ids)
    tess = sample["tess"]
    assert np.array_equal(out.layout.perm.cpu().numpy(), tess["perm"])
    assert np.array_equal(out.layout.offsets.cpu().numpy(), tess["offsets"])
    far_pairs = [(i, j) for (i, j) in sample["blocks"] if j not in tess["nbrs"][i]]
    assert len(far_pairs) >= 2
    err = bench.compare_sample(sample, gpu)
    print(f"{workload} precision={precision}: sampled far blocks vs oracle {err:.3e} "
          f"({len(far_pairs)} blocks, oracle {secs:.1f} s)")
    assert err <= bound, err


def test_laplace2d_n65536_fp64_blackbox_full_size():
    from paper_2501_05528_gb300 import tblr as tb
    _run("laplace2d_n65536", tb.FP64, tb.SKETCH_BLACKBOX, 4, 1e-10)


def test_laplace3d_n262144_mixed_tagged_full_size():
    from paper_2501_05528_gb300 import tblr as tb
    _run("laplace3d_n262144", tb.MIXED, tb.SKETCH_TAGGED, 2, 1e-6)
