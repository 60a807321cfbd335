"""Benchmark: tagged uniform-BLR compressions per second on one GB300 (or N, weak scaling).

One step = one full reconstruct_tag (Table 1) of the workload through the C ABI:
tessellation, near-field offsets, test matrices, sketch, tag decode, combine,
col (U and V), coupling and near field.  Inputs (points, T, G, H) are resident
in HBM before timing; L2 is flushed (a 256 MiB write) before every step.

Also reported:
  e2e          the same metric through tblr_compress_host (host buffers,
               host<->device copies inside the timed region);
  roofline     the sketch kernel (the dominant one) timed with CUDA events on
               its stream inside the timed steps, against the FP64 pipe peak;
  cpu_baseline the CPU oracle timed on this host on a bounded sample of the
               same workload, also used to check the GPU result's accuracy;
  clocks       nvidia-smi samples taken during the timed region.

``--impl reference`` times the CPU oracle alone (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tagged-BLR compressions/s at rel.err≤1e-6 vs FP64; p50/p99 latency; % roofline"
UNIT = "compressions/s"
FP64_PEAK_TFLOPS = 1.26   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")

WORKLOADS = {
    # 2D Laplace, N = 65,536 i.i.d. uniform points, 16 x 16 boxes (~256 per box), k = 32, FP64
    "laplace2d_n65536": dict(d=2, n=65536, grid=(16, 16), k=32, p=10, e=3, kernel="laplace2d",
                             seed=0x7A660002),
    # same recipe, 16,384 points on 8 x 8 boxes: the small case used for ncu captures
    "laplace2d_n16384": dict(d=2, n=16384, grid=(8, 8), k=32, p=10, e=3, kernel="laplace2d",
                             seed=0x7A660012),
    # 3D Laplace, jittered 64^3 lattice (jitter U[-h/4, h/4]), 8 x 8 x 8 boxes of 512 points,
    # k = 64; run with --precision mixed
    "laplace3d_n262144": dict(d=3, n=262144, grid=(8, 8, 8), k=64, p=10, e=3, kernel="laplace3d",
                              seed=0x7A660003, lattice=64, cpu_boxes=2),
    # same recipe on a 32^3 lattice, 4 x 4 x 4 boxes of 512 points
    "laplace3d_n32768": dict(d=3, n=32768, grid=(4, 4, 4), k=64, p=10, e=3, kernel="laplace3d",
                             seed=0x7A660013, lattice=32, cpu_boxes=2),
}


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def reduce_max(value, world, device="cpu"):
    """Max of a per-rank scalar over all ranks (the slowest rank sets the time)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(steps, world, seconds):
    """Whole-job throughput: every rank ran `steps` independent compressions."""
    return steps * world / seconds


def make_inputs(w, rank=0):
    from paper_2501_05528_gb300 import inputs
    d = w["d"]
    if "lattice" in w:
        pts = inputs.jittered_lattice(w["lattice"], d, 0.25, seed=w["seed"] + 7919 * rank)
    else:
        pts = inputs.uniform_points(w["n"], d, seed=w["seed"] + 7919 * rank)
    b = int(np.prod(w["grid"]))
    ell = 3 ** d + 1 + w["e"]
    T, G, H = inputs.tagging_draws(b, ell, w["n"], w["k"] + w["p"], seed=w["seed"] + 1 + 7919 * rank)
    if w.get("selfadjoint"):
        H = G  # Psi = Omega: the self-adjoint mode's R = S
    return pts, T, G, H



def launches_per_compression(mixed, tagged, selfadjoint=False):
    """Kernel launches of the library for one compression: tessellate 4, near-field offsets 2,
    col 2 (1 self-adjoint), coupling 1, near field 2, decode 1; mixed precision adds the
    coupling's 4 operand passes (box-padded offsets, staged coordinates, V planes, U rows) and
    the near field's 2 conversions (coordinates, V^T); then either test matrices + sketch +
    combine (3; mixed 5 with staged coordinates and X planes) or the tagged sketch (FP64: gather
    + sketch; mixed: staged coordinates, [G|H] planes, tau, sketch)."""
    base = 4 + 2 + (1 if selfadjoint else 2) + 1 + 2 + 1 + (4 + 2 if mixed else 0)
    return base + ((4 if mixed else 2) if tagged else (5 if mixed else 3))

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ----------------------------------------------------------- CPU oracle sample

def oracle_sample(w, pts, T, G, H, boxes):
    """The CPU oracle on a bounded sample: sketch rows, combine and col for `boxes`,
    and the coupling blocks among them.  Returns (seconds, fraction of one
    compression the sample stands for, per-box results)."""
    from oracle import tagging as orc
    t0 = time.perf_counter()
    d = w["d"]
    tess = orc.tessellate(pts, w["grid"], (0.0,) * d, (1.0,) * d)
    op = orc.make_operator(w["kernel"], pts, tess)
    r = w["k"] + w["p"]
    Om = orc.extended_test_matrix(T, G, tess)
    Ps = orc.extended_test_matrix(T, H, tess)
    z, tau, rho = orc.decode(T, tess)
    off = tess["offsets"]
    ks = orc.box_ranks(tess, w["k"])
    U, V = {}, {}
    for i in boxes:
        rows = np.arange(off[i], off[i + 1])
        Y = orc.sketch_rows(op, Om, rows)
        Z = orc.sketch_rows(op, Ps, rows)
        S = sum(z[i, j] * Y[:, j * r:(j + 1) * r] for j in range(T.shape[1]))
        R = sum(z[i, j] * Z[:, j * r:(j + 1) * r] for j in range(T.shape[1]))
        U[i] = orc.col(S, ks[i])
        V[i] = orc.col(R, ks[i])
    blocks = {}
    for i in boxes:
        for j in boxes:
            Ri = np.arange(off[i], off[i + 1])
            Cj = np.arange(off[j], off[j + 1])
            At = U[i].T @ op.block(Ri, Cj) @ V[j]
            blocks[(i, j)] = U[i] @ At @ V[j].T
    secs = time.perf_counter() - t0
    b = len(off) - 1
    return secs, len(boxes) / b, dict(tess=tess, U=U, V=V, blocks=blocks, ranks=ks)


def sample_boxes(grid, count):
    b = int(np.prod(grid))
    step = max(1, b // count)
    return list(range(step // 2, b, step))[:count]


def compare_sample(sample, gpu):
    """Relative Frobenius difference of the sampled far-field reconstructed blocks
    U_i Atilde_ij V_j^T, GPU against oracle.  (Near pairs are left out: there
    only U Atilde V^T + B is determined, and the sample has no B.)"""
    off = sample["tess"]["offsets"]
    nbrs = sample["tess"]["nbrs"]
    num = den = 0.0
    for (i, j), ref in sample["blocks"].items():
        if j in nbrs[i]:
            continue
        ki, kj = int(sample["ranks"][i]), int(sample["ranks"][j])
        Ui = gpu["u"][off[i]:off[i + 1], :ki]
        Vj = gpu["v"][off[j]:off[j + 1], :kj]
        blk = Ui @ gpu["at"][i, j][:ki, :kj] @ Vj.T
        num += np.sum((blk - ref) ** 2)
        den += np.sum(ref ** 2)
    return math.sqrt(num / den) if den > 0 else float("nan")


# ------------------------------------------------------------------ GPU arm

class Runner:
    """Preallocated buffers and the step chain of one compression (C-ABI calls)."""

    def __init__(self, tb, torch, w, pts, T, G, H):
        self.tb, self.torch = tb, torch
        dev = torch.device("cuda", torch.cuda.current_device())
        t = lambda a: torch.as_tensor(a, device=dev)
        self.pts, self.T, self.G, self.H = t(pts), t(T), t(G), t(H)
        d = w["d"]
        self.tagged = w.get("sketch", 0) == 1
        self.selfadjoint = bool(w.get("selfadjoint"))
        self.prob = tb.make_problem(d, w["kernel"], w["n"], w["grid"], (0.0,) * d, (1.0,) * d,
                                    w["k"], w["p"], w["e"], precision=w.get("precision", 0),
                                    sketch=w.get("sketch", 0), selfadjoint=self.selfadjoint,
                                    zrule=w.get("zrule", 0))
        self.sz = tb.tblr_sizes_of(self.prob)
        lay = tb.tblr_tessellate(self.prob, self.pts)
        nf_off, m_max = tb.tblr_nearfield_offsets(self.prob, lay)
        torch.cuda.synchronize()
        self.m_max = int(m_max.item())
        self.total = int(nf_off[-1].item())
        self.out = tb.tblr_compress(self.prob, lay, self.T, self.G, self.H,
                                    nf=(nf_off, self.m_max, self.total))
        self.lay = lay
        n, sz = w["n"], self.sz
        f64 = dict(dtype=torch.float64, device=dev)
        self.omega = torch.empty(sz.sketch_cols * n, **f64)
        self.S = torch.empty(n, sz.r, **f64)
        self.R = torch.empty(n, sz.r, **f64)
        self.tws = torch.empty(tb.lib().tblr_tessellate_workspace(tb.ctypes.byref(self.prob)),
                               dtype=torch.uint8, device=dev)
        self.colws = torch.empty(tb.lib().tblr_col_workspace(tb.ctypes.byref(self.prob)),
                                 dtype=torch.uint8, device=dev)
        skb = (tb.lib().tblr_tagged_sketch_workspace if self.tagged else
               tb.lib().tblr_sketch_workspace)(tb.ctypes.byref(self.prob))
        self.skws = torch.empty(max(1, skb), dtype=torch.uint8, device=dev)
        self.cplws = torch.empty(max(1, tb.lib().tblr_coupling_workspace(tb.ctypes.byref(self.prob))),
                                 dtype=torch.uint8, device=dev)
        self.nfws = torch.empty(tb.lib().tblr_nearfield_workspace(tb.ctypes.byref(self.prob),
                                                                  self.m_max),
                                dtype=torch.uint8, device=dev)
        self.mmax_dev = torch.empty(1, dtype=torch.int32, device=dev)
        self.host_total = torch.empty(1, dtype=torch.int64).pin_memory()
        self.host_mmax = torch.empty(1, dtype=torch.int32).pin_memory()
        self.launches_per_step = launches_per_compression(
            w.get("precision", 0) == 1, self.tagged, self.selfadjoint)

    def step(self, ev=None):
        tb, L, P, o = self.tb, self.tb.lib(), self.tb.ctypes.byref(self.prob), self.out
        p, s = self.tb._p, self.tb._stream()
        ck = self.tb._check
        lay = self.lay
        ck(L.tblr_tessellate(P, p(self.pts), lay.ref, p(self.tws), self.tws.numel(), s), "tess")
        ck(L.tblr_nearfield_offsets(P, lay.ref, p(o.nf_off), p(self.mmax_dev), s), "nf_off")
        # sizes of this step's near-field output, read back as a user would
        self.host_total.copy_(o.nf_off[-1:], non_blocking=True)
        self.host_mmax.copy_(self.mmax_dev, non_blocking=True)
        self.torch.cuda.current_stream().synchronize()
        total, m_max = int(self.host_total[0]), int(self.host_mmax[0])
        assert total == self.total and m_max == self.m_max
        if self.tagged:
            ck(L.tblr_decode(P, lay.ref, p(self.T), p(o.z), p(o.tau), p(o.rho), s), "decode")
            if ev is not None:
                ev[0].record()
            ck(L.tblr_tagged_sketch(P, lay.ref, None, p(o.tau), p(self.G), p(self.H), p(self.S),
                                    p(self.R), p(self.skws), self.skws.numel(), s), "tagged")
            if ev is not None:
                ev[1].record()
        else:
            ck(L.tblr_test_matrices(P, lay.ref, p(self.T), p(self.G), p(self.H), p(self.omega), s),
               "tm")
            if ev is not None:
                ev[0].record()
            ck(L.tblr_sketch(P, lay.ref, None, p(self.omega), p(o.yz), p(self.skws),
                             self.skws.numel(), s), "sketch")
            if ev is not None:
                ev[1].record()
            ck(L.tblr_decode(P, lay.ref, p(self.T), p(o.z), p(o.tau), p(o.rho), s), "decode")
            ck(L.tblr_combine(P, lay.ref, p(o.yz), p(o.z), p(self.S), p(self.R), s), "combine")
        ck(L.tblr_col(P, lay.ref, p(self.S), p(o.u), p(o.ranks), p(self.colws), self.colws.numel(),
                      s), "col U")
        if self.selfadjoint:
            o.v.copy_(o.u)  # R = S, so V = U (a device copy, no kernel)
        else:
            ck(L.tblr_col(P, lay.ref, p(self.R), p(o.v), p(o.ranks), p(self.colws),
                          self.colws.numel(), s), "col V")
        ck(L.tblr_coupling(P, lay.ref, None, p(o.u), p(o.v), p(o.ranks), m_max, p(o.at),
                           p(self.cplws), self.cplws.numel(), s), "coupling")
        ck(L.tblr_nearfield(P, lay.ref, None, p(o.u), p(o.at), p(o.v), p(o.ranks), p(o.nf_off),
                            m_max, p(o.bnear), p(self.nfws), self.nfws.numel(), s), "nearfield")


def measured_peak(key, fallback):
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


# DRAM bytes of one sketch launch, per (kernel, workload), from one 1-pass ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel as it stands; kept in sync with
# the kernel (remove the entry when the kernel changes).
SKETCH_TRAFFIC = {("fp64-blackbox", "laplace2d_n65536"): 24849398272 + 623482880}


def padded_cols(ncols, tagged):
    """Columns the tensor-core sketch computes for `ncols` outputs: the fewest tiles of at
    most 160 columns, of equal width rounded up to 32 (128 or 160 for the black-box apply)."""
    ntiles = -(-max(ncols, 1) // 160)
    width = -(-(-(-max(ncols, 1) // ntiles)) // 32) * 32
    if not tagged:
        width = 128 if width <= 128 else 160
    return width * ntiles


def roofline(w, achieved, sketch_ms, traffic, tagged=False, ncols=None):
    """Roofline of the sketch kernel: FP64 pipe for the FP64 path, BF16 tensor pipe for
    the mixed path, where each algorithmic multiply-add costs 6 split BF16 products on
    tile-padded columns.  The tagged sketch's algorithmic work is 2 n^2 (2 r) instead of
    2 n^2 (2 ell r)."""
    if w.get("precision", 0) == 0:
        return {"bound": "alu", "kernel": "apply_fp64_kernel (sketch)" + (", tagged" if tagged else ""),
                "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": traffic, "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2.07 GHz",
                "sketch_ms": sketch_ms}
    peak, src = measured_peak("bf16_tflops", 1900.0)
    factor = 6.0 * (padded_cols(ncols, tagged) / ncols if ncols else 1.0)
    return {"bound": "tensor", "kernel": "mixed_apply_kernel (sketch)" + (", tagged" if tagged else ""),
            "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "peak_source": f"{src} dense bf16 burst",
            "executed_tflops": factor * achieved, "executed_frac": factor * achieved / peak,
            "sketch_ms": sketch_ms}


def mixed_vs_fp64(tb, torch, w, run):
    """Full-matrix relative Frobenius difference between the mixed-precision result
    and the FP64 GPU result on the same inputs (the FP64 path matches the CPU
    oracle to 1e-10 in the parity tests), computed on the host."""
    from paper_2501_05528_gb300 import metrics
    d = w["d"]
    prob64 = tb.make_problem(d, w["kernel"], w["n"], w["grid"], (0.0,) * d, (1.0,) * d, w["k"],
                             w["p"], w["e"], precision=tb.FP64, sketch=tb.SKETCH_TAGGED,
                             selfadjoint=bool(w.get("selfadjoint")), zrule=w.get("zrule", 0))
    ref = tb.compress(prob64, run.pts, run.T, run.G, run.H)
    torch.cuda.synchronize()
    h = lambda t: t.cpu().numpy()
    off, nbr, nnbr = h(run.lay.offsets), h(run.lay.nbr), h(run.lay.nnbr)
    s3 = run.sz.s3
    reps = []
    for o in (run.out, ref):
        B = metrics.blocks_from_flat(h(o.bnear), h(o.nf_off), nbr, nnbr, off, s3)
        reps.append(dict(U=h(o.u), V=h(o.v), At=h(o.at), B=B))
    err = metrics.ublr_difference_all(off, nbr, nnbr, s3, h(run.out.ranks), reps[0], reps[1])
    return {"relerr_vs_fp64": err, "bound": 1e-6, "within_bound": bool(err <= 1e-6),
            "reference": "FP64 GPU path (tag-factored, equal to the black-box FP64 result to "
                         "1e-10) on the same inputs, full matrix, Frobenius"}


def run_gpu(args, w):
    import torch
    import torch.distributed as dist
    from paper_2501_05528_gb300 import tblr as tb

    rank, local, world = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://", rank=rank, world_size=world,
                                device_id=torch.device("cuda", local))
    tb.lib()
    pts, T, G, H = make_inputs(w, rank)
    run = Runner(tb, torch, w, pts, T, G, H)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        flush.fill_(1)
        run.step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    stp = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier()
    with sampler:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for i in range(args.steps):
            flush.fill_(1)
            stp[i][0].record()
            run.step(evs[i])
            stp[i][1].record()
        t1.record()
        barrier()
    total_ms = t0.elapsed_time(t1)
    step_ms = [a.elapsed_time(b) for a, b in stp]
    sketch_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = reduce_max(total_ms, world, "cuda")
    value = weak_value(args.steps, world, total_ms / 1e3)

    # end to end through the host-buffer entry point (pinned host memory)
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
    hp, hT, hG, hH = pin(pts), pin(T), pin(G), pin(H)
    sz = run.sz
    n, b, k, s3 = w["n"], sz.b, w["k"], sz.s3
    outs = dict(perm=torch.empty(n, dtype=torch.int32).pin_memory(),
                offsets=torch.empty(b + 1, dtype=torch.int32).pin_memory(),
                nbr=torch.empty(b * s3, dtype=torch.int32).pin_memory(),
                ranks=torch.empty(b, dtype=torch.int32).pin_memory(),
                u=torch.empty(n, k, dtype=torch.float64).pin_memory(),
                v=torch.empty(n, k, dtype=torch.float64).pin_memory(),
                at=torch.empty(b, b, k, k, dtype=torch.float64).pin_memory(),
                bnear=torch.empty(run.total, dtype=torch.float64).pin_memory())
    tb.tblr_compress_host(run.prob, hp, hT, hG, hH, outputs=outs)   # warm-up (sizes the cache)
    h2d = sum(x.numel() * x.element_size() for x in (hp, hT, hG, hH))
    d2h = sum(outs[kk].numel() * outs[kk].element_size() for kk in outs if kk != "bnear_size")
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        flush.fill_(1)
        tb.tblr_compress_host(run.prob, hp, hT, hG, hH, outputs=outs)
    barrier()
    te = time.perf_counter() - te
    e2e_value = weak_value(e2e_steps, world, reduce_max(te, world, "cuda"))

    accuracy = None
    if rank == 0 and w.get("precision", 0) == 1 and not args.no_fp64_check:
        accuracy = mixed_vs_fp64(tb, torch, w, run)

    result = None
    if rank == 0:
        cols = (1 if run.selfadjoint else 2) * sz.r if run.tagged else sz.sketch_cols
        flops = 2.0 * w["n"] * w["n"] * cols
        sk = statistics.mean(sketch_ms) / 1e3
        achieved = flops / sk / 1e12
        gpu_res = dict(u=run.out.u.cpu().numpy(), v=run.out.v.cpu().numpy(),
                       at=run.out.at.cpu().numpy())
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            boxes = sample_boxes(w["grid"], w.get("cpu_boxes", args.cpu_sample_boxes))
            secs, frac, sample = oracle_sample(w, pts, T, G, H, boxes)
            relerr = compare_sample(sample, gpu_res)
            cpu = {"value": frac / secs, "unit": UNIT, "cores": len(os.sched_getaffinity(0)),
                   "kind": "oracle",
                   "sample": (f"oracle sketch rows, combine and col for {len(boxes)} of "
                              f"{sz.b} boxes plus their {len(boxes)**2} coupling blocks, "
                              f"{secs:.1f} s, scaled by boxes/{len(boxes)}; numpy BLAS threads "
                              f"on all cores, elementwise ops on one"),
                   "gpu_relerr_vs_oracle_sampled": relerr}
        lat = sorted(step_ms)
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if w.get("precision", 0) == 0 else "bf16x3+f32/f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "N": w["n"], "d": w["d"],
                       "grid": list(w["grid"]), "k": w["k"], "p": w["p"], "e": w["e"],
                       "ell": sz.ell, "sketch_cols": sz.sketch_cols, "kernel": w["kernel"],
                       "precision": "fp64" if w.get("precision", 0) == 0 else "mixed",
                       "sketch": ("tagged, self-adjoint (H = G, V = U)" if run.selfadjoint else
                                  "tagged") if run.tagged else "blackbox",
                       "zrule": "minratio (§5.3 LP)" if w.get("zrule") else "project",
                       "l2": "flushed by a 256 MiB write before every step",
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": run.launches_per_step * args.steps,
            "roofline": roofline(w, achieved, statistics.mean(sketch_ms),
                                 args.traffic if args.traffic is not None else SKETCH_TRAFFIC.get(
                                     ("fp64-blackbox" if w.get("precision", 0) == 0 and
                                      not run.tagged else "other", args.workload)),
                                 tagged=run.tagged, ncols=cols),
            "cpu_baseline": cpu,
            "clocks": sampler.summary(),
        }
        if accuracy is not None:
            result["accuracy"] = accuracy
        rho = run.out.rho.cpu().numpy()
        rho = rho[np.isfinite(rho)]
        if rho.size:  # eq. aspect_ratio over the boxes (§5.1; minimised with --zrule minratio)
            result["aspect_ratio"] = {"median": float(np.median(rho)), "p90": float(np.percentile(rho, 90)),
                                      "max": float(rho.max())}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return result


def run_reference(args, w):
    rank, _, world = env_rank()
    if rank != 0:
        return None
    pts, T, G, H = make_inputs(w, 0)
    boxes = sample_boxes(w["grid"], w.get("cpu_boxes", args.cpu_sample_boxes))
    for _ in range(args.warmup):
        oracle_sample(w, pts, T, G, H, boxes)
    times = []
    frac = None
    for _ in range(args.steps):
        secs, frac, _ = oracle_sample(w, pts, T, G, H, boxes)
        times.append(secs)
    value = frac / statistics.mean(times)
    cores = len(os.sched_getaffinity(0))
    sample = (f"oracle sketch rows, combine and col for {len(boxes)} boxes and their coupling "
              f"blocks per step, scaled by boxes/{len(boxes)}")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "N": w["n"], "d": w["d"],
                       "grid": list(w["grid"]), "k": w["k"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample}}


# ------------------------------------------------------- batched and served

def batch_specs(count, seed):
    """Independent 2-D/3-D Laplace problems: N ~ U{4096..65536}, box size in {128, 256, 512},
    k in {16, 32, 64}, points uniform in the unit square or cube, grid side
    max(3, round((N / box)^(1/d)))."""
    rng = np.random.default_rng(seed)
    specs = []
    for j in range(count):
        d = int(rng.choice([2, 3]))
        n = int(rng.integers(4096, 65537))
        box = int(rng.choice([128, 256, 512]))
        k = int(rng.choice([16, 32, 64]))
        side = max(3, int(round((n / box) ** (1.0 / d))))
        specs.append(dict(d=d, n=n, grid=(side,) * d, k=k, p=10, e=3,
                          kernel="laplace2d" if d == 2 else "laplace3d", seed=seed + 1000 + j))
    return specs


def spec_inputs(s):
    from paper_2501_05528_gb300 import inputs
    pts = inputs.uniform_points(s["n"], s["d"], seed=s["seed"])
    b = int(np.prod(s["grid"]))
    T, G, H = inputs.tagging_draws(b, 3 ** s["d"] + 1 + s["e"], s["n"], s["k"] + s["p"],
                                   seed=s["seed"] + 1)
    return pts, T, G, H


def spec_problem(tb, s, precision, sketch):
    d = s["d"]
    return tb.make_problem(d, s["kernel"], s["n"], s["grid"], (0.0,) * d, (1.0,) * d, s["k"],
                           s["p"], s["e"], precision=precision, sketch=sketch)


def run_batch(args):
    """Config 4: the whole batch of independent jobs replayed as one CUDA graph per step."""
    import torch
    from paper_2501_05528_gb300 import tblr as tb
    torch.cuda.set_device(0)
    prec = 1 if args.precision == "mixed" else 0
    sk = 1 if args.sketch == "tagged" else 0
    specs = batch_specs(args.jobs, 0x7A660004)
    dev = torch.device("cuda")
    jobs = []
    for s in specs:
        pts, T, G, H = spec_inputs(s)
        t = lambda a: torch.as_tensor(a, device=dev)
        jobs.append(tb.BatchJob(spec_problem(tb, s, prec, sk), t(pts), t(T), t(G), t(H)))
    tb.tblr_batch_plan(jobs)
    # Autotuner: the tensor-core sketch's tile width, once per size class (kernel, sketch
    # columns, floor(log2 N)), timed on the class's first job before the graph is captured.
    tuned = {}
    if prec == 1 and sk == 1:
        for job in jobs:
            if tb.tblr_tuned_width(job.prob):
                continue
            _, tau, _ = tb.tblr_decode(job.prob, job.lay, job.T)
            w, _, _ = tb.tblr_tune_tagged_sketch(job.prob, job.lay, tau, job.G, job.H)
            tuned[f"kernel{job.prob.kernel}_cols{2 * (job.prob.k + job.prob.p)}_log2n"
                  f"{job.prob.n.bit_length() - 1}"] = w
        torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        graph = tb.Graph(jobs, n_streams=8)
        for _ in range(args.warmup):
            graph.launch()
        stream.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(0)
        with sampler:
            t0.record()
            for _ in range(args.steps):
                graph.launch()
            t1.record()
            stream.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    assert tb.tblr_device_timeouts() == 0
    return {"metric": METRIC, "value": args.jobs / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == 0 else "bf16x3+f32/f64", "data": "synthetic",
            "config": {"workload": f"batch of {args.jobs} independent 2-D/3-D Laplace jobs",
                       "N": "U{4096..65536}", "box": "{128,256,512}", "k": "{16,32,64}",
                       "precision": args.precision, "sketch": args.sketch,
                       "execution": "one CUDA graph per step, 8 worker streams",
                       "autotuned_tile_widths": tuned,
                       "l2": "per-step working set tens of GB, far above L2"},
            "gpu_launches": len(jobs) * launches_per_compression(prec == 1, sk == 1) * args.steps,
            "clocks": sampler.summary(), "cpu_baseline": None}


def run_serve(args):
    """Config 5 (kernel operators): a seeded Poisson stream of requests of the sizes of
    configs 1-3 through the continuous-batching server; p50/p99 latency and throughput."""
    import torch
    from paper_2501_05528_gb300 import tblr as tb
    torch.cuda.set_device(0)
    prec = 1 if args.precision == "mixed" else 0
    sk = 1 if args.sketch == "tagged" else 0
    shapes = [  # config 1 geometry, config 2, a config-3-shaped 3-D job at 1/8 of its size
        dict(d=2, n=1024, grid=(4, 4), k=8, p=10, e=3, kernel="laplace2d", seed=11),
        dict(d=2, n=65536, grid=(16, 16), k=32, p=10, e=3, kernel="laplace2d", seed=12),
        dict(d=3, n=32768, grid=(4, 4, 4), k=64, p=10, e=3, kernel="laplace3d", seed=13),
    ]
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
    prepared = []
    for s in shapes:
        prob = spec_problem(tb, s, prec, sk)
        pts, T, G, H = (pin(x) for x in spec_inputs(s))
        warm = tb.tblr_compress_host(prob, pts, T, G, H)
        prepared.append((prob, pts, T, G, H, warm["bnear_size"]))
    rng = np.random.default_rng(0x7A660005)
    kinds = rng.integers(0, len(shapes), size=args.requests)
    gaps = rng.exponential(1.0 / args.rate, size=args.requests)
    # Output buffers are pooled per request kind (8 sets, one per stream slot) since the
    # benchmark does not read the results; each request's buffers stay valid until it ends.
    pools = [[tb.host_outputs(p[0], p[5]) for _ in range(8)] for p in prepared]
    outs = [pools[k][i % 8] for i, k in enumerate(kinds)]
    free = torch.cuda.mem_get_info()[0]
    srv = tb.Server(mem_budget_bytes=int(0.6 * free), max_inflight=8)
    tickets = []
    t0 = time.perf_counter()
    t_next = t0
    for i, k in enumerate(kinds):
        t_next += gaps[i]
        delay = t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        prob, pts, T, G, H, _ = prepared[k]
        tickets.append(srv.submit(prob, pts, T, G, H, outs[i]))
    lat = []
    for t in tickets:
        st, l = srv.wait(t)
        assert st == tb.TBLR_OK
        lat.append(l)
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    lat.sort()
    return {"metric": METRIC, "value": args.requests / wall, "unit": UNIT, "n_gpus": 1,
            "steps": args.requests, "warmup": len(shapes), "ms_per_step": 1e3 * wall / args.requests,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == 0 else "bf16x3+f32/f64", "data": "synthetic",
            "config": {"workload": "Poisson request stream, kernel operators, sizes of configs 1-3",
                       "rate_req_s": args.rate, "requests": args.requests,
                       "mix": "uniform over {N=1,024 2-D k=8; N=65,536 2-D k=32; N=32,768 3-D k=64}",
                       "precision": args.precision, "sketch": args.sketch,
                       "server": "8 stream slots, budget 60% of free HBM, host buffers pinned"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "server_stats": {k: stats[k] for k in ("completed", "failed", "mem_peak", "throughput")},
            "gpu_launches": args.requests * launches_per_compression(prec == 1, sk == 1),
            "cpu_baseline": None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="laplace2d_n65536", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-sample-boxes", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-check", action="store_true",
                    help="skip the mixed-vs-FP64 accuracy check of the mixed path")
    ap.add_argument("--zrule", default="project", choices=["project", "minratio"],
                    help="null vector of each box: projection (default) or the §5.3 aspect-ratio LP")
    ap.add_argument("--selfadjoint", action="store_true",
                    help="self-adjoint mode (A = A^T, H = G): V = U, half the coupling")
    ap.add_argument("--sketch", default="blackbox", choices=["blackbox", "tagged"],
                    help="black-box sketch Y = A Omega (the paper's order) or the tag-factored S, R")
    ap.add_argument("--mode", default="single", choices=["single", "batch", "serve"],
                    help="single compressions, a 64-job batch (one CUDA graph), or a request stream")
    ap.add_argument("--jobs", type=int, default=64)
    ap.add_argument("--rate", type=float, default=200.0, help="serve: Poisson arrival rate, req/s")
    ap.add_argument("--requests", type=int, default=200, help="serve: number of requests")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="sketch contraction precision (everything else stays FP64)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per sketch launch from an ncu capture, if current")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    w["precision"] = 1 if args.precision == "mixed" else 0
    w["sketch"] = 1 if args.sketch == "tagged" else 0
    w["zrule"] = 1 if args.zrule == "minratio" else 0
    if args.selfadjoint:
        if w["sketch"] != 1:
            raise SystemExit("--selfadjoint needs --sketch tagged")
        w["selfadjoint"] = True
    if args.impl == "reference":
        res = run_reference(args, w)
    elif args.mode == "batch":
        res = run_batch(args)
    elif args.mode == "serve":
        res = run_serve(args)
    else:
        res = run_gpu(args, w)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
