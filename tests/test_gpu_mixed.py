"""GPU parity of the mixed-precision (tcgen05, three-part BF16, FP32 accumulation) path.

Bound: the split-precision apply and the whole compression built on it must
match the FP64 oracle within 1e-6 relative Frobenius error (the stated bound
for the mixed path).  Each operand is carried as three BF16 parts (2^-24
relative), the dropped products are <= 2^-24, FP32 kernel entries are within
~1 ulp, and the FP32 tensor-core accumulation is flushed every 64 points into
compensated sums, so a sketch is expected near 1e-7.  Cases have ragged row
and column tails and cover every tile width of the tensor-core kernel.
"""
import numpy as np
import pytest

from oracle import tagging as orc
from paper_2501_05528_gb300 import inputs
from paper_2501_05528_gb300 import metrics

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MIXED_BOUND = 1e-6


def _tb():
    from paper_2501_05528_gb300 import tblr
    return tblr


APPLY_CASES = [
    ("laplace2d", 2, (6, 6), 3001, 468),
    ("laplace3d", 3, (4, 4, 4), 2501, 200),
    ("laplace2d", 2, (3, 3), 130, 16),
]


@pytest.mark.parametrize("kind,d,grid,n,ncols", APPLY_CASES)
def test_mixed_apply_matches_fp64_oracle(kind, d, grid, n, ncols):
    tb = _tb()
    pts = inputs.uniform_points(n, d, seed=n)
    X = np.random.default_rng(n + 1).standard_normal((n, ncols))
    prob = tb.make_problem(d, kind, n, grid, (0.0,) * d, (1.0,) * d, 4, 10, 0)
    dev = torch.device("cuda")
    lay = tb.tblr_tessellate(prob, torch.as_tensor(pts, device=dev))
    perm = lay.perm.cpu().numpy()
    xt = torch.as_tensor(np.ascontiguousarray(X[perm].T), device=dev)   # K-major, box-major rows
    y_mixed = tb.tblr_apply(prob, lay, xt, ncols, precision=tb.MIXED).cpu().numpy()
    assert tb.tblr_device_timeouts() == 0
    y_fp64 = tb.tblr_apply(prob, lay, xt, ncols, precision=tb.FP64).cpu().numpy()
    op = orc.KernelOperator(kind, pts[perm])
    ref = op.apply(X[perm])
    err = metrics.rel(y_mixed, ref)
    print(f"mixed apply {kind} n={n} ncols={ncols}: rel err {err:.3e}")
    assert err < MIXED_BOUND
    assert metrics.rel(y_fp64, ref) < 1e-12
    # every row and column (including the ragged tails) is accurate
    row_err = np.linalg.norm(y_mixed - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert row_err.max() < 10 * MIXED_BOUND


@pytest.mark.parametrize("sketch", [0, 1], ids=["blackbox", "tagged"])
@pytest.mark.parametrize("kind,d,grid,n,k,e", [("laplace2d", 2, (6, 6), 3001, 8, 3),
                                              ("laplace3d", 3, (4, 4, 4), 2501, 6, 1),
                                              ("laplace3d", 3, (5, 5, 5), 6001, 12, 3)])
def test_mixed_compression_within_bound(kind, d, grid, n, k, e, sketch):
    tb = _tb()
    pts = inputs.uniform_points(n, d, seed=7 * n)
    b = int(np.prod(grid))
    ell = orc.tag_columns(d, e)
    T, G, H = inputs.tagging_draws(b, ell, n, k + 10, seed=7 * n + 1)
    lo, hi = (0.0,) * d, (1.0,) * d
    ref = orc.reconstruct_tag(pts, grid, lo, hi, kind, T, G, H, k, 10)
    prob = tb.make_problem(d, kind, n, grid, lo, hi, k, 10, e, precision=tb.MIXED, sketch=sketch)
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(a, device=dev)
    out = tb.compress(prob, t(pts), t(T), t(G), t(H))
    assert tb.tblr_device_timeouts() == 0
    tess = ref["tess"]
    s3 = 3 ** d
    nbr, cnt = metrics.padded_neighbours(tess["nbrs"], s3)
    off = tess["offsets"]
    B = metrics.blocks_from_flat(out.bnear.cpu().numpy(), out.nf_off.cpu().numpy(), nbr, cnt, off, s3)
    rep = dict(U=out.u.cpu().numpy(), V=out.v.cpu().numpy(), At=out.at.cpu().numpy(), B=B)
    rep_o = dict(U=ref["U"], V=ref["V"], At=ref["coupling"], B=ref["nearfield"])
    err = metrics.ublr_difference(off, nbr, cnt, s3, ref["ranks"], rep, rep_o)
    print(f"mixed compression {kind} n={n} sketch={sketch}: rel err vs FP64 oracle {err:.3e}")
    assert err < MIXED_BOUND


# 2r = 22, 60, 90, 120, 148 sketch columns: tile widths 32, 64, 96, 128 and 160
@pytest.mark.parametrize("kind,d,grid,n,k", [("laplace2d", 2, (4, 4), 1900, 1),
                                            ("laplace3d", 3, (3, 3, 3), 2100, 20),
                                            ("laplace2d", 2, (5, 4), 2750, 35),
                                            ("laplace3d", 3, (3, 3, 2), 2900, 50),
                                            ("laplace2d", 2, (3, 3), 3100, 64)])
def test_mixed_tagged_sketch_every_tile_width(kind, d, grid, n, k):
    """S_i = sum_c tau_i(c) A(I_i, I_c) G(I_c) and R_j = sum_c tau_j(c) A(I_c, I_j)^T H(I_c)
    (the tag-factored form of the combination S_i = sum_j z_ij Y_j of §5.3), written out
    densely here from the oracle's tessellation and projected tags."""
    tb = _tb()
    r = k + 10
    pts = inputs.uniform_points(n, d, seed=11 * n)
    lo, hi = (0.0,) * d, (1.0,) * d
    b = int(np.prod(grid))
    ell = orc.tag_columns(d, 3)
    T, G, H = inputs.tagging_draws(b, ell, n, r, seed=11 * n + 1)
    tess = orc.tessellate(pts, grid, lo, hi)
    _, tau, _ = orc.decode(T, tess)
    perm = tess["perm"]
    box = np.repeat(np.arange(b), np.diff(tess["offsets"]))
    A = orc.dense_matrix(orc.KernelOperator(kind, pts[perm]))
    W = tau[box[:, None], box[None, :]]
    S_ref = (A * W) @ G[perm]
    R_ref = (A.T * W) @ H[perm]   # row p of R: sum_q tau_{box p}(box q) A(q, p) H(q)
    prob = tb.make_problem(d, kind, n, grid, lo, hi, k, 10, 3, precision=tb.MIXED,
                           sketch=tb.SKETCH_TAGGED)
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    lay = tb.tblr_tessellate(prob, t(pts))
    assert np.array_equal(lay.perm.cpu().numpy(), perm)
    s, rr = tb.tblr_tagged_sketch(prob, lay, t(tau), t(G), t(H))
    s, rr = s.cpu().numpy(), rr.cpu().numpy()
    assert tb.tblr_device_timeouts() == 0
    for got, ref in ((s, S_ref), (rr, R_ref)):
        err = metrics.rel(got, ref)
        print(f"mixed tagged sketch {kind} n={n} 2r={2 * r}: rel err {err:.3e}")
        assert err < MIXED_BOUND / 4
        row_err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert row_err.max() < MIXED_BOUND


# Coupling blocks on the tensor cores: boxes of 130 to 800 points (several
# 128-row tiles and 64-point chunks, ragged tails), every rank tile (k -> 16,
# 32, 64 columns, k = 1), ranks below k and zero, empty boxes, and the
# self-adjoint mirror.  Columns of U and V past a box's rank hold garbage that must be ignored.
@pytest.mark.parametrize("kind,d,grid,n,k,hi,selfadjoint", [
    ("laplace2d", 2, (3, 3), 3001, 6, 1.0, False),
    ("laplace3d", 3, (2, 2, 2), 2100, 20, 1.0, False),
    ("laplace2d", 2, (4, 4), 2600, 45, 0.6, False),
    ("laplace3d", 3, (2, 2, 2), 1500, 64, 1.0, False),
    ("laplace2d", 2, (3, 3), 3001, 32, 1.0, True),
    ("laplace3d", 3, (2, 2, 2), 2100, 64, 1.0, True),
    ("laplace2d", 2, (2, 2), 3000, 1, 1.0, False),          # ~750-point boxes: 6 row tiles
    ("laplace3d", 3, (2, 2, 1), 2800, 40, 1.0, True),
])
def test_mixed_coupling_matches_dense_definition(kind, d, grid, n, k, hi, selfadjoint):
    """Atilde_ij = U_i(:, :k_i)^T A(I_i, I_j) V_j(:, :k_j) (§2.5), zero past the ranks."""
    tb = _tb()
    rng = np.random.default_rng(1000 + n + k)
    pts = inputs.uniform_points(n, d, seed=n + k) * hi      # hi < 1 leaves boxes empty
    lo, top = (0.0,) * d, (1.0,) * d
    tess = orc.tessellate(pts, grid, lo, top)
    perm, off = tess["perm"], tess["offsets"]
    b = len(off) - 1
    m = np.diff(off)
    ranks = np.minimum(k, m).astype(np.int32)
    busy = np.flatnonzero(m > 0)
    ranks[busy[1]] = max(1, k // 2)
    ranks[busy[2]] = 0
    ranks[busy[3]] = 1
    U = rng.standard_normal((n, k)) / 16
    V = U if selfadjoint else rng.standard_normal((n, k)) / 16
    garbage = 1e30
    U = U.copy()
    V = V if selfadjoint else V.copy()
    for i in range(b):
        U[off[i]:off[i + 1], ranks[i]:] = garbage
        if not selfadjoint:
            V[off[i]:off[i + 1], ranks[i]:] = -garbage
    A = orc.dense_matrix(orc.KernelOperator(kind, pts[perm]))
    ref = np.zeros((b, b, k, k))
    for i in range(b):
        for j in range(b):
            ki, kj = ranks[i], ranks[j]
            ref[i, j, :ki, :kj] = (U[off[i]:off[i + 1], :ki].T @ A[off[i]:off[i + 1], off[j]:off[j + 1]]
                                   @ V[off[j]:off[j + 1], :kj])
    prob = tb.make_problem(d, kind, n, grid, lo, top, k, 10, 3, precision=tb.MIXED,
                           sketch=tb.SKETCH_TAGGED, selfadjoint=selfadjoint)
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    lay = tb.tblr_tessellate(prob, t(pts))
    assert np.array_equal(lay.perm.cpu().numpy(), perm)
    u_d = t(U)
    v_d = u_d if selfadjoint else t(V)
    at = tb.tblr_coupling(prob, lay, u_d, v_d, t(ranks), int(m.max())).cpu().numpy()
    assert tb.tblr_device_timeouts() == 0
    for i in range(b):
        for j in range(b):
            if ranks[i] == 0 or ranks[j] == 0:
                assert not at[i, j].any()
                continue
            assert not at[i, j, ranks[i]:, :].any() and not at[i, j, :, ranks[j]:].any()
            blk = np.linalg.norm(at[i, j] - ref[i, j]) / np.linalg.norm(ref[i, j])
            assert blk < MIXED_BOUND, (i, j, blk)
    err = metrics.rel(at, ref)
    print(f"mixed coupling {kind} n={n} k={k} selfadjoint={selfadjoint}: rel err {err:.3e}")
    assert err < MIXED_BOUND / 4


def test_simt_coupling_form_matches_dense_definition(tmp_path):
    """TBLR_COUPLING_SIMT=1 (read once per process, so run in a child) selects the FP32 SIMT form
    of the mixed coupling; both forms must meet the same bound against U_i^T A_ij V_j (§2.5)."""
    import os
    import subprocess
    import sys
    out = tmp_path / "at.npy"
    code = f"""
import numpy as np, torch
from oracle import tagging as orc
from paper_2501_05528_gb300 import inputs, tblr as tb
n, d, grid, k = 2100, 3, (2, 2, 2), 20
pts = inputs.uniform_points(n, d, seed=5)
tess = orc.tessellate(pts, grid, (0.,) * d, (1.,) * d)
rng = np.random.default_rng(6)
U, V = rng.standard_normal((n, k)) / 16, rng.standard_normal((n, k)) / 16
ranks = np.minimum(k, np.diff(tess["offsets"])).astype(np.int32)
prob = tb.make_problem(d, "laplace3d", n, grid, (0.,) * d, (1.,) * d, k, 10, 3,
                       precision=tb.MIXED, sketch=tb.SKETCH_TAGGED)
t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
lay = tb.tblr_tessellate(prob, t(pts))
at = tb.tblr_coupling(prob, lay, t(U), t(V), t(ranks), int(np.diff(tess["offsets"]).max()))
assert tb.tblr_device_timeouts() == 0
np.save({str(out)!r}, at.cpu().numpy())
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, TBLR_COUPLING_SIMT="1", PYTHONPATH=root)
    subprocess.run([sys.executable, "-c", code], check=True, cwd=root, env=env, timeout=600)
    at_simt = np.load(out)
    n, d, grid, k = 2100, 3, (2, 2, 2), 20
    pts = inputs.uniform_points(n, d, seed=5)
    tess = orc.tessellate(pts, grid, (0.0,) * d, (1.0,) * d)
    perm, off = tess["perm"], tess["offsets"]
    rng = np.random.default_rng(6)
    U, V = rng.standard_normal((n, k)) / 16, rng.standard_normal((n, k)) / 16
    A = orc.dense_matrix(orc.KernelOperator("laplace3d", pts[perm]))
    b = len(off) - 1
    ref = np.zeros((b, b, k, k))
    for i in range(b):
        for j in range(b):
            ref[i, j] = U[off[i]:off[i + 1]].T @ A[off[i]:off[i + 1], off[j]:off[j + 1]] @ V[off[j]:off[j + 1]]
    err = metrics.rel(at_simt, ref)
    print(f"SIMT coupling form: rel err {err:.3e}")
    assert err < MIXED_BOUND / 4


def test_tile_width_tuner_records_an_admissible_width():
    """The tagged sketch's tile-width autotuner: every candidate gives the same samples within the
    mixed bound, the chosen width is admissible and recorded for the class, and later sketches of
    the class reproduce the tuner's result bit for bit."""
    tb = _tb()
    tb.tblr_tune_clear()
    n, d, grid, k = 2900, 3, (3, 3, 2), 50      # 2r = 120 sketch columns: all five widths admissible
    pts = inputs.uniform_points(n, d, seed=4242)
    lo, hi = (0.0,) * d, (1.0,) * d
    b = int(np.prod(grid))
    T, G, H = inputs.tagging_draws(b, orc.tag_columns(d, 3), n, k + 10, seed=4243)
    tess = orc.tessellate(pts, grid, lo, hi)
    _, tau, _ = orc.decode(T, tess)
    prob = tb.make_problem(d, "laplace3d", n, grid, lo, hi, k, 10, 3, precision=tb.MIXED,
                           sketch=tb.SKETCH_TAGGED)
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    lay = tb.tblr_tessellate(prob, t(pts))
    try:
        assert tb.tblr_tuned_width(prob) == 0
        s0, r0 = (x.cpu().numpy() for x in tb.tblr_tagged_sketch(prob, lay, t(tau), t(G), t(H)))
        w, s1, r1 = tb.tblr_tune_tagged_sketch(prob, lay, t(tau), t(G), t(H))
        assert w in (32, 64, 96, 128, 160)
        assert tb.tblr_tuned_width(prob) == w
        s2, r2 = (x.cpu().numpy() for x in tb.tblr_tagged_sketch(prob, lay, t(tau), t(G), t(H)))
        assert tb.tblr_device_timeouts() == 0
        s1, r1 = s1.cpu().numpy(), r1.cpu().numpy()
        assert np.array_equal(s1, s2) and np.array_equal(r1, r2)
        assert metrics.rel(s1, s0) < MIXED_BOUND / 4 and metrics.rel(r1, r0) < MIXED_BOUND / 4
    finally:
        tb.tblr_tune_clear()
    assert tb.tblr_tuned_width(prob) == 0
