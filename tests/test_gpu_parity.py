"""GPU parity: every step of the CUDA path against the CPU oracle, on the same seeded inputs.

Cases are sized so the oracle finishes in seconds while spanning several tiles
with ragged tails (n not a multiple of the 16-row tile, sketch columns not a
multiple of 256), plus the degenerate geometries: empty boxes, boxes with fewer
points than k, a grid without far field, and d = 1.

Tolerances (FP64 path): index lists and the test matrices bit-exact; sketch
and per-step floating outputs within 1e-11 relative (they differ only by
summation order and 1-ulp differences of log/rsqrt); the reconstruction
A_uBLR within 1e-10 relative Frobenius (the FP64 parity bound).  The exactly
uniform BLR case must also reproduce A itself to 1e-12.
"""
import numpy as np
import pytest

from oracle import tagging as orc
from paper_2501_05528_gb300 import inputs
from paper_2501_05528_gb300 import metrics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tb():
    from paper_2501_05528_gb300 import tblr
    return tblr


CASES = {
    "exact_ublr_2d": dict(kind="dense", d=2, grid=(4, 4), k=8, e=3, seed=1),
    "laplace2d_ragged": dict(kind="laplace2d", d=2, grid=(6, 6), n=3001, k=8, e=3, seed=2),
    "laplace3d_ragged": dict(kind="laplace3d", d=3, grid=(4, 4, 4), n=2501, k=6, e=1, seed=3),
    "dense_1d_small_boxes": dict(kind="dense1d", d=1, grid=(9,), n=70, k=16, e=0, seed=4),
    "laplace2d_empty_boxes": dict(kind="laplace2d_holes", d=2, grid=(5, 5), n=900, k=6, e=2, seed=5),
    "laplace2d_no_farfield": dict(kind="laplace2d", d=2, grid=(2, 2), n=300, k=5, e=3, seed=6),
}


def _make_inputs(c):
    d, grid, seed = c["d"], c["grid"], c["seed"]
    lo, hi = (0.0,) * d, (1.0,) * d
    dense = None
    if c["kind"] == "dense":
        pts, owner = inputs.box_points(grid, 64, seed)
        dense = inputs.exact_ublr_matrix(owner, c["k"], seed + 100)
        kind = "dense"
    elif c["kind"] == "dense1d":
        pts = inputs.uniform_points(c["n"], 1, seed)
        dense = np.random.default_rng(seed + 100).standard_normal((c["n"], c["n"]))
        kind = "dense"
    elif c["kind"] == "laplace2d_holes":
        pts = inputs.uniform_points(c["n"], 2, seed)
        keep = ~((pts[:, 0] > 0.4) & (pts[:, 0] < 0.8) & (pts[:, 1] > 0.2) & (pts[:, 1] < 0.6))
        pts = pts[keep]
        kind = "laplace2d"
    else:
        pts = inputs.uniform_points(c["n"], d, seed)
        kind = c["kind"]
    b = int(np.prod(grid))
    ell = orc.tag_columns(d, c["e"])
    r = c["k"] + 10
    T, G, H = inputs.tagging_draws(b, ell, len(pts), r, seed + 200)
    return dict(pts=pts, kind=kind, dense=dense, T=T, G=G, H=H, lo=lo, hi=hi, ell=ell, r=r)


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    tb = _tb()
    c = CASES[request.param]
    x = _make_inputs(c)
    d, grid, k = c["d"], c["grid"], c["k"]
    n = len(x["pts"])
    res = orc.reconstruct_tag(x["pts"], grid, x["lo"], x["hi"], x["kind"], x["T"], x["G"], x["H"],
                              k, 10, dense=x["dense"])
    dev = torch.device("cuda")
    prob = tb.make_problem(d, x["kind"], n, grid, x["lo"], x["hi"], k, 10, c["e"])
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    pts, T, G, H = t(x["pts"]), t(x["T"]), t(x["G"]), t(x["H"])
    dense = None if x["dense"] is None else t(x["dense"])
    lay = tb.tblr_tessellate(prob, pts)
    nf_off, m_max = tb.tblr_nearfield_offsets(prob, lay)
    om = tb.tblr_test_matrices(prob, lay, T, G, H)
    yz = tb.tblr_sketch(prob, lay, om, dense=dense)
    z, tau, rho = tb.tblr_decode(prob, lay, T)
    s, rr = tb.tblr_combine(prob, lay, yz, z)
    u, ranks = tb.tblr_col(prob, lay, s)
    v, ranks_v = tb.tblr_col(prob, lay, rr)
    mm, total = int(m_max.item()), int(nf_off[-1].item())
    at = tb.tblr_coupling(prob, lay, u, v, ranks, mm, dense=dense)
    bn = tb.tblr_nearfield(prob, lay, u, at, v, ranks, nf_off, mm, total, dense=dense)
    full = tb.tblr_compress(prob, lay, T, G, H, dense=dense)
    torch.cuda.synchronize()
    h = lambda a: a.cpu().numpy()
    gpu = dict(perm=h(lay.perm), offsets=h(lay.offsets), nbr=h(lay.nbr), nnbr=h(lay.nnbr),
               colour=h(lay.colour), pts=h(lay.pts).reshape(d, n).T, omega=h(om).reshape(-1, n).T,
               yz=h(yz), z=h(z), tau=h(tau), rho=h(rho), s=h(s), rr=h(rr), u=h(u), v=h(v),
               ranks=h(ranks), ranks_v=h(ranks_v), at=h(at), nf_off=h(nf_off), m_max=mm,
               bnear=h(bn)[:total], full=full, prob=prob)
    return dict(name=request.param, c=c, x=x, res=res, gpu=gpu, n=n)


def test_tessellation_bit_exact(case):
    g, res = case["gpu"], case["res"]
    tess = res["tess"]
    s3 = 3 ** case["c"]["d"]
    assert np.array_equal(g["perm"], tess["perm"])
    assert np.array_equal(g["offsets"], tess["offsets"])
    nbr, cnt = metrics.padded_neighbours(tess["nbrs"], s3)
    assert np.array_equal(g["nbr"], nbr)
    assert np.array_equal(g["nnbr"], cnt)
    assert np.array_equal(g["colour"], tess["colour"])
    assert np.array_equal(g["pts"], case["x"]["pts"][tess["perm"]])
    off = tess["offsets"]
    assert g["m_max"] == int(np.max(np.diff(off)))


def test_test_matrices_bit_exact(case):
    g, res = case["gpu"], case["res"]
    assert np.array_equal(g["omega"], np.hstack([res["Omega"], res["Psi"]]))


def test_sketch_matches(case):
    g, res = case["gpu"], case["res"]
    ref = np.hstack([res["Y"], res["Z"]])
    assert metrics.rel(g["yz"], ref) < 1e-12


def test_decode_matches(case):
    g, res = case["gpu"], case["res"]
    assert np.abs(g["z"] - res["z"]).max() < 1e-13
    assert np.abs(g["tau"] - res["tau"]).max() < 1e-12 * max(1.0, np.abs(res["tau"]).max())
    assert np.array_equal(np.isnan(g["rho"]), np.isnan(res["rho"]))
    ok = ~np.isnan(res["rho"])
    assert np.allclose(g["rho"][ok], res["rho"][ok], rtol=1e-10, atol=0)


def test_combine_matches(case):
    """S = sum_j z_j Y_j: errors are measured against the size of the summands
    (|z| |Y|), since with no far field S itself is pure cancellation noise."""
    g, res = case["gpu"], case["res"]
    yz = np.hstack([res["Y"], res["Z"]])
    scale = np.linalg.norm(yz) * max(1.0, np.abs(res["z"]).max())
    assert np.linalg.norm(g["s"] - res["S"]) <= 1e-12 * scale
    assert np.linalg.norm(g["rr"] - res["R"]) <= 1e-12 * scale
    if np.linalg.norm(res["S"]) > 1e-6 * scale:
        assert metrics.rel(g["s"], res["S"]) < 1e-11
        assert metrics.rel(g["rr"], res["R"]) < 1e-11


def test_ranks_and_bases(case):
    g, res = case["gpu"], case["res"]
    assert np.array_equal(g["ranks"], res["ranks"])
    assert np.array_equal(g["ranks_v"], res["ranks"])
    off = res["tess"]["offsets"]
    for i in range(len(off) - 1):
        ki = int(res["ranks"][i])
        rows = slice(off[i], off[i + 1])
        Ug, Uo = g["u"][rows, :ki], res["U"][rows, :ki]
        if ki:
            assert np.abs(Ug.T @ Ug - np.eye(ki)).max() < 1e-13
            # range of the sample captured by each basis (basis-independent)
            S = res["S"][rows]
            Pg = Ug @ (Ug.T @ S)
            Po = Uo @ (Uo.T @ S)
            assert np.linalg.norm(Pg - Po) <= 1e-10 * np.linalg.norm(S)
        assert np.all(g["u"][rows, ki:] == 0.0)


def test_reconstruction_matches_oracle(case):
    g, res = case["gpu"], case["res"]
    tess = res["tess"]
    s3 = 3 ** case["c"]["d"]
    off = tess["offsets"]
    nbr, cnt = metrics.padded_neighbours(tess["nbrs"], s3)
    Bg = metrics.blocks_from_flat(g["bnear"], g["nf_off"], nbr, cnt, off, s3)
    rep_g = dict(U=g["u"], V=g["v"], At=g["at"], B=Bg)
    rep_o = dict(U=res["U"], V=res["V"], At=res["coupling"], B=res["nearfield"])
    err = metrics.ublr_difference(off, nbr, cnt, s3, res["ranks"], rep_g, rep_o)
    assert err <= 1e-10, err
    for key in Bg:
        ref = res["nearfield"][key]
        if ref.size:
            assert np.linalg.norm(Bg[key] - ref) <= 1e-10 * max(np.linalg.norm(ref), 1e-300) + 1e-12


def test_whole_pipeline_equals_step_chain(case):
    g = case["gpu"]
    f = g["full"]
    total = f.total
    for name, ref in (("yz", g["yz"]), ("z", g["z"]), ("u", g["u"]), ("v", g["v"]), ("at", g["at"])):
        assert np.array_equal(getattr(f, name).cpu().numpy(), ref), name
    assert np.array_equal(f.bnear.cpu().numpy()[:total], g["bnear"])


def test_exact_ublr_reproduces_a(case):
    if case["name"] != "exact_ublr_2d":
        pytest.skip("exactly uniform BLR input only")
    g, res = case["gpu"], case["res"]
    tess = res["tess"]
    perm, off = tess["perm"], tess["offsets"]
    A = case["x"]["dense"][np.ix_(perm, perm)]
    nbr, cnt = metrics.padded_neighbours(tess["nbrs"], 9)
    Bg = metrics.blocks_from_flat(g["bnear"], g["nf_off"], nbr, cnt, off, 9)
    rec = dict(res)
    rec.update(U=g["u"], V=g["v"], coupling=g["at"], nearfield=Bg)
    Ar = orc.assemble(rec)
    assert np.linalg.norm(A - Ar) / np.linalg.norm(A) <= 1e-12


def test_host_buffer_entry_point_matches(case):
    tb = _tb()
    g, x = case["gpu"], case["x"]
    o = tb.tblr_compress_host(g["prob"], x["pts"], x["T"], x["G"], x["H"], dense=x["dense"])
    assert np.array_equal(o["perm"].numpy(), g["perm"])
    assert np.array_equal(o["u"].numpy(), g["u"])
    assert np.array_equal(o["at"].numpy(), g["at"])
    assert np.array_equal(o["bnear"].numpy()[:o["bnear_size"]], g["bnear"])


def test_tagged_sketch_matches_the_black_box_samples(case):
    """TBLR_SKETCH_TAGGED forms S = sum_c tau_c A_ic G_c directly; it must equal the oracle's
    S = sum_j z_j Y_j (eq. extend_test_mat), and the tagged pipeline its reconstruction."""
    tb = _tb()
    c, x, res, g = case["c"], case["x"], case["res"], case["gpu"]
    d, grid, k = c["d"], c["grid"], c["k"]
    n = case["n"]
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    prob = tb.make_problem(d, x["kind"], n, grid, x["lo"], x["hi"], k, 10, c["e"],
                           sketch=tb.SKETCH_TAGGED)
    pts, T, G, H = t(x["pts"]), t(x["T"]), t(x["G"]), t(x["H"])
    dense = None if x["dense"] is None else t(x["dense"])
    lay = tb.tblr_tessellate(prob, pts)
    z, tau, rho = tb.tblr_decode(prob, lay, T)
    s, rr = tb.tblr_tagged_sketch(prob, lay, tau, G, H, dense=dense)
    full = tb.tblr_compress(prob, lay, T, G, H, dense=dense)
    torch.cuda.synchronize()
    yz = np.hstack([res["Y"], res["Z"]])
    scale = np.linalg.norm(yz) * max(1.0, np.abs(res["z"]).max())
    assert np.linalg.norm(s.cpu().numpy() - res["S"]) <= 1e-12 * scale
    assert np.linalg.norm(rr.cpu().numpy() - res["R"]) <= 1e-12 * scale
    tess = res["tess"]
    s3 = 3 ** d
    off = tess["offsets"]
    nbr, cnt = metrics.padded_neighbours(tess["nbrs"], s3)
    B = metrics.blocks_from_flat(full.bnear.cpu().numpy(), full.nf_off.cpu().numpy(), nbr, cnt,
                                 off, s3)
    rep = dict(U=full.u.cpu().numpy(), V=full.v.cpu().numpy(), At=full.at.cpu().numpy(), B=B)
    rep_o = dict(U=res["U"], V=res["V"], At=res["coupling"], B=res["nearfield"])
    err = metrics.ublr_difference(off, nbr, cnt, s3, res["ranks"], rep, rep_o)
    assert err <= 1e-10, err


@pytest.mark.parametrize("precision,bound", [(0, 1e-10), (1, 1e-6)], ids=["fp64", "mixed"])
@pytest.mark.parametrize("kind,d,grid,n,k,e", [("laplace2d", 2, (6, 5), 3001, 8, 3),
                                              ("laplace3d", 3, (4, 4, 3), 4001, 10, 1)])
def test_selfadjoint_mode_matches_oracle_with_psi_equal_omega(kind, d, grid, n, k, e, precision,
                                                              bound):
    """TBLR_SKETCH_SELFADJOINT (A = A^T, H = G): the oracle run with H = G gives R = S, so
    V = U; the GPU forms S once, copies U to V and the coupling for i <= j only, mirroring
    Atilde_ji = Atilde_ij^T.  The result must equal the oracle's general algorithm on the
    same draws."""
    tb = _tb()
    pts = inputs.uniform_points(n, d, seed=5 * n)
    b = int(np.prod(grid))
    ell = orc.tag_columns(d, e)
    T, G, _ = inputs.tagging_draws(b, ell, n, k + 10, seed=5 * n + 1)
    lo, hi = (0.0,) * d, (1.0,) * d
    ref = orc.reconstruct_tag(pts, grid, lo, hi, kind, T, G, G, k, 10)
    assert np.allclose(ref["U"], ref["V"], rtol=0, atol=1e-12)     # R = S in the oracle too
    prob = tb.make_problem(d, kind, n, grid, lo, hi, k, 10, e, precision=precision,
                           sketch=tb.SKETCH_TAGGED, selfadjoint=True)
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    out = tb.compress(prob, t(pts), t(T), t(G), t(G))
    torch.cuda.synchronize()
    u, v, at = out.u.cpu().numpy(), out.v.cpu().numpy(), out.at.cpu().numpy()
    assert np.array_equal(u, v)
    mirrored = np.transpose(at, (1, 0, 3, 2))
    off_diag = ~np.eye(b, dtype=bool)
    assert np.array_equal(at[off_diag], mirrored[off_diag])     # written once, mirrored
    tess = ref["tess"]
    s3 = 3 ** d
    nbr, cnt = metrics.padded_neighbours(tess["nbrs"], s3)
    off = tess["offsets"]
    B = metrics.blocks_from_flat(out.bnear.cpu().numpy(), out.nf_off.cpu().numpy(), nbr, cnt, off, s3)
    rep = dict(U=u, V=v, At=at, B=B)
    rep_o = dict(U=ref["U"], V=ref["V"], At=ref["coupling"], B=ref["nearfield"])
    err = metrics.ublr_difference(off, nbr, cnt, s3, ref["ranks"], rep, rep_o)
    print(f"self-adjoint {kind} precision={precision}: rel err vs oracle {err:.3e}")
    assert err <= bound, err


@pytest.mark.parametrize("d,grid,n,k,e", [(2, (6, 6), 3001, 8, 3), (2, (7, 5), 2500, 6, 1),
                                         (3, (4, 4, 4), 4001, 8, 3)])
def test_minratio_decode_and_compression_match_oracle(d, grid, n, k, e):
    """TBLR_Z_MINRATIO (§5.3): the per-box LP on the GPU reaches the oracle's optimum
    (aspect ratios to 1e-9, the same null vectors), and the whole compression with those
    vectors matches the oracle's to the FP64 bound."""
    tb = _tb()
    kind = "laplace2d" if d == 2 else "laplace3d"
    pts = inputs.uniform_points(n, d, seed=9 * n)
    b = int(np.prod(grid))
    T, G, H = inputs.tagging_draws(b, orc.tag_columns(d, e), n, k + 10, seed=9 * n + 1)
    lo, hi = (0.0,) * d, (1.0,) * d
    ref = orc.reconstruct_tag(pts, grid, lo, hi, kind, T, G, H, k, 10, zrule="minratio")
    _, _, rho0 = orc.decode(T, ref["tess"])
    prob = tb.make_problem(d, kind, n, grid, lo, hi, k, 10, e, zrule=tb.Z_MINRATIO)
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    lay = tb.tblr_tessellate(prob, t(pts))
    z, tau, rho = tb.tblr_decode(prob, lay, t(T))
    z, tau, rho = z.cpu().numpy(), tau.cpu().numpy(), rho.cpu().numpy()
    assert tb.tblr_decode_lp_failures() == 0
    fin = np.isfinite(ref["rho"])
    assert np.array_equal(np.isfinite(rho), fin)
    assert np.max(np.abs(rho[fin] - ref["rho"][fin]) / ref["rho"][fin]) <= 1e-9
    assert np.nanmean(rho) < np.nanmean(rho0)
    assert np.max(np.abs(z - ref["z"])) <= 1e-8
    out = tb.compress(prob, t(pts), t(T), t(G), t(H))
    torch.cuda.synchronize()
    tess = ref["tess"]
    s3 = 3 ** d
    nbr, cnt = metrics.padded_neighbours(tess["nbrs"], s3)
    off = tess["offsets"]
    B = metrics.blocks_from_flat(out.bnear.cpu().numpy(), out.nf_off.cpu().numpy(), nbr, cnt, off, s3)
    rep = dict(U=out.u.cpu().numpy(), V=out.v.cpu().numpy(), At=out.at.cpu().numpy(), B=B)
    rep_o = dict(U=ref["U"], V=ref["V"], At=ref["coupling"], B=ref["nearfield"])
    err = metrics.ublr_difference(off, nbr, cnt, s3, ref["ranks"], rep, rep_o)
    print(f"minratio d={d} e={e}: mean rho {np.nanmean(rho):.3f} (projected {np.nanmean(rho0):.3f}), "
          f"reconstruction rel err {err:.3e}")
    assert err <= 1e-10, err


@pytest.mark.parametrize("kind,d,grid,n,k", [("laplace2d", 2, (4, 4), 1500, 6),
                                            ("laplace3d", 3, (3, 3, 3), 1800, 5)])
def test_algorithm3_basic_through_the_tagged_sketch(kind, d, grid, n, k):
    """Algorithm 3 (§4.2, the plain per-box range finder): tags tau_ic = [c not in N_i] make
    the tag-factored sketch S_i = A(I_i, F_i) G(F_i) (and R_i likewise); S, R, the ranks and the
    bases must match the oracle's Algorithm 3 run with the same shared G, H."""
    tb = _tb()
    p = 10
    r = k + p
    lo, hi = (0.0,) * d, (1.0,) * d
    pts = inputs.uniform_points(n, d, seed=31 + d)
    b = int(np.prod(grid))
    T, G, H = inputs.tagging_draws(b, orc.tag_columns(d, 3), n, r, seed=32 + d)
    tess = orc.tessellate(pts, grid, lo, hi)
    perm, off = tess["perm"], tess["offsets"]
    op = orc.KernelOperator(kind, pts[perm])
    Ub, Vb, ks = orc.basic_bases(op, tess, k, r, None, shared=(G[perm], H[perm]))
    prob = tb.make_problem(d, kind, n, grid, lo, hi, k, p, 3, sketch=tb.SKETCH_TAGGED)
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    lay = tb.tblr_tessellate(prob, t(pts))
    tau = tb.tblr_far_indicator(prob, lay).cpu().numpy()
    tau_ref = np.ones((b, b))
    for i in range(b):
        tau_ref[i, tess["nbrs"][i]] = 0.0
    assert np.array_equal(tau, tau_ref)
    s, rr = tb.tblr_tagged_sketch(prob, lay, t(tau), t(G), t(H))
    s_h, r_h = s.cpu().numpy(), rr.cpu().numpy()
    for i in range(b):
        rows = slice(off[i], off[i + 1])
        if off[i + 1] == off[i]:
            continue
        Om, Ps = G[perm].copy(), H[perm].copy()
        for j in tess["nbrs"][i]:
            Om[off[j]:off[j + 1]] = 0.0
            Ps[off[j]:off[j + 1]] = 0.0
        Y = op.apply(Om)[rows]
        Z = op.apply(Ps, adjoint=True)[rows]
        if np.linalg.norm(Y) > 0:
            assert metrics.rel(s_h[rows], Y) < 1e-11
            assert metrics.rel(r_h[rows], Z) < 1e-11
    u, ranks = tb.tblr_col(prob, lay, s)
    v, _ = tb.tblr_col(prob, lay, rr)
    assert np.array_equal(ranks.cpu().numpy(), ks)
    u, v = u.cpu().numpy(), v.cpu().numpy()
    for i in range(b):
        if ks[i] == 0:
            continue
        rows = slice(off[i], off[i + 1])
        for got, ref in ((u, Ub), (v, Vb)):
            P1 = got[rows, :ks[i]] @ got[rows, :ks[i]].T
            P2 = ref[rows, :ks[i]] @ ref[rows, :ks[i]].T
            assert np.abs(P1 - P2).max() < 1e-9
