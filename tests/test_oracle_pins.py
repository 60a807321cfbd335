"""Pins for the CPU oracle: checks against what the paper and the mathematics fix.

None of these compares the oracle with itself.  Each test names the passage or
the mathematical fact it relies on: printed structure of the worked example,
closed forms (Cramer's rule, a matrix with known SVD, kernel values at 3-4-5
triangles), invariants (eq. projected_tags, T z = 0, rho >= 1, orthonormal
bases), exact recovery of an exactly uniform BLR matrix, brute-force SVDs of
the far-field block rows, Algorithm 3 as a textbook cross-check, and the
matvec counts of §4.2 and Table 1.  The planted-mistake tests at the end show
that a plausible error in the oracle makes one of these pins fail.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import tagging as orc
from paper_2501_05528_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tess_for(grid, per_box, seed):
    pts, owner = inputs.box_points(grid, per_box, seed)
    d = len(grid)
    tess = orc.tessellate(pts, grid, (0.0,) * d, (1.0,) * d)
    return pts, owner, tess


# ----------------------------------------------------------------- geometry

def test_worked_example_1d_neighbours_and_tag_submatrix():
    """§2.5 / §4.1: 8 boxes in 1-D, N_3 = {2,3,4}, T is 8 x 4, T^(3) = rows 2..4."""
    fields = {}
    with open(os.path.join(GOLDEN, "worked_example_1d.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            fields[key] = [int(v) for v in vals]
    b = fields["boxes"][0]
    d = fields["dimension"][0]
    _, _, tess = _tess_for((b,), 5, seed=11)
    assert tess["b"] == b
    assert orc.tag_columns(d, 0) == fields["tag_columns"][0]
    got = [int(j) + 1 for j in tess["nbrs"][2]]          # box 3, 1-based
    assert got == fields["neighbours_of_3"]
    T = np.arange(b * 4, dtype=float).reshape(b, 4)
    Ti = T[tess["nbrs"][2], :]
    rows = fields["tag_submatrix_rows_of_3"]
    assert np.array_equal(Ti, T[[r - 1 for r in rows], :])


@pytest.mark.parametrize("grid", [(7,), (5, 4), (3, 4, 5)])
def test_tessellation_properties(grid):
    """Every point lies in its box; stable order; |N_i| closed form; colours unique per N_i."""
    d = len(grid)
    rng = np.random.default_rng(3)
    lo = np.array([-1.0, 0.5, 2.0][:d])
    hi = lo + np.array([2.0, 1.5, 0.25][:d])
    pts = lo + rng.random((600, d)) * (hi - lo)
    pts[0] = hi                                             # upper face -> last box
    tess = orc.tessellate(pts, grid, lo, hi)
    h = (hi - lo) / np.array(grid)
    off, perm, cell = tess["offsets"], tess["perm"], tess["cell"]
    assert off[-1] == len(pts) and np.all(np.diff(off) >= 0)
    assert sorted(perm.tolist()) == list(range(len(pts)))
    for i in range(tess["b"]):
        members = perm[off[i]:off[i + 1]]
        assert np.all(np.diff(members) > 0)                 # stable: input order kept
        x = pts[members]
        lower = lo + cell[i] * h
        upper = lo + (cell[i] + 1) * h
        assert np.all(x >= lower - 1e-12) and np.all(x <= upper + 1e-12)
        # |N_i| = prod_a (1 + [q_a > 0] + [q_a < n_a - 1])
        expect = 1
        for a in range(d):
            expect *= 1 + (cell[i, a] > 0) + (cell[i, a] < grid[a] - 1)
        assert len(tess["nbrs"][i]) == expect
        assert i in tess["nbrs"][i]
        cols = tess["colour"][tess["nbrs"][i]]
        assert len(set(cols.tolist())) == len(cols)          # one box per colour in N_i
    assert tess["cell"][orc.box_index(orc.box_coordinates(pts[:1], grid, lo, hi), grid)[0]].tolist() == [g - 1 for g in grid]
    for i in range(tess["b"]):
        for j in tess["nbrs"][i]:
            assert i in tess["nbrs"][j]                       # symmetric relation


# -------------------------------------------------------------------- kernels

def test_kernel_closed_forms():
    """§7.1: log|x - y| with a zero diagonal; 3-D Laplace 1/(4 pi |x - y|)."""
    p2 = np.array([[0.0, 0.0], [0.3, 0.4], [0.6, 0.8]])
    op = orc.KernelOperator("laplace2d", p2)
    K = op.block(np.arange(3), np.arange(3))
    assert K[0, 0] == 0.0 and K[1, 1] == 0.0
    assert abs(K[0, 1] - math.log(0.5)) < 1e-15
    assert abs(K[2, 0] - math.log(1.0)) < 1e-15
    p3 = np.array([[0.0, 0.0, 0.0], [0.0, 0.3, 0.4], [0.2, 0.2, 0.1]])
    op3 = orc.KernelOperator("laplace3d", p3)
    K3 = op3.block(np.arange(3), np.arange(3))
    assert K3[1, 1] == 0.0
    assert abs(K3[0, 1] - 1.0 / (4 * math.pi * 0.5)) < 1e-15
    assert abs(K3[2, 0] - 1.0 / (4 * math.pi * 0.3)) < 1e-14
    X = np.random.default_rng(0).standard_normal((3, 2))
    assert np.allclose(op3.apply(X), K3 @ X, rtol=0, atol=1e-14)


# ---------------------------------------------------------- test matrices

@pytest.mark.parametrize("grid,e", [((6,), 0), ((5, 5), 3), ((4, 3, 3), 1)])
def test_tagged_combination_cancels_near_rows(grid, e):
    """eq. projected_tags: sum_j z_j Omega_j vanishes on I_c for c in N_i, equals tau_c G_c elsewhere."""
    d = len(grid)
    pts, _, tess = _tess_for(grid, 6, seed=5)
    ell = orc.tag_columns(d, e)
    r = 4
    T, G, _ = inputs.tagging_draws(tess["b"], ell, len(pts), r, seed=9)
    Om = orc.extended_test_matrix(T, G, tess)
    z, tau, _ = orc.decode(T, tess)
    off, perm = tess["offsets"], tess["perm"]
    scale = np.abs(Om).max()
    for i in range(tess["b"]):
        comb = sum(z[i, j] * Om[:, j * r:(j + 1) * r] for j in range(ell))
        for c in range(tess["b"]):
            blk = comb[off[c]:off[c + 1]]
            if c in tess["nbrs"][i]:
                assert np.abs(blk).max() <= 1e-13 * scale
            else:
                ref = tau[i, c] * G[perm[off[c]:off[c + 1]]]
                assert np.allclose(blk, ref, rtol=0, atol=1e-13 * scale)


# ------------------------------------------------------------------ decode

@pytest.mark.parametrize("d,e", [(1, 0), (2, 0), (2, 3), (3, 0), (3, 3)])
def test_decode_null_vector(d, e):
    """T(N_i,:) z_i = 0, |z_i| = 1, rho_i >= 1, and z_i is the projection of 1/sqrt(ell) onto
    the null space computed independently from scipy's SVD-based null_space."""
    grid = (5,) * d if d < 3 else (4, 4, 4)
    pts, _, tess = _tess_for(grid, 2, seed=1)
    ell = orc.tag_columns(d, e)
    T, _, _ = inputs.tagging_draws(tess["b"], ell, 1, 1, seed=d * 10 + e)
    z, tau, rho = orc.decode(T, tess)
    w = np.ones(ell) / math.sqrt(ell)
    for i in range(tess["b"]):
        Ti = T[tess["nbrs"][i]]
        assert np.abs(Ti @ z[i]).max() < 1e-13
        assert abs(np.linalg.norm(z[i]) - 1) < 1e-14
        Nsp = scipy.linalg.null_space(Ti)
        ref = Nsp @ (Nsp.T @ w)
        ref /= np.linalg.norm(ref)
        assert np.allclose(z[i], ref, rtol=0, atol=1e-12)
        assert np.allclose(tau[i], T @ z[i], atol=1e-14)
        if not np.isnan(rho[i]):
            assert rho[i] >= 1.0


def test_decode_matches_cramers_rule():
    """§5.2 eq. cramers_rule (alternating signs): for ell = 3^d + 1 and an interior box the null
    vector is the signed cofactor vector, and each projected tag is det([t_q; T^(i)]) / |c|."""
    d = 2
    pts, _, tess = _tess_for((5, 5), 2, seed=2)
    ell = orc.tag_columns(d, 0)
    T, _, _ = inputs.tagging_draws(tess["b"], ell, 1, 1, seed=77)
    z, tau, _ = orc.decode(T, tess)
    interior = [i for i in range(tess["b"]) if len(tess["nbrs"][i]) == 3 ** d]
    assert interior
    for i in interior:
        Ti = T[tess["nbrs"][i]]
        c = orc.cofactor_null_vector(Ti)
        cn = c / np.linalg.norm(c)
        s = np.sign(cn @ z[i])
        assert np.allclose(z[i], s * cn, atol=1e-12)
        for q in range(tess["b"]):
            det = np.linalg.det(np.vstack([T[q], Ti]))
            assert abs(tau[i, q] - s * det / np.linalg.norm(c)) < 1e-11 * max(1.0, abs(det))


# --------------------------------------------------------------------- col

def test_col_known_svd():
    """§2.3 / §2.4: col(S, k) spans the k dominant left singular vectors; closed-form S."""
    rng = np.random.default_rng(4)
    m, r, k = 40, 12, 5
    Q1 = np.linalg.qr(rng.standard_normal((m, r)))[0]
    Q2 = np.linalg.qr(rng.standard_normal((r, r)))[0]
    sig = 2.0 ** -np.arange(r)
    S = Q1 @ np.diag(sig) @ Q2.T
    U = orc.col(S, k)
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-14)
    for c in range(k):
        assert abs(abs(U[:, c] @ Q1[:, c]) - 1) < 1e-12
        p = np.argmax(np.abs(U[:, c]))
        assert U[p, c] > 0


# ------------------------------------------------- exact uniform BLR (P1)

def _exact_case(grid, per_box, k, e, seed):
    pts, owner = inputs.box_points(grid, per_box, seed)
    A = inputs.exact_ublr_matrix(owner, k, seed + 1)
    d = len(grid)
    tess = orc.tessellate(pts, grid, (0.0,) * d, (1.0,) * d)
    ell = orc.tag_columns(d, e)
    T, G, H = inputs.tagging_draws(tess["b"], ell, len(pts), k + 10, seed + 2)
    res = orc.reconstruct_tag(pts, grid, (0.0,) * d, (1.0,) * d, "dense", T, G, H, k, 10, dense=A)
    return pts, owner, A, res


@pytest.mark.parametrize("grid,per_box,k,e", [((4, 4), 64, 8, 3), ((8,), 20, 3, 0), ((4, 4, 4), 12, 4, 2)])
def test_exact_ublr_is_recovered_to_roundoff(grid, per_box, k, e):
    """§2.5 eq. uniformBLRfull: an exactly uniform BLR matrix is reconstructed to <= 1e-12."""
    pts, owner, A, res = _exact_case(grid, per_box, k, e, seed=100 + len(grid))
    perm = res["tess"]["perm"]
    As = A[np.ix_(perm, perm)]
    Ar = orc.assemble(res)
    err = np.linalg.norm(As - Ar) / np.linalg.norm(As)
    assert err <= 1e-12, err
    U = res["U"]
    assert np.allclose(U.T @ U, np.diag(np.diag(U.T @ U)), atol=1e-13)


def test_exact_ublr_bases_span_the_true_bases():
    """P1: range(U_i) equals the generator's range(U_i^true) to 1e-12 (far-field block rows)."""
    grid, per_box, k = (4, 4), 64, 8
    pts, owner = inputs.box_points(grid, per_box, 300)
    A = inputs.exact_ublr_matrix(owner, k, 301)
    tess = orc.tessellate(pts, grid, (0.0, 0.0), (1.0, 1.0))
    T, G, H = inputs.tagging_draws(tess["b"], 13, len(pts), k + 10, 302)
    res = orc.reconstruct_tag(pts, grid, (0.0, 0.0), (1.0, 1.0), "dense", T, G, H, k, 10, dense=A)
    off, perm = tess["offsets"], tess["perm"]
    for i in range(tess["b"]):
        rows = perm[off[i]:off[i + 1]]
        F = orc.far_field(tess["nbrs"][i], tess["b"])
        cols = np.concatenate([perm[off[c]:off[c + 1]] for c in F])
        far = A[np.ix_(rows, cols)]                       # exactly rank k
        Ui = res["U"][off[i]:off[i + 1], :k]
        resid = far - Ui @ (Ui.T @ far)
        assert np.linalg.norm(resid) <= 1e-12 * np.linalg.norm(far)
        farT = A[np.ix_(cols, rows)].T
        Vi = res["V"][off[i]:off[i + 1], :k]
        assert np.linalg.norm(farT - Vi @ (Vi.T @ farT)) <= 1e-12 * np.linalg.norm(farT)


def test_nearfield_probe_equals_discrepancy_on_exact_input():
    """eq. sparse_struct_ids vs eq. discrepancymatrix: with exact far blocks the probe's
    same-colour far residuals vanish, so B_ij = A_ij - U_i Atilde_ij V_j^T."""
    pts, owner, A, res = _exact_case((4, 4), 64, 8, 3, seed=400)
    tess, op = res["tess"], res["op"]
    for (i, j), blk in res["nearfield"].items():
        exact = orc.discrepancy_block(op, res["U"], res["coupling"], res["V"], tess, i, j)
        assert np.abs(blk - exact).max() <= 1e-12 * np.abs(exact).max()


def test_blockwise_definitions_match_table1_literal_steps():
    """Per-block Atilde_ij = U_i^T A_ij V_j and the per-block probe sum agree with the literal
    Table 1 steps (dense V, dense identity probes) on a kernel matrix."""
    pts = inputs.uniform_points(700, 2, seed=8)
    grid = (4, 4)
    tess = orc.tessellate(pts, grid, (0, 0), (1, 1))
    k = 6
    T, G, H = inputs.tagging_draws(tess["b"], 13, len(pts), k + 10, 9)
    res = orc.reconstruct_tag(pts, grid, (0, 0), (1, 1), "laplace2d", T, G, H, k, 10)
    op, ks = res["op"], res["ranks"]
    for (i, j) in [(0, 15), (5, 6), (3, 12), (9, 9)]:
        blk = orc.coupling_block(op, res["U"], res["V"], tess, i, j, ks[i], ks[j])
        assert np.allclose(blk, res["coupling"][i, j][:ks[i], :ks[j]], rtol=0, atol=1e-12)
    for (i, j) in [(0, 0), (0, 5), (5, 10), (15, 10)]:
        blk = orc.nearfield_block(op, res["U"], res["coupling"], res["V"], tess, i, j, k)
        assert np.allclose(blk, res["nearfield"][(i, j)], rtol=0, atol=1e-11)


# ------------------------------------------------------ brute force (P2)

@pytest.mark.parametrize("kind,d,grid,n", [("laplace2d", 2, (5, 5), 900), ("laplace3d", 3, (4, 4, 4), 1200)])
def test_kernel_bases_against_bruteforce_svd(kind, d, grid, n):
    """§2.4: the far-field block row's error after projection onto U_i lies between
    sigma_{k+1}(A(I_i, F_i)) and a randomized range-finder bound (rho_i weights the tags)."""
    pts = inputs.uniform_points(n, d, seed=21)
    lo, hi = (0.0,) * d, (1.0,) * d
    tess = orc.tessellate(pts, grid, lo, hi)
    k = 6
    T, G, H = inputs.tagging_draws(tess["b"], orc.tag_columns(d, 3), n, k + 10, 22)
    res = orc.reconstruct_tag(pts, grid, lo, hi, kind, T, G, H, k, 10)
    op, off = res["op"], tess["offsets"]
    A = orc.dense_matrix(op)
    checked = 0
    for i in range(tess["b"]):
        F = orc.far_field(tess["nbrs"][i], tess["b"])
        if len(F) == 0:
            continue
        rows = np.arange(off[i], off[i + 1])
        cols = np.concatenate([np.arange(off[c], off[c + 1]) for c in F])
        far = A[np.ix_(rows, cols)]
        s = np.linalg.svd(far, compute_uv=False)
        Ui = res["U"][rows, :res["ranks"][i]]
        e2 = np.linalg.norm(far - Ui @ (Ui.T @ far), 2)
        tail = s[k] if len(s) > k else 0.0
        assert e2 >= tail * (1 - 1e-10)
        m_i = len(rows)
        bound = 10 * res["rho"][i] * math.sqrt(k + 10) * math.sqrt(m_i) * max(tail, 1e-300) + 1e-13 * s[0]
        assert e2 <= bound, (i, e2, tail)
        checked += 1
    assert checked > 0


def test_algorithm3_basic_gives_the_same_subspaces():
    """Algorithm 3 (plain per-box randomized range finder) spans the same U_i, V_i on exact input."""
    pts, owner, A, res = _exact_case((4, 4), 40, 5, 3, seed=500)
    tess, op = res["tess"], res["op"]
    Ub, Vb, ks = orc.basic_bases(op, tess, 5, 15, np.random.default_rng(501))
    off = tess["offsets"]
    for i in range(tess["b"]):
        rows = slice(off[i], off[i + 1])
        P1 = res["U"][rows] @ res["U"][rows].T
        P2 = Ub[rows] @ Ub[rows].T
        assert np.abs(P1 - P2).max() < 1e-11
        Q1 = res["V"][rows] @ res["V"][rows].T
        Q2 = Vb[rows] @ Vb[rows].T
        assert np.abs(Q1 - Q2).max() < 1e-11


# ----------------------------------------------------- matvec counts (P3)

def test_matvec_counts_from_the_paper():
    """§4.2: 2 (3^d+1+e) r for step I, constant in N; Table 1: b k and 3^d m for steps II, III."""
    rows = []
    with open(os.path.join(GOLDEN, "matvec_counts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(v) for v in line.split()])
    ran = 0
    for d, e, k, p, b, m, s1, s2, s3 in rows:
        ell = orc.tag_columns(d, e)
        assert 2 * ell * (k + p) == s1
        if b == 173:
            # §7.1: reconstruct_tag needs 8.3x fewer matvecs than forming A (N = 100,000)
            assert abs(100000 / (s1 + s2 + s3) - 8.3) < 0.01
            continue
        n_side = round(b ** (1.0 / d))
        grid = (n_side,) * d
        pts, owner = inputs.box_points(grid, m, seed=600 + d)
        A = inputs.exact_ublr_matrix(owner, k, 601)
        tess = orc.tessellate(pts, grid, (0.0,) * d, (1.0,) * d)
        T, G, H = inputs.tagging_draws(tess["b"], ell, len(pts), k + p, 602)
        res = orc.reconstruct_tag(pts, grid, (0.0,) * d, (1.0,) * d, "dense", T, G, H, k, p, dense=A)
        assert res["matvecs"] == (s1, s2, s3)
        ran += 1
    assert ran >= 3


def test_stage_one_matvecs_do_not_grow_with_n():
    """§4.2 / §7.1: the number of step-I samples is independent of the problem size."""
    counts = set()
    for n in (300, 1200):
        pts = inputs.uniform_points(n, 2, seed=n)
        tess = orc.tessellate(pts, (5, 5), (0, 0), (1, 1))
        T, G, H = inputs.tagging_draws(25, 13, n, 8, 1)
        op = orc.make_operator("laplace2d", pts, tess)
        op.apply(orc.extended_test_matrix(T, G, tess))
        op.apply(orc.extended_test_matrix(T, H, tess), adjoint=True)
        counts.add(op.matvecs)
    assert counts == {2 * 13 * 8}


# ------------------------------------------------- planted mistakes (on CPU)

def _recovery_error(monkeypatch_fn=None):
    pts, owner = inputs.box_points((4, 4), 30, 700)
    A = inputs.exact_ublr_matrix(owner, 4, 701)
    tess = orc.tessellate(pts, (4, 4), (0, 0), (1, 1))
    T, G, H = inputs.tagging_draws(16, 13, len(pts), 14, 702)
    res = orc.reconstruct_tag(pts, (4, 4), (0, 0), (1, 1), "dense", T, G, H, 4, 10, dense=A)
    perm = res["tess"]["perm"]
    As = A[np.ix_(perm, perm)]
    return np.linalg.norm(As - orc.assemble(res)) / np.linalg.norm(As)


def test_power_method_accuracy_estimate():
    """§7's accuracy measure ||A - A_uBLR||_2 / ||A||_2 by 20 power iterations: exact on a
    closed form (singular values known), and within a few per cent of the dense 2-norms on a
    small Laplace compression."""
    rng = np.random.default_rng(777)
    n = 40
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    D = Q1 @ np.diag(np.r_[3.0, 1.0, np.linspace(0.5, 0.0, n - 2)]) @ Q2.T   # ||D||_2 = 3
    A = Q2 @ np.diag(np.r_[2.0, np.full(n - 1, 0.25)]) @ Q1.T               # ||A||_2 = 2
    est = orc.power_method_relerr(lambda x: D @ x, lambda x: D.T @ x, lambda x: A @ x,
                                  lambda x: A.T @ x, n, rng.standard_normal(n))
    assert abs(est - 1.5) < 1e-9, est
    # a tagged compression of the 2-D Laplace kernel
    pts = inputs.uniform_points(900, 2, seed=778)
    grid, k = (4, 4), 6
    T, G, H = inputs.tagging_draws(16, orc.tag_columns(2, 3), 900, k + 10, seed=779)
    res = orc.reconstruct_tag(pts, grid, (0.0, 0.0), (1.0, 1.0), "laplace2d", T, G, H, k, 10)
    Ad = orc.dense_matrix(orc.KernelOperator("laplace2d", pts[res["tess"]["perm"]]))
    Dd = Ad - orc.assemble(res)
    exact = np.linalg.norm(Dd, 2) / np.linalg.norm(Ad, 2)
    est = orc.power_method_relerr(lambda x: Dd @ x, lambda x: Dd.T @ x, lambda x: Ad @ x,
                                  lambda x: Ad.T @ x, 900, rng.standard_normal(900))
    assert 0.0 < exact < 1e-2
    assert abs(est / exact - 1.0) < 0.05, (est, exact)


def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible slip in the oracle breaks the exact-recovery pin by orders of magnitude."""
    assert _recovery_error() < 1e-12
    real_decode = orc.decode

    def decode_no_projection(T, tess):          # dropped the null-space projection
        z, tau, rho = real_decode(T, tess)
        w = np.ones(T.shape[1]) / math.sqrt(T.shape[1])
        z = z + 0.1 * w
        return z, T @ z.T, rho
    monkeypatch.setattr(orc, "decode", decode_no_projection)
    assert _recovery_error() > 1e-6
    monkeypatch.undo()

    real_ext = orc.extended_test_matrix

    def ext_wrong_index(T, G, tess):             # tags of the wrong box
        return real_ext(np.roll(T, 1, axis=0), G, tess)
    calls = {"n": 0}

    def ext_wrong_second(T, G, tess):
        calls["n"] += 1
        return ext_wrong_index(T, G, tess) if calls["n"] == 2 else real_ext(T, G, tess)
    monkeypatch.setattr(orc, "extended_test_matrix", ext_wrong_second)
    assert _recovery_error() > 1e-6
    monkeypatch.undo()

    real_coupling = orc.coupling

    def coupling_transposed(op, U, V, tess, k):  # Atilde_ji instead of Atilde_ij
        return real_coupling(op, U, V, tess, k).transpose(1, 0, 2, 3).copy()
    monkeypatch.setattr(orc, "coupling", coupling_transposed)
    assert _recovery_error() > 1e-6
    monkeypatch.undo()

    real_nf = orc.nearfield

    def nearfield_sign(op, U, At, V, tess, k):   # added the low-rank part instead of subtracting
        B = real_nf(op, U, At, V, tess, k)
        off = tess["offsets"]
        out = {}
        for (i, j), blk in B.items():
            mi = off[i + 1] - off[i]
            out[(i, j)] = blk + 2 * (U[off[i]:off[i + 1]] @ At[i, j] @ V[off[j]:off[j + 1]].T)[:mi]
        return out
    monkeypatch.setattr(orc, "nearfield", nearfield_sign)
    assert _recovery_error() > 1e-6


# ------------------------------------------------ §5.3 aspect-ratio minimisation

def _grid_and_T(d, grid, e, seed):
    rng = np.random.default_rng(seed)
    pts = rng.random((64 * int(np.prod(grid)), d))
    tess = orc.tessellate(pts, grid, (0.0,) * d, (1.0,) * d)
    T = rng.standard_normal((tess["b"], orc.tag_columns(d, e)))
    return tess, T


@pytest.mark.parametrize("d,grid,e", [(2, (6, 6), 3), (2, (7, 5), 1), (3, (4, 4, 4), 3)])
def test_minratio_never_worse_and_stays_in_the_null_space(d, grid, e):
    """§5.3: the optimised vector is a unit null vector of T(N_i, :), its aspect ratio
    (eq. aspect_ratio) is at most the projected direction's, and equal where the null
    space is a line."""
    tess, T = _grid_and_T(d, grid, e, seed=31 + d + e)
    z0, tau0, rho0 = orc.decode(T, tess)
    z, tau, rho = orc.decode_minratio(T, tess)
    for i in range(tess["b"]):
        N = tess["nbrs"][i]
        assert abs(np.linalg.norm(z[i]) - 1.0) < 1e-12
        assert np.abs(T[N] @ z[i]).max() < 1e-12
        F = orc.far_field(N, tess["b"])
        a = np.abs(T[F] @ z[i])
        assert abs(a.max() / a.min() - rho[i]) <= 1e-12 * rho[i]
        assert rho[i] <= rho0[i] * (1 + 1e-12)
        if T.shape[1] - len(N) == 1:
            assert abs(rho[i] - rho0[i]) <= 1e-10 * rho0[i]
    assert np.nanmean(rho) < np.nanmean(rho0)      # the optimisation does something


def test_minratio_matches_brute_force_on_two_dimensional_null_spaces():
    """With ell - |N_i| = 2 the null vectors are cos(t) x1 + sin(t) x2: a fine sweep of t
    inside the sign cell of the projected direction never beats the linear program and
    comes within the sweep's resolution of it."""
    tess, T = _grid_and_T(2, (7, 7), 1, seed=77)          # ell = 11, interior |N_i| = 9
    from scipy.linalg import null_space
    z0, tau0, _ = orc.decode(T, tess)
    _, _, rho = orc.decode_minratio(T, tess)
    t = np.linspace(0.0, 2 * np.pi, 200001)
    checked = 0
    for i in range(tess["b"]):
        N = tess["nbrs"][i]
        if len(N) != 9:
            continue
        F = orc.far_field(N, tess["b"])
        X = null_space(T[N])
        sigma = np.sign(tau0[i, F])
        def ratio(tt):
            sg = ((T[F] @ X) @ np.vstack([np.cos(tt), np.sin(tt)])) * sigma[:, None]
            r_ = sg.max(axis=0) / sg.min(axis=0)
            r_[~(sg > 0).all(axis=0)] = np.inf
            return r_
        coarse = ratio(t)
        j = int(np.argmin(coarse))
        fine = np.linspace(t[max(j - 2, 0)], t[min(j + 2, len(t) - 1)], 200001)
        best = min(coarse.min(), ratio(fine).min())   # the ratio has a kink at the optimum
        assert best >= rho[i] * (1 - 1e-9)
        assert best <= rho[i] * (1 + 1e-7)
        checked += 1
    assert checked >= 9


def test_minratio_keeps_exact_recovery():
    """The choice of null vector does not matter for exactness: with the §5.3 vectors an
    exactly uniform BLR matrix is still reconstructed to roundoff."""
    grid, per_box, k, e, seed = (4, 4), 64, 8, 3, 140
    pts, owner = inputs.box_points(grid, per_box, seed)
    A = inputs.exact_ublr_matrix(owner, k, seed + 1)
    tess = orc.tessellate(pts, grid, (0.0, 0.0), (1.0, 1.0))
    T, G, H = inputs.tagging_draws(tess["b"], orc.tag_columns(2, e), len(pts), k + 10, seed + 2)
    res = orc.reconstruct_tag(pts, grid, (0.0, 0.0), (1.0, 1.0), "dense", T, G, H, k, 10, dense=A,
                              zrule="minratio")
    perm = res["tess"]["perm"]
    As = A[np.ix_(perm, perm)]
    err = np.linalg.norm(As - orc.assemble(res)) / np.linalg.norm(As)
    assert err <= 1e-12, err
    _, _, rho0 = orc.decode(T, tess)
    assert np.nanmax(res["rho"] / rho0) <= 1 + 1e-12
