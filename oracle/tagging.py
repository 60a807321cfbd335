"""FP64 CPU oracle for tagged uniform-BLR compression (reconstruct_tag, Table 1).

TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, readable statement of
what the CUDA library computes.  Only the tests, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline leg may import it; the library never does.
It shares no code with the CUDA path: numpy (and its LAPACK/BLAS) is the only
dependency, plus scipy's linear-programming solver for the §5.3 aspect-ratio
minimisation, and every quantity is float64.

Steps, in the paper's order (Table 1, ``reconstruct_tag``):

1. geometry: boxes of a regular grid, neighbour lists N_i (§2.5);
2. tagging matrix T and extended test matrices Omega, Psi (§4.1, eq. tagmat,
   eq. extend_test_mat; Algorithm 2);
3. sketches Y = A Omega, Z = A^T Psi (Algorithm 2, "Sketch");
4. tag decode z_i in null(T(N_i, :)) (§4.1 eq. tagsubmat; §5.3 for ell > 3^d+1),
   projected tags tau_i = T z_i and aspect ratio rho_i (§5.1 eq. aspect_ratio);
5. combine S_i = sum_j z_ij Y_j(I_i, :) and R_i likewise (Algorithm 2),
   whose near-field rows cancel (§4.1 eq. projected_tags);
6. U_i = col(S_i, k), V_i = col(R_i, k) (§2.3, §2.4);
7. coupling Atilde = U^T (A V) (§2.5 eq. uniformBLRfull; Table 1 step 2);
8. near field B from the 3^d identity probes (§6.1 eq. sparse_struct_ids;
   Table 1 step 3), B_ij for i in N_j (§2.5 eq. discrepancymatrix).

Readings taken where the paper leaves a choice (each is stated where used):
* z_i = the unit vector of null(T(N_i,:)) closest to the all-ones direction,
  i.e. the normalised orthogonal projection of 1/sqrt(ell) onto the null space;
* col(S, k) = the k dominant left singular vectors of S (randomized range
  finder truncation), each column signed so its largest-magnitude entry is
  positive (lowest index on ties); k_i = min(k, m_i), and 0 when box i has no
  far field;
* boxes are indexed column-major over grid coordinates (x fastest); points
  inside a box keep their input order; a coordinate on the upper face belongs
  to the last box;
* kernel matrices have a zero diagonal (§7.1).
"""
from __future__ import annotations

import itertools
import math

import numpy as np


# ---------------------------------------------------------------- geometry (§2.5)

def box_coordinates(points, grid, lo, hi):
    """Integer grid coordinates q_a = clamp(floor((x_a - lo_a)/(hi_a - lo_a) * n_a))."""
    points = np.asarray(points, dtype=np.float64)
    n, d = points.shape
    q = np.empty((n, d), dtype=np.int64)
    for a in range(d):
        t = (points[:, a] - lo[a]) / (hi[a] - lo[a]) * float(grid[a])
        q[:, a] = np.clip(np.floor(t), 0, grid[a] - 1).astype(np.int64)
    return q


def box_index(q, grid):
    """Column-major box index q_1 + n_1 (q_2 + n_2 q_3)."""
    idx = np.zeros(q.shape[:-1], dtype=np.int64)
    stride = 1
    for a in range(q.shape[-1]):
        idx = idx + q[..., a] * stride
        stride *= int(grid[a])
    return idx


def tessellate(points, grid, lo, hi):
    """Boxes, the stable box-major permutation, I_i ranges, N_i and colours.

    Returns a dict with
      perm     (N,)   original index of the p-th point in box-major order,
      offsets  (b+1,) I_i = perm[offsets[i]:offsets[i+1]],
      nbrs     list of ascending int arrays, N_i (box i itself included),
      colour   (b,)   sum_a (q_a mod 3) 3^(a-1): boxes of one colour are never
                       neighbours of a common box twice (§6.1 identity probes),
      cell     (b, d) grid coordinates of each box.
    """
    grid = [int(g) for g in grid]
    d = len(grid)
    b = int(np.prod(grid))
    q = box_coordinates(points, grid, lo, hi)
    box = box_index(q, grid)
    perm = np.argsort(box, kind="stable")
    counts = np.bincount(box, minlength=b)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    cell = np.stack(np.unravel_index(np.arange(b), grid, order="F"), axis=-1)
    nbrs = []
    for i in range(b):
        # boxes share a boundary (or are i itself) iff their grid coordinates
        # differ by at most one on every axis
        cheb = np.max(np.abs(cell - cell[i]), axis=1)
        nbrs.append(np.flatnonzero(cheb <= 1))
    colour = np.zeros(b, dtype=np.int64)
    for a in range(d):
        colour += (cell[:, a] % 3) * 3 ** a
    return dict(perm=perm, offsets=offsets, nbrs=nbrs, colour=colour, cell=cell,
                grid=grid, d=d, b=b)


def far_field(nbrs_i, b):
    """F_i = [b] minus N_i."""
    mask = np.ones(b, dtype=bool)
    mask[nbrs_i] = False
    return np.flatnonzero(mask)


def tag_columns(d, e):
    """ell = 3^d + 1 + e tag columns (§4.1; §5.3 uses e extra columns, §7 uses e = 3)."""
    return 3 ** d + 1 + e


# ------------------------------------------------------------ operators (§7.1)

class KernelOperator:
    """The kernel matrix A(p, q) = K(x_p, x_q), zero diagonal, in box-major order.

    kind 'laplace2d': K = log |x - y|                 (§7.1)
    kind 'laplace3d': K = 1 / (4 pi |x - y|)
    Applies are blocked over rows; ``matvecs`` counts applied columns (§4.2).
    """

    def __init__(self, kind, points_sorted, row_block=512):
        self.kind = kind
        self.x = np.asarray(points_sorted, dtype=np.float64)
        self.n = len(self.x)
        self.row_block = row_block
        self.matvecs = 0

    def block(self, rows, cols):
        rows = np.asarray(rows)
        cols = np.asarray(cols)
        diff = self.x[rows][:, None, :] - self.x[cols][None, :, :]
        dist = np.sqrt(np.sum(diff * diff, axis=-1))
        with np.errstate(divide="ignore"):
            if self.kind == "laplace2d":
                K = np.log(dist)
            elif self.kind == "laplace3d":
                K = 1.0 / (4.0 * math.pi * dist)
            else:
                raise ValueError(self.kind)
        K[rows[:, None] == cols[None, :]] = 0.0
        return K

    def apply(self, X, adjoint=False):
        """A X (the kernels here are symmetric, so A^T X = A X)."""
        X = np.asarray(X, dtype=np.float64)
        self.matvecs += X.shape[1]
        Y = np.empty((self.n, X.shape[1]))
        allc = np.arange(self.n)
        for s in range(0, self.n, self.row_block):
            rows = np.arange(s, min(self.n, s + self.row_block))
            Y[rows] = self.block(rows, allc) @ X
        return Y


class DenseOperator:
    """An explicit matrix, given in box-major order, used as a black box."""

    def __init__(self, A_sorted):
        self.A = np.asarray(A_sorted, dtype=np.float64)
        self.n = self.A.shape[0]
        self.matvecs = 0

    def block(self, rows, cols):
        return self.A[np.ix_(np.asarray(rows), np.asarray(cols))]

    def apply(self, X, adjoint=False):
        self.matvecs += X.shape[1]
        return (self.A.T if adjoint else self.A) @ X


def make_operator(kind, points, tess, dense=None):
    perm = tess["perm"]
    if kind == "dense":
        return DenseOperator(np.asarray(dense)[np.ix_(perm, perm)])
    return KernelOperator(kind, np.asarray(points)[perm])


# --------------------------------------------- test matrices (§4.1, Algorithm 2)

def extended_test_matrix(T, G, tess):
    """Omega(I_i, j r : (j+1) r) = t_ij G_i  (eq. extend_test_mat), box-major rows.

    G holds one row per point in the original point order; G_i = G[I_i].
    """
    b, ell = T.shape
    n, r = G.shape
    perm, off = tess["perm"], tess["offsets"]
    Om = np.zeros((n, ell * r))
    for i in range(b):
        rows = np.arange(off[i], off[i + 1])
        Gi = G[perm[rows]]
        for j in range(ell):
            Om[rows, j * r:(j + 1) * r] = T[i, j] * Gi
    return Om


# ----------------------------------------------------- tag decode (§4.1, §5.1)

def decode(T, tess):
    """z_i in null(T(N_i, :)), projected tags tau_i = T z_i, aspect ratios rho_i.

    z_i is the normalised orthogonal projection of w = 1/sqrt(ell) onto
    null(T(N_i, :)) (a reading: for ell = 3^d+1 and an interior box the null
    space is a line and this is the paper's z up to sign; otherwise §5.3 leaves
    the choice open).  The projector onto the row space of T(N_i,:) comes from
    a reduced QR of T(N_i,:)^T (§2.2), so it does not depend on QR sign
    conventions.  rho_i follows eq. aspect_ratio over the far field F_i; it is
    nan when F_i is empty.
    """
    b, ell = T.shape
    z = np.zeros((b, ell))
    tau = np.zeros((b, b))
    rho = np.full(b, np.nan)
    w = np.ones(ell) / math.sqrt(ell)
    for i in range(b):
        Ti = T[tess["nbrs"][i], :]
        Q, _ = np.linalg.qr(Ti.T)            # ell x |N_i|, orthonormal
        zi = w - Q @ (Q.T @ w)
        zi /= np.linalg.norm(zi)
        z[i] = zi
        tau[i] = T @ zi
        F = far_field(tess["nbrs"][i], b)
        if len(F):
            a = np.abs(tau[i, F])
            rho[i] = a.max() / a.min()
    return z, tau, rho


def decode_minratio(T, tess):
    """§5.3: per box, the vector of null(T(N_i, :)) minimising the aspect ratio of
    eq. aspect_ratio, instead of the projected direction of `decode`.

    With X_i an orthonormal basis of the null space (s columns) and c_j = X_i^T t_j
    for j in F_i, a null vector X_i a has projected tags c_j^T a.  Reading (the
    paper optimises over spherical coordinates "over a convex region"): keep the
    signs sigma_j of `decode`'s projected tags; inside that sign cell the ratio
    max_j sigma_j c_j^T a / min_j sigma_j c_j^T a is scale invariant and quasi-convex,
    and its minimum is the linear program

        minimise rho   subject to   1 <= sigma_j c_j^T a <= rho   (j in F_i),

    over (a, rho) in R^(s+1).  z_i = X_i a / ||X_i a|| keeps the sign pattern, so
    tau_i = T z_i and rho_i = max |tau_i(F_i)| / min |tau_i(F_i)| equals the LP's rho.
    A one-dimensional null space (s = 1) or an empty far field leaves `decode`'s z.
    """
    from scipy.linalg import null_space
    from scipy.optimize import linprog
    z0, tau0, rho0 = decode(T, tess)
    b, ell = T.shape
    z, tau, rho = z0.copy(), tau0.copy(), rho0.copy()
    for i in range(b):
        F = far_field(tess["nbrs"][i], b)
        if not len(F):
            continue
        X = null_space(T[tess["nbrs"][i], :])
        s_dim = X.shape[1]
        if s_dim <= 1:
            continue
        sigma = np.sign(tau0[i, F])
        C = (T[F] @ X) * sigma[:, None]
        m = len(F)
        A_ub = np.vstack([np.hstack([-C, np.zeros((m, 1))]), np.hstack([C, -np.ones((m, 1))])])
        b_ub = np.concatenate([-np.ones(m), np.zeros(m)])
        c = np.zeros(s_dim + 1)
        c[-1] = 1.0
        res = linprog(c, A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * (s_dim + 1),
                      method="highs")
        if res.status != 0:
            raise RuntimeError(f"aspect-ratio LP failed for box {i}: {res.message}")
        zi = X @ res.x[:s_dim]
        zi /= np.linalg.norm(zi)
        z[i] = zi
        tau[i] = T @ zi
        a = np.abs(tau[i, F])
        rho[i] = a.max() / a.min()
    return z, tau, rho


# -------------------------------------------- combine and col (Algorithm 2, §2.3)

def combine(Y, z, tess, r):
    """S_i = sum_j z_ij Y_j(I_i, :), stacked box-major into an N x r array."""
    b, ell = z.shape
    off = tess["offsets"]
    S = np.zeros((Y.shape[0], r))
    for i in range(b):
        rows = slice(off[i], off[i + 1])
        for j in range(ell):
            S[rows] += z[i, j] * Y[rows, j * r:(j + 1) * r]
    return S


def signed_columns(U):
    """Flip each column so its largest-magnitude entry is positive (lowest index on ties)."""
    U = U.copy()
    for c in range(U.shape[1]):
        p = int(np.argmax(np.abs(U[:, c])))
        if U[p, c] < 0:
            U[:, c] = -U[:, c]
    return U


def col(S, k):
    """k orthonormal columns spanning the dominant range of S (§2.3, §2.4 step 4)."""
    if k == 0 or S.shape[0] == 0:
        return np.zeros((S.shape[0], 0))
    Us, _, _ = np.linalg.svd(S, full_matrices=False)
    return signed_columns(Us[:, :k])


def box_ranks(tess, k):
    """k_i = min(k, m_i), or 0 when box i has no far field."""
    b = tess["b"]
    m = np.diff(tess["offsets"])
    ks = np.minimum(k, m)
    for i in range(b):
        if len(far_field(tess["nbrs"][i], b)) == 0:
            ks[i] = 0
    return ks.astype(np.int64)


def bases(S, tess, k):
    """U (N x k, box-major rows) with U_i = col(S_i, k_i) in its first k_i columns."""
    off = tess["offsets"]
    ks = box_ranks(tess, k)
    U = np.zeros((S.shape[0], k))
    for i in range(tess["b"]):
        rows = slice(off[i], off[i + 1])
        U[rows, :ks[i]] = col(S[rows], ks[i])
    return U, ks


# ----------------------------------------- steps II and III (§6.1, Table 1)

def block_diagonal(U, tess, k):
    """diag(U_1, ..., U_b) as a dense N x (b k) matrix (§2.5)."""
    off = tess["offsets"]
    b = tess["b"]
    D = np.zeros((U.shape[0], b * k))
    for i in range(b):
        D[off[i]:off[i + 1], i * k:(i + 1) * k] = U[off[i]:off[i + 1]]
    return D


def coupling(op, U, V, tess, k):
    """Atilde = U^T (A V), as a (b, b, k, k) array (Table 1 step 2; b k matvecs)."""
    b = tess["b"]
    Ud = block_diagonal(U, tess, k)
    Vd = block_diagonal(V, tess, k)
    At = Ud.T @ op.apply(Vd)
    return At.reshape(b, k, b, k).transpose(0, 2, 1, 3).copy()


def identity_probe(tess, gamma, m):
    """Omega_B for colour gamma: I_{m_c} in rows I_c, columns 0:m_c, for every box c of that colour."""
    off = tess["offsets"]
    P = np.zeros((off[-1], m))
    for c in np.flatnonzero(tess["colour"] == gamma):
        mc = off[c + 1] - off[c]
        P[off[c]:off[c + 1], :mc] = np.eye(mc)
    return P


def nearfield(op, U, At, V, tess, k):
    """B_ij for every near pair (j in N_i), from the 3^d identity probes (eq. sparse_struct_ids).

    Y_B = (A - U Atilde V^T) Omega_B; B_ij = Y_B(I_i, 0:m_j) for the probe of
    box j's colour (Table 1 step 3, 3^d m matvecs).  Returns {(i, j): m_i x m_j}.
    """
    b = tess["b"]
    off = tess["offsets"]
    m = int(np.max(np.diff(off)))
    Ud = block_diagonal(U, tess, k)
    Vd = block_diagonal(V, tess, k)
    Atd = At.transpose(0, 2, 1, 3).reshape(b * k, b * k)
    B = {}
    for gamma in range(3 ** tess["d"]):
        P = identity_probe(tess, gamma, m)
        YB = op.apply(P) - Ud @ (Atd @ (Vd.T @ P))
        for i in range(b):
            for j in tess["nbrs"][i]:
                if tess["colour"][j] == gamma:
                    mj = off[j + 1] - off[j]
                    B[(i, int(j))] = YB[off[i]:off[i + 1], :mj].copy()
    return B


# ------------------------------------------------- reconstruct_tag (Table 1)

def reconstruct_tag(points, grid, lo, hi, kind, T, G, H, k, p=10, dense=None, zrule="project"):
    """Full compression A ~ U Atilde V^T + B with tagging bases (Table 1, middle column).

    ``T`` is b x ell with ell = 3^d + 1 + e; ``G``, ``H`` are N x (k + p) in the
    original point order.  ``zrule`` picks the null vector of each box: "project"
    (`decode`) or "minratio" (§5.3, `decode_minratio`).  Returns a dict of every
    intermediate and output and the matvec counts of the three steps.
    """
    tess = tessellate(points, grid, lo, hi)
    r = k + p
    assert G.shape[1] == r and H.shape[1] == r and T.shape[0] == tess["b"]
    op = make_operator(kind, points, tess, dense)
    Om = extended_test_matrix(T, G, tess)
    Ps = extended_test_matrix(T, H, tess)
    Y = op.apply(Om)
    Z = op.apply(Ps, adjoint=True)
    mv1 = op.matvecs
    z, tau, rho = (decode_minratio if zrule == "minratio" else decode)(T, tess)
    S = combine(Y, z, tess, r)
    R = combine(Z, z, tess, r)
    U, ks = bases(S, tess, k)
    V, _ = bases(R, tess, k)
    At = coupling(op, U, V, tess, k)
    mv2 = op.matvecs - mv1
    B = nearfield(op, U, At, V, tess, k)
    mv3 = op.matvecs - mv1 - mv2
    return dict(tess=tess, op=op, Omega=Om, Psi=Ps, Y=Y, Z=Z, z=z, tau=tau, rho=rho,
                S=S, R=R, U=U, V=V, ranks=ks, coupling=At, nearfield=B,
                matvecs=(mv1, mv2, mv3), k=k, r=r)


# ------------------------------------------- per-block definitions (sampling)

def sketch_rows(op, X, rows):
    """(A X)(rows, :) for a subset of rows, one block of A at a time."""
    return op.block(rows, np.arange(op.n)) @ X


def coupling_block(op, U, V, tess, i, j, ki, kj):
    """Atilde_ij = U_i^T A_ij V_j (§2.5 eq. uniformBLRblock, per block)."""
    off = tess["offsets"]
    Ri = np.arange(off[i], off[i + 1])
    Cj = np.arange(off[j], off[j + 1])
    return U[Ri, :ki].T @ op.block(Ri, Cj) @ V[Cj, :kj]


def nearfield_block(op, U, At, V, tess, i, j, k):
    """B_ij as the colour-gamma(j) identity probe returns it (eq. sparse_struct_ids):

    sum over boxes c with colour(c) = colour(j) of (A_ic - U_i Atilde_ic V_c^T),
    restricted to the first m_j columns (a box c with m_c < m_j adds nothing to
    columns m_c..m_j-1).
    """
    off = tess["offsets"]
    Ri = np.arange(off[i], off[i + 1])
    mj = off[j + 1] - off[j]
    out = np.zeros((len(Ri), mj))
    for c in np.flatnonzero(tess["colour"] == tess["colour"][j]):
        Cc = np.arange(off[c], off[c + 1])
        w = min(len(Cc), mj)
        blk = op.block(Ri, Cc) - U[Ri] @ At[i, c] @ V[Cc].T
        out[:, :w] += blk[:, :w]
    return out


def discrepancy_block(op, U, At, V, tess, i, j):
    """B_ij = A_ij - U_i Atilde_ij V_j^T exactly (eq. discrepancymatrix); a diagnostic."""
    off = tess["offsets"]
    Ri = np.arange(off[i], off[i + 1])
    Cj = np.arange(off[j], off[j + 1])
    return op.block(Ri, Cj) - U[Ri] @ At[i, j] @ V[Cj].T


# ------------------------------------------------------------ dense assembly

def assemble(res):
    """A_uBLR = U Atilde V^T + B as a dense box-major matrix (small N only)."""
    tess, k = res["tess"], res["k"]
    Ud = block_diagonal(res["U"], tess, k)
    Vd = block_diagonal(res["V"], tess, k)
    b = tess["b"]
    Atd = res["coupling"].transpose(0, 2, 1, 3).reshape(b * k, b * k)
    A = Ud @ Atd @ Vd.T
    off = tess["offsets"]
    for (i, j), blk in res["nearfield"].items():
        A[off[i]:off[i + 1], off[j]:off[j + 1]] += blk
    return A


def dense_matrix(op):
    """The operator's full matrix in box-major order (small N only)."""
    return op.block(np.arange(op.n), np.arange(op.n))


# ------------------------------------------------- accuracy (§7, power method)

def power_method_relerr(apply_diff, apply_diff_t, apply_a, apply_a_t, n, x0, iters=20):
    """||A - A_uBLR||_2 / ||A||_2, each norm by `iters` power iterations on M^T M (§7)."""
    def norm_est(f, ft):
        x = x0 / np.linalg.norm(x0)
        s = 0.0
        for _ in range(iters):
            y = ft(f(x))
            s = np.linalg.norm(y)
            if s == 0.0:
                return 0.0
            x = y / s
        return math.sqrt(s)
    return norm_est(apply_diff, apply_diff_t) / norm_est(apply_a, apply_a_t)


# ---------------------------------------------- Algorithm 3 (cross-check only)

def basic_bases(op, tess, k, r, rng, shared=None):
    """Algorithm 3: per box, a Gaussian test matrix zeroed on N_i, then col (2 b r matvecs).
    shared = (G, H), n x r in box-major order: every box uses G and H (zeroed on its N_i)
    instead of fresh draws from rng."""
    off = tess["offsets"]
    n = op.n
    U = np.zeros((n, k))
    V = np.zeros((n, k))
    ks = box_ranks(tess, k)
    for i in range(tess["b"]):
        if shared is None:
            Om = rng.standard_normal((n, r))
            Ps = rng.standard_normal((n, r))
        else:
            Om, Ps = shared[0].copy(), shared[1].copy()
        for j in tess["nbrs"][i]:
            Om[off[j]:off[j + 1]] = 0.0
            Ps[off[j]:off[j + 1]] = 0.0
        Y = op.apply(Om)
        Z = op.apply(Ps, adjoint=True)
        rows = slice(off[i], off[i + 1])
        U[rows, :ks[i]] = col(Y[rows], ks[i])
        V[rows, :ks[i]] = col(Z[rows], ks[i])
    return U, V, ks


def cofactor_null_vector(Ti):
    """For a (ell-1) x ell matrix, the signed cofactor vector c_j = (-1)^j det(Ti without column j).

    Ti c = 0 by Laplace expansion of det([t; Ti]) with t a copy of one row of Ti
    (§5.2 eq. cramers_rule, read with alternating signs).
    """
    n1, ell = Ti.shape
    assert n1 == ell - 1
    c = np.empty(ell)
    for j in range(ell):
        c[j] = (-1) ** j * np.linalg.det(np.delete(Ti, j, axis=1))
    return c


def all_neighbour_offsets(d):
    """The 3^d offsets in [-1, 1]^d (used by tests to enumerate stencils)."""
    return list(itertools.product((-1, 0, 1), repeat=d))
