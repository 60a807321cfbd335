"""Accuracy metrics between two compressed uniform-BLR representations.

Used by the parity tests and by the benchmark to state the error of a
compression against a reference one; none of the compression arithmetic lives
here.  For a far block the two low-rank products are expressed in a joint
orthonormal basis: with Q_U = orth([U1, U2]) and Q_V = orth([V1, V2]),
  ||U1 A1 V1^T - U2 A2 V2^T||_F = ||C1 A1 D1^T - C2 A2 D2^T||_F,
  C = Q_U^T U, D = Q_V^T V  (exact, as the columns of U lie in range(Q_U)),
a small dense difference with no cancellation; near blocks are compared
densely.  The N x N matrices are never formed.
"""
from __future__ import annotations

import numpy as np


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def near_pairs(nbr, nnbr, s3):
    out = []
    for i in range(len(nnbr)):
        for s in range(int(nnbr[i])):
            out.append((i, int(nbr[i * s3 + s]), s))
    return out


def ublr_difference(off, nbr, nnbr, s3, ranks, rep1, rep2, pairs=None):
    """||A1 - A2||_F / ||A2||_F for two representations (U, V, At[b,b,k,k], B dict).

    rep = dict(U=(n,k), V=(n,k), At=(b,b,k,k), B={(i,j): m_i x m_j}).  Both use
    the same tessellation (checked bit-exactly elsewhere).  ``pairs`` restricts
    the sum to a sample of (i, j) box pairs.
    """
    b = len(off) - 1
    near = {(i, j) for (i, j, _) in near_pairs(nbr, nnbr, s3)}
    if pairs is None:
        pairs = [(i, j) for i in range(b) for j in range(b)]
    joint_u, joint_v = {}, {}

    def joint(cache, M1, M2, key):
        if key not in cache:
            Q = np.linalg.qr(np.hstack([M1, M2]))[0] if M1.size else np.zeros((M1.shape[0], 0))
            cache[key] = (Q.T @ M1, Q.T @ M2)
        return cache[key]

    num = 0.0
    den = 0.0
    for (i, j) in pairs:
        ri = slice(off[i], off[i + 1])
        rj = slice(off[j], off[j + 1])
        ki, kj = int(ranks[i]), int(ranks[j])
        U1, U2 = rep1["U"][ri, :ki], rep2["U"][ri, :ki]
        V1, V2 = rep1["V"][rj, :kj], rep2["V"][rj, :kj]
        A1 = rep1["At"][i, j][:ki, :kj]
        A2 = rep2["At"][i, j][:ki, :kj]
        if (i, j) in near:
            D1 = U1 @ A1 @ V1.T + rep1["B"][(i, j)]
            D2 = U2 @ A2 @ V2.T + rep2["B"][(i, j)]
            num += np.sum((D1 - D2) ** 2)
            den += np.sum(D2 ** 2)
        elif ki and kj:
            C1, C2 = joint(joint_u, U1, U2, i)
            E1, E2 = joint(joint_v, V1, V2, j)
            num += np.sum((C1 @ A1 @ E1.T - C2 @ A2 @ E2.T) ** 2)
            den += np.sum(A2 ** 2)
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))


def blocks_from_flat(bnear, nf_off, nbr, nnbr, off, s3):
    """Split the flat near-field array into {(i, j): m_i x m_j} blocks."""
    out = {}
    for i in range(len(nnbr)):
        mi = int(off[i + 1] - off[i])          # Python ints: offsets exceed 2^31 at scale
        for s in range(int(nnbr[i])):
            j = int(nbr[i * s3 + s])
            mj = int(off[j + 1] - off[j])
            st = int(nf_off[i * s3 + s])
            out[(i, j)] = np.asarray(bnear[st:st + mi * mj]).reshape(mi, mj)
    return out


def padded_neighbours(nbrs, s3):
    b = len(nbrs)
    arr = -np.ones(b * s3, dtype=np.int64)
    cnt = np.zeros(b, dtype=np.int64)
    for i, lst in enumerate(nbrs):
        arr[i * s3:i * s3 + len(lst)] = lst
        cnt[i] = len(lst)
    return arr, cnt


def ublr_difference_all(off, nbr, nnbr, s3, ranks, rep1, rep2):
    """ublr_difference over every box pair, vectorised over column boxes.

    Far blocks use the joint-basis identity with all k columns of each basis
    (columns beyond k_i are zero in both representations, so they add nothing).
    """
    b = len(off) - 1
    k = rep1["U"].shape[1]
    near = {(i, j) for (i, j, _) in near_pairs(nbr, nnbr, s3)}
    C1 = np.zeros((b, 2 * k, k))
    C2 = np.zeros((b, 2 * k, k))
    E1 = np.zeros((b, 2 * k, k))
    E2 = np.zeros((b, 2 * k, k))
    for i in range(b):
        ri = slice(off[i], off[i + 1])
        for (X1, X2, D1, D2) in ((rep1["U"], rep2["U"], C1, C2), (rep1["V"], rep2["V"], E1, E2)):
            M = np.hstack([X1[ri], X2[ri]])
            if M.shape[0] == 0:
                continue
            Q = np.linalg.qr(M)[0]
            w = Q.shape[1]
            D1[i, :w] = Q.T @ X1[ri]
            D2[i, :w] = Q.T @ X2[ri]
    num = 0.0
    den = 0.0
    farmask = np.ones((b, b), dtype=bool)
    for (i, j) in near:
        farmask[i, j] = False
    for i in range(b):
        js = np.flatnonzero(farmask[i])
        if len(js):
            T1 = np.einsum("ab,jbc,jdc->jad", C1[i], rep1["At"][i, js], E1[js], optimize=True)
            T2 = np.einsum("ab,jbc,jdc->jad", C2[i], rep2["At"][i, js], E2[js], optimize=True)
            num += float(np.sum((T1 - T2) ** 2))
            den += float(np.sum(rep2["At"][i, js] ** 2))
    for (i, j) in near:
        ri = slice(off[i], off[i + 1])
        rj = slice(off[j], off[j + 1])
        D1 = rep1["U"][ri] @ rep1["At"][i, j] @ rep1["V"][rj].T + rep1["B"][(i, j)]
        D2 = rep2["U"][ri] @ rep2["At"][i, j] @ rep2["V"][rj].T + rep2["B"][(i, j)]
        num += float(np.sum((D1 - D2) ** 2))
        den += float(np.sum(D2 ** 2))
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))
