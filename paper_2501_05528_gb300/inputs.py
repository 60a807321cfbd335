"""Seeded synthetic inputs for tagged uniform-BLR compression.

This module only draws random data.  It holds none of the compression
method's arithmetic, and both the CUDA library and the CPU oracle take what it
returns as plain inputs:

* point sets shaped like the integral-equation workloads (§7.1: i.i.d.
  uniform points in the unit square; a jittered lattice in the unit cube);
* the Gaussian tagging matrix ``T`` (b x ell, §4.1 eq. tagmat) and the
  Gaussian blocks ``G``, ``H`` that Algorithm 2 draws once per box.  They are
  drawn per point in the caller's original point order (N x r); box i's block
  ``G_i`` is the rows of ``G`` that belong to box i, in their original order;
* an exactly uniform BLR test matrix (every far block is ``U_i C_ij V_j^T``
  with shared orthonormal bases, every near block dense Gaussian), whose
  compression must be exact up to rounding (§2.5, eq. uniformBLRfull).

Every generator is a pure function of its arguments and seed (numpy's PCG64).
"""
from __future__ import annotations

import numpy as np


def uniform_points(n: int, d: int, seed: int) -> np.ndarray:
    """n points drawn i.i.d. uniform in [0,1)^d, shape (n, d), float64."""
    rng = np.random.default_rng(seed)
    return rng.random((n, d))


def jittered_lattice(n_side: int, d: int, jitter: float, seed: int) -> np.ndarray:
    """Cell centres of an n_side^d lattice in [0,1]^d moved by U[-jitter*h, jitter*h] per axis.

    h = 1/n_side.  With jitter < 0.5 every point stays inside its own cell, so
    a box grid whose side divides n_side holds the same number of points in
    every box.  Points are returned in a random order (shape (n_side^d, d)).
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / n_side
    axes = [np.arange(n_side, dtype=np.float64)] * d
    cells = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, d)
    pts = (cells + 0.5) * h + rng.uniform(-jitter * h, jitter * h, size=cells.shape)
    return pts[rng.permutation(len(pts))]


def box_points(grid, per_box: int, seed: int, margin: float = 0.05):
    """Exactly ``per_box`` points inside every box of a regular grid on [0,1]^d.

    Returns (points, box_coords): points (N, d) in a random order, and for each
    point the integer grid coordinates (N, d) of the box it was drawn in.  Points
    keep a relative ``margin`` away from box faces.
    """
    rng = np.random.default_rng(seed)
    grid = [int(g) for g in grid]
    d = len(grid)
    nbox = int(np.prod(grid))
    coords = np.stack(np.unravel_index(np.arange(nbox), grid, order="F"), axis=-1)
    h = 1.0 / np.asarray(grid, dtype=np.float64)
    pts, owner = [], []
    for c in coords:
        u = rng.uniform(margin, 1.0 - margin, size=(per_box, d))
        pts.append((c + u) * h)
        owner.append(np.repeat(c[None, :], per_box, axis=0))
    pts = np.concatenate(pts)
    owner = np.concatenate(owner)
    order = rng.permutation(len(pts))
    return pts[order], owner[order]


def tagging_draws(b: int, ell: int, n: int, r: int, seed: int):
    """Gaussian T (b x ell) and Gaussian G, H (n x r), in that draw order."""
    rng = np.random.default_rng(seed)
    T = rng.standard_normal((b, ell))
    G = rng.standard_normal((n, r))
    H = rng.standard_normal((n, r))
    return T, G, H


def exact_ublr_matrix(box_coords: np.ndarray, k: int, seed: int) -> np.ndarray:
    """A dense N x N matrix that is exactly uniform BLR of block rank k.

    ``box_coords`` gives each point's integer box coordinates (as returned by
    :func:`box_points`); rows and columns follow that (original) point order.
    Two boxes are near when their coordinates differ by at most one on every
    axis.  Near blocks are dense N(0,1); a far block (i, j) is
    ``U_i C_ij V_j^T`` with U_i, V_j the Q factors of Gaussian m_i x k matrices
    and C_ij ~ N(0,1) * 2^-|i-j| (i, j = column-major box indices).
    """
    rng = np.random.default_rng(seed)
    n, d = box_coords.shape
    shape = box_coords.max(axis=0) + 1
    lin = np.ravel_multi_index(tuple(box_coords.T), tuple(shape), order="F")
    nbox = int(np.prod(shape))
    members = [np.flatnonzero(lin == i) for i in range(nbox)]
    U = [np.linalg.qr(rng.standard_normal((len(mb), k)))[0] for mb in members]
    V = [np.linalg.qr(rng.standard_normal((len(mb), k)))[0] for mb in members]
    cells = np.stack(np.unravel_index(np.arange(nbox), tuple(shape), order="F"), axis=-1)
    A = np.empty((n, n))
    for i in range(nbox):
        for j in range(nbox):
            rows, cols = members[i], members[j]
            if np.max(np.abs(cells[i] - cells[j])) <= 1:
                blk = rng.standard_normal((len(rows), len(cols)))
            else:
                C = rng.standard_normal((k, k)) * 2.0 ** (-abs(i - j))
                blk = U[i] @ C @ V[j].T
            A[np.ix_(rows, cols)] = blk
    return A


# Workload recipes (sizes, distributions and seeds of the benchmark cases).
def workload(name: str):
    """Return a dict describing one named synthetic workload.

    Keys: d, grid, lo, hi, points, k, p, e, kernel ('laplace2d', 'laplace3d' or
    'dense'), dense (the matrix for 'dense'), seed.
    """
    if name == "exact_ublr_2d_n1024":
        pts, owner = box_points((4, 4), 64, seed=0x7A660001)
        A = exact_ublr_matrix(owner, k=8, seed=0x7A660101)
        return dict(d=2, grid=(4, 4), lo=(0.0, 0.0), hi=(1.0, 1.0), points=pts,
                    k=8, p=10, e=3, kernel="dense", dense=A, seed=0x7A660201)
    if name == "laplace2d_n65536":
        pts = uniform_points(65536, 2, seed=0x7A660002)
        return dict(d=2, grid=(16, 16), lo=(0.0, 0.0), hi=(1.0, 1.0), points=pts,
                    k=32, p=10, e=3, kernel="laplace2d", dense=None, seed=0x7A660202)
    if name == "laplace3d_n262144":
        pts = jittered_lattice(64, 3, 0.25, seed=0x7A660003)
        return dict(d=3, grid=(8, 8, 8), lo=(0.0,) * 3, hi=(1.0,) * 3, points=pts,
                    k=64, p=10, e=3, kernel="laplace3d", dense=None, seed=0x7A660203)
    raise KeyError(name)
