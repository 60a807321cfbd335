"""The uniform-BLR comparison metric is exact under basis rotations and sees small changes."""
import numpy as np

from oracle import tagging as orc
from paper_2501_05528_gb300 import inputs
from paper_2501_05528_gb300 import metrics


def _result():
    pts = inputs.uniform_points(400, 2, seed=31)
    T, G, H = inputs.tagging_draws(16, 13, 400, 14, seed=32)
    return orc.reconstruct_tag(pts, (4, 4), (0, 0), (1, 1), "laplace2d", T, G, H, 4, 10)


def test_metric_invariant_under_rotation_and_sensitive():
    res = _result()
    tess = res["tess"]
    off = tess["offsets"]
    nbr, cnt = metrics.padded_neighbours(tess["nbrs"], 9)
    rep = dict(U=res["U"], V=res["V"], At=res["coupling"], B=res["nearfield"])
    rng = np.random.default_rng(0)
    U2, At2 = res["U"].copy(), res["coupling"].copy()
    for i in range(16):
        ki = res["ranks"][i]
        Q = np.linalg.qr(rng.standard_normal((ki, ki)))[0]
        U2[off[i]:off[i + 1], :ki] = res["U"][off[i]:off[i + 1], :ki] @ Q
        for j in range(16):
            At2[i, j][:ki] = Q.T @ res["coupling"][i, j][:ki]
    rot = dict(rep, U=U2, At=At2)
    assert metrics.ublr_difference(off, nbr, cnt, 9, res["ranks"], rot, rep) < 1e-14
    assert metrics.ublr_difference_all(off, nbr, cnt, 9, res["ranks"], rot, rep) < 1e-14
    A3 = res["coupling"].copy()
    A3[0, 15] *= 1 + 1e-8
    d = metrics.ublr_difference(off, nbr, cnt, 9, res["ranks"], dict(rep, At=A3), rep)
    full = orc.assemble(res)
    p2 = dict(res, coupling=A3)
    ref = np.linalg.norm(orc.assemble(p2) - full) / np.linalg.norm(full)
    assert abs(d - ref) <= 1e-3 * ref
    d_all = metrics.ublr_difference_all(off, nbr, cnt, 9, res["ranks"], dict(rep, At=A3), rep)
    assert abs(d_all - ref) <= 1e-3 * ref
