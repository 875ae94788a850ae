"""The near-field operation count bench.py reports (the numerator of its tensor
roofline line) against the oracle's definition of Method 3: the same near pairs
and the same (target, target corner, source corner) head-block applications
that oracle.interp.Interp.near_field_rows sums, counted on the oracle's own
neighbour tables and grids."""
import numpy as np
import pytest

import bench
from oracle import interp as oi
from paper_1602_01863_gb300 import synth


def oracle_counts(n, nd, width, scheme):
    I = oi.Interp(synth.draw_model(3, 1, 2), n, nd, scheme=scheme, width=width, build_dense_kc=False)
    L = n * nd
    g = I.dense.gint
    lin = {tuple(x): i for i, x in enumerate(g)}
    R2 = oi.near_radius2(width, nd)
    rad = int(np.floor(np.sqrt(R2)))
    offs = [np.array((a, b, c)) for a in range(-rad, rad + 1) for b in range(-rad, rad + 1)
            for c in range(-rad, rad + 1) if a * a + b * b + c * c <= R2]
    cell0 = [kd for kd in range(I.Nk) if kd // I.Ndiv == 0]          # coarse-major order: cell 0
    pairs = heads = 0
    for kd in cell0:
        reached = set()
        for d in offs:
            kp = lin[tuple(np.mod(g[kd] + d, L))]
            for lp in range(8):
                if I.f[kp, lp] != 0.0:
                    pairs += 1
                    reached.add(int(I.corner[kp, lp]))
        heads += sum(1 for l in range(8) if I.f[kd, l] != 0.0) * len(reached)
    return pairs, heads, I.Nkc


@pytest.mark.parametrize("n,nd,width,scheme", [(5, 2, 1.0, "8nb"), (5, 3, 1.0, "8nb"), (6, 4, 1.0, "8nb"),
                                               (5, 2, 1.5, "8nb"), (5, 2, 1.0, "1nb")])
def test_near_field_work_matches_oracle_definition(n, nd, width, scheme):
    pairs, heads, nkc = oracle_counts(n, nd, width, scheme)
    t, nch = 2, 3
    w = bench.near_field_work(nd, width, t, nch, nkc, nb1=(scheme == "1nb"))
    assert w["near_pairs_per_cell"] == pairs
    assert w["head_blocks_per_cell"] == heads
    assert w["useful_flops"] == nkc * nch * (pairs * 2 * (2 * t) * 2 + heads * 2 * t * t * 8)
