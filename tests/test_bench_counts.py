"""The near-field operation count bench.py reports (the numerator of its tensor
roofline line) against the oracle's definition of Method 3.

Two pins:
  * the near pairs and (target, target corner, source corner) head-block
    applications bench.py enumerates are the ones oracle.interp.Interp.near_field_rows
    sums, counted on the oracle's own neighbour tables and grids;
  * the flops: a direct execution of the factored form of the Method-3
    correction (Sec. 4, Eq. diverg) -- y1 and z accumulated pair by pair, then
    the head block applied once to y1 - h_head(q_c) z for each target corner --
    counts the real additions and multiplications it performs while it computes
    the correction, the result is checked against the oracle's pair-by-pair
    correction, and bench.near_field_work must give the same count."""
import numpy as np
import pytest

import bench
from oracle import interp as oi
from oracle import model as om
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
def test_near_field_pairs_and_heads_match_oracle_definition(n, nd, width, scheme):
    pairs, heads, nkc = oracle_counts(n, nd, width, scheme)
    w = bench.near_field_work(nd, width, 2, 3, nkc, nb1=(scheme == "1nb"))
    assert w["near_pairs_per_cell"] == pairs
    assert w["head_blocks_per_cell"] == heads


def counted_factored_near_field(I, psi, cell):
    """The factored Method-3 correction of the targets of one coarse cell,
    executed entry by entry with a count of the real flops performed:
    a complex entry times a real scalar added to a sum is 2 multiplies and 2
    adds; a complex multiply-add is 4 multiplies and 4 adds."""
    n, nd, L, t = I.n, I.nd, I.n * I.nd, I.t
    kap = I.model.kappa
    g, cg = I.dense.gint, I.coarse.gint
    lin = {tuple(x): i for i, x in enumerate(g)}
    R2 = oi.near_radius2(I.width, nd)
    rad = int(np.floor(np.sqrt(R2)))
    offs = [(a, b, c) for a in range(-rad, rad + 1) for b in range(-rad, rad + 1)
            for c in range(-rad, rad + 1) if a * a + b * b + c * c <= R2]
    P = psi.reshape(I.Nk, I.nv, I.nc)
    alpha = -(I.model.e_k / I.Nkc) * 4 * np.pi / I.model.eps_inf
    flops = 0
    targets = [kd for kd in range(I.Nk) if kd // I.Ndiv == cell]
    out = np.zeros((len(targets), t), dtype=np.complex128)
    for j, kd in enumerate(targets):
        y1, z = {}, {}
        for d in offs:
            kp = lin[tuple(np.mod(g[kd] + np.array(d), L))]
            h = om.h_head(d, L, kap)
            for lp in range(8):
                if I.f[kp, lp] == 0.0:
                    continue
                s = int(I.corner[kp, lp])
                x = (I.f[kp, lp] * (I.Dv[kp, lp].conj() @ P[kp] @ I.Dc[kp, lp].T)).reshape(-1)
                y1[s] = y1.get(s, 0) + h * x
                z[s] = z.get(s, 0) + 1.0 * x
                flops += 2 * (4 * t)                       # t complex x real multiply-adds, twice
        for l in range(8):
            if I.f[kd, l] == 0.0:
                continue
            a = int(I.corner[kd, l])
            u = np.zeros(t, dtype=np.complex128)
            for s in y1:
                hc = om.h_head(tuple(cg[a] - cg[s]), n, kap)
                w = y1[s] - hc * z[s]
                flops += 4 * t                             # t complex scalings and subtractions
                Ov = om.overlap_v(I.coarse.Uv[a], I.coarse.Uv[s])
                Oc = om.overlap_c(I.coarse.Uc[a], I.coarse.Uc[s])
                A = alpha * np.einsum("vw,cd->vcwd", Ov, Oc).reshape(t, t)
                u += A @ w
                flops += 8 * t * t                         # t x t complex multiply-adds
            out[j] += I.f[kd, l] * (I.Dv[kd, l].T @ u.reshape(I.nv, I.nc) @ I.Dc[kd, l].conj()).reshape(-1)
    return targets, out / I.Ndiv, flops


@pytest.mark.parametrize("nv,nc,n,nd", [(1, 2, 4, 2), (2, 2, 4, 3)])
def test_near_field_flops_are_those_of_the_factored_form(nv, nc, n, nd):
    I = oi.Interp(synth.draw_model(19, nv, nc), n, nd, width=1.0, build_dense_kc=False)
    psi = synth.random_vectors(8, I.N)
    targets, got, flops = counted_factored_near_field(I, psi, 0)
    ref = I.near_field_rows(psi, np.array(targets))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()          # it computes the correction
    nch = 3
    w = bench.near_field_work(nd, 1.0, I.t, nch, I.Nkc)
    assert w["useful_flops"] == flops * nch * I.Nkc
