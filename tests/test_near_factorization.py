"""The factorisation the tensor-core near field implements, in FP64 on the CPU,
against the oracle's pair-by-pair Method 3 correction.

Per coarse cell C and source slot s (a coarse point that is a corner of some
source point near a target of C), the kernel forms
    y1(k, s) = sum_{k'} h_head(q_d(k, k')) x(k', s),   z(k, s) = sum_{k'} x(k', s)
over the near source pairs (k', corner s) -- a pattern matrix times the
gathered rows x -- and then, for every active corner l of each target k,
    u(k, l) += alpha O^v(l, s) [y1 - h_head(q_c(l, s)) z] O^c(l, s)^T,
which the prolongation carries to the dense point.  Because h_head(q_c),
O^v and O^c depend only on the coarse pair (l, s), this regrouping of the
sum over near pairs (Sec. 4, Method 3; Eq. diverg) is exact: the GPU's
deviation from the oracle (a few 1e-3 of the correction) is TF32 rounding,
not an approximation of the method."""
import numpy as np
import pytest

from oracle import interp as oi
from oracle import model as om
from paper_1602_01863_gb300 import synth


def factorised_near_field(I, psi, cell):
    n, nd, L, Ndiv, t = I.n, I.nd, I.n * I.nd, I.Ndiv, I.t
    kap = I.model.kappa
    g, cg = I.dense.gint, I.coarse.gint
    lin = {tuple(x): i for i, x in enumerate(g)}
    R2 = oi.near_radius2(I.width, nd)
    rad = int(np.floor(np.sqrt(R2)))
    offs = [np.array((a, b, c)) for a in range(-rad, rad + 1) for b in range(-rad, rad + 1)
            for c in range(-rad, rad + 1) if a * a + b * b + c * c <= R2]
    P = psi.reshape(I.Nk, I.nv, I.nc)
    targets = [kd for kd in range(I.Nk) if kd // Ndiv == cell]
    near = {}                                    # (target, source point) -> dense offset
    rows = {}                                    # slot -> source pairs (k', corner)
    for kd in targets:
        for d in offs:
            kp = lin[tuple(np.mod(g[kd] + d, L))]
            near[(kd, kp)] = tuple(d)
            for lp in range(8):
                if I.f[kp, lp] != 0.0:
                    rows.setdefault(int(I.corner[kp, lp]), set()).add((kp, lp))
    alpha = -(I.model.e_k / I.Nkc) * 4 * np.pi / I.model.eps_inf
    out = np.zeros((len(targets), t), dtype=np.complex128)
    for s, rset in rows.items():
        rlist = sorted(rset)
        X = np.stack([(I.f[kp, lp] * (I.Dv[kp, lp].conj() @ P[kp] @ I.Dc[kp, lp].T)).reshape(-1)
                      for kp, lp in rlist])                                  # gathered rows [R, t]
        Sy = np.zeros((len(targets), len(rlist)))
        Sz = np.zeros((len(targets), len(rlist)))
        for j, kd in enumerate(targets):
            for r, (kp, lp) in enumerate(rlist):
                if (kd, kp) in near:
                    Sy[j, r] = om.h_head(near[(kd, kp)], L, kap)
                    Sz[j, r] = 1.0
        y1, z = Sy @ X, Sz @ X                                               # stage 1
        for j, kd in enumerate(targets):
            for l in range(8):
                if I.f[kd, l] == 0.0:
                    continue
                a = int(I.corner[kd, l])
                hc = om.h_head(tuple(cg[a] - cg[s]), n, kap)
                Ov = om.overlap_v(I.coarse.Uv[a], I.coarse.Uv[s])
                Oc = om.overlap_c(I.coarse.Uc[a], I.coarse.Uc[s])
                u = alpha * (Ov @ (y1[j] - hc * z[j]).reshape(I.nv, I.nc) @ Oc.T)   # stage 2
                out[j] += I.f[kd, l] * (I.Dv[kd, l].T @ u @ I.Dc[kd, l].conj()).reshape(-1)
    return targets, out / Ndiv


@pytest.mark.parametrize("nv,nc,n,nd,width,scheme", [(2, 2, 4, 2, 1.0, "8nb"), (1, 3, 5, 3, 1.0, "8nb"),
                                                     (2, 2, 5, 2, 1.5, "8nb"), (2, 2, 4, 2, 1.0, "1nb")])
def test_two_gemm_factorisation_is_exact(nv, nc, n, nd, width, scheme):
    I = oi.Interp(synth.draw_model(17, nv, nc), n, nd, scheme=scheme, width=width, build_dense_kc=False)
    psi = synth.random_vectors(5, I.N)
    for cell in (0, I.Nkc // 2, I.Nkc - 1):
        targets, got = factorised_near_field(I, psi, cell)
        ref = I.near_field_rows(psi, np.array(targets))
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
