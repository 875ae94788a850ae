"""Grids, trilinear weights and the synthetic model crystal (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions
  * Coarse mesh (Sec. 3): k~_(i1,i2,i3) = sum_j i_j k^_j, i_j in [0, n).
    Coarse index ic = (i1 * n + i2) * n + i3.
  * Dense mesh: k_(i),(j) = sum_j (i_j + j_j / n_div) k^_j, j_j in [0, n_div).
    Dense index is coarse-major: kd = ic * N_div + js, js = (j1*nd + j2)*nd + j3.
    Global integer coordinate g = i * n_div + j on an L = n * n_div grid.
  * Reciprocal basis vectors are orthonormal (cubic, |k^_j| = 1 per coarse
    spacing * n), so the Cartesian q of an index difference is that
    difference divided by the grid size, reduced to the minimum image.
  * Transition index within one k: tr = v * nc + c.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

from paper_1602_01863_gb300.synth import ModelParams, gvectors_all, gvectors_nonzero

CORNERS = np.array([(l1, l2, l3) for l1 in (0, 1) for l2 in (0, 1) for l3 in (0, 1)],
                   dtype=np.int64)           # neighbour lmn = l1*4 + l2*2 + l3 (Eq. neighborhood)


# --------------------------------------------------------------------- grids
def coarse_coords(n: int) -> np.ndarray:
    """[n^3, 3] integer coordinates i of the coarse points, ic order."""
    i = np.arange(n)
    return np.stack(np.meshgrid(i, i, i, indexing="ij"), axis=-1).reshape(-1, 3)


def dense_coords(n: int, nd: int) -> tuple[np.ndarray, np.ndarray]:
    """(i, j) of every dense point in coarse-major order: [N_k, 3] each."""
    ci = coarse_coords(n)
    sj = coarse_coords(nd)
    i = np.repeat(ci, nd ** 3, axis=0)
    j = np.tile(sj, (n ** 3, 1))
    return i, j


def dense_global(n: int, nd: int) -> np.ndarray:
    """Global integer coordinates g = i * n_div + j, coarse-major order."""
    i, j = dense_coords(n, nd)
    return i * nd + j


def coarse_index(i: np.ndarray, n: int) -> np.ndarray:
    i = np.mod(i, n)
    return (i[..., 0] * n + i[..., 1]) * n + i[..., 2]


def trilinear_weight(j: np.ndarray, l: np.ndarray, nd: int) -> np.ndarray:
    """f^{lmn} = f^l_{j1} f^m_{j2} f^n_{j3}, f^0_j = 1 - j/n_div, f^1_j = j/n_div."""
    fj = np.where(l == 0, 1.0 - j / nd, j / nd)
    return np.prod(fj, axis=-1)


def neighbour_tables(n: int, nd: int, scheme: str = "8nb"):
    """Corner coarse index and weight for every (dense kd, corner lmn).

    Returns (corner_ic [N_k, 8], f [N_k, 8]).  Eq. neighborhood with a periodic
    wrap of the corner index; weights from the trilinear prefactors, or for
    the one-neighbour (Rohlfing-Louie) scheme f = 1 on the nearest corner,
    j/n_div = 1/2 going to l = 0.
    """
    i, j = dense_coords(n, nd)
    corner_ic = coarse_index(i[:, None, :] + CORNERS[None, :, :], n)
    if scheme == "8nb":
        f = trilinear_weight(j[:, None, :], CORNERS[None, :, :], nd)
    elif scheme == "1nb":
        near_l = (2 * j > nd).astype(np.int64)                 # nearest corner per axis
        f = np.all(CORNERS[None, :, :] == near_l[:, None, :], axis=-1).astype(np.float64)
    else:
        raise ValueError(scheme)
    return corner_ic, f


def min_image_candidates(delta: int, L: int) -> list[int]:
    """Minimum-image representatives of an index difference on a periodic
    L-point axis.  A tie (component exactly L/2) returns both images."""
    r = delta % L
    if 2 * r < L:
        return [r]
    if 2 * r > L:
        return [r - L]
    return [r, r - L]


def _image_list(delta3, L):
    cands = [min_image_candidates(int(d), L) for d in delta3]
    out = []
    for a in cands[0]:
        for b in cands[1]:
            for c in cands[2]:
                out.append(np.array([a, b, c], dtype=np.float64) / L)
    return out


def h_full(delta3, L: int, model: ModelParams) -> float:
    """Direct-term shape h(q) = sum_G lambda_G^2 4 pi / (|q + G|^2 + kappa^2),
    lambda_G = exp(-|G|^2 / 2), q the minimum image (ties averaged)."""
    if model.h_const:
        return float(model.h0)
    G = gvectors_all() if model.direct_shells == 27 else np.zeros((1, 3), dtype=np.int64)
    lam2 = np.exp(-(G * G).sum(axis=1))
    vals = []
    for q in _image_list(delta3, L):
        qg = q[None, :] + G
        vals.append(np.sum(lam2 * 4.0 * np.pi / ((qg * qg).sum(axis=1) + model.kappa ** 2)))
    return float(np.mean(vals))


def h_head(delta3, L: int, kappa: float) -> float:
    """Divergent head shape 1 / (|q|^2 + kappa^2) (Eq. diverg, a/q^2 term
    regularised by the model's kappa), minimum image, ties averaged."""
    vals = [1.0 / (float(q @ q) + kappa ** 2) for q in _image_list(delta3, L)]
    return float(np.mean(vals))


def h_table(L: int, fn) -> np.ndarray:
    """[L, L, L] table of fn(delta) over all index differences mod L."""
    t = np.empty((L, L, L))
    for a in range(L):
        for b in range(L):
            for c in range(L):
                t[a, b, c] = fn((a, b, c))
    return t


# --------------------------------------------------------------------- model
def harmonics(kfrac: np.ndarray) -> np.ndarray:
    """[..., 7]: (1, cos 2pi k1, sin 2pi k1, cos 2pi k2, sin 2pi k2, cos 2pi k3, sin 2pi k3)."""
    c = np.cos(2 * np.pi * kfrac)
    s = np.sin(2 * np.pi * kfrac)
    one = np.ones(kfrac.shape[:-1])
    return np.stack([one, c[..., 0], s[..., 0], c[..., 1], s[..., 1], c[..., 2], s[..., 2]], axis=-1)


def gauge(gen: np.ndarray, kfrac: np.ndarray) -> np.ndarray:
    """Smooth periodic band gauge U(k) = expm(i sum_a [sin(2pi k_a) H_a1 + (1 - cos 2pi k_a) H_a2]).

    Columns are the periodic Bloch parts u_nk in a fixed reference basis, so
    the overlap of Eq. completeness is d_{nk}^{n'k~} = [U(k~)^H U(k)]_{n'n}.
    """
    kfrac = np.atleast_2d(kfrac)
    out = np.empty((kfrac.shape[0], gen.shape[-1], gen.shape[-1]), dtype=np.complex128)
    for p, k in enumerate(kfrac):
        A = np.zeros(gen.shape[-2:], dtype=np.complex128)
        for a in range(3):
            A += np.sin(2 * np.pi * k[a]) * gen[a, 0] + (1 - np.cos(2 * np.pi * k[a])) * gen[a, 1]
        out[p] = expm(1j * A)
    return out


def energies(model: ModelParams, kfrac: np.ndarray) -> np.ndarray:
    """Delta E_vc(k) = E_gap + B sum_i (1 - cos 2 pi k_i) + o_vc  -> [..., nv, nc]."""
    band = model.e_gap + model.band_width * np.sum(1 - np.cos(2 * np.pi * kfrac), axis=-1)
    return band[..., None, None] + model.offsets


def form_factors(model: ModelParams, Uv, Uc, kfrac) -> np.ndarray:
    """M_vc(k, G) = [U_v(k)^H mu(k, G) U_c(k)]_vc  -> [Npts, 26, nv, nc]."""
    mu = np.einsum("ph,hgmn->pgmn", harmonics(kfrac), model.mu)
    return np.einsum("pmv,pgmn,pnc->pgvc", Uv.conj(), mu, Uc)


def dipoles(model: ModelParams, Uv, Uc, kfrac) -> np.ndarray:
    """P^alpha_vc(k) = <u_ck| pi^alpha(k) |u_vk> = [U_v(k)^T pi^alpha(k) conj(U_c(k))]_vc
    -> [Npts, 3, nv, nc].  The conjugate sits on the conduction state, as in
    P_vck = <c k+q|e^{iqr}|v k> (Sec. 2), so P transforms like the transition
    basis u*_vk u_ck under a change of band gauge."""
    pi = np.einsum("ph,hamn->pamn", harmonics(kfrac), model.dip)
    return np.einsum("pmv,pamn,pnc->pavc", Uv, pi, Uc.conj())


def coulomb_bar() -> np.ndarray:
    """v(G) = 4 pi / |G|^2 on the 26 non-zero G (G = 0 removed, Sec. 2)."""
    g = gvectors_nonzero()
    return 4 * np.pi / (g * g).sum(axis=1)


class GridModel:
    """The model evaluated on one periodic L^3 grid of points (integer coords)."""

    def __init__(self, model: ModelParams, gint: np.ndarray, L: int, with_form_factors: bool = True):
        self.model = model
        self.gint = gint
        self.L = L
        self.kfrac = gint / L
        self.Uv = gauge(model.gen_v, self.kfrac)
        self.Uc = gauge(model.gen_c, self.kfrac)
        self.dE = energies(model, self.kfrac)
        self.M = form_factors(model, self.Uv, self.Uc, self.kfrac) if with_form_factors else None
        self.P = dipoles(model, self.Uv, self.Uc, self.kfrac)


def overlap_v(Uv_a, Uv_b):
    """O^v(k, k')_{vv'} = sum_m U_v(k)_{mv} conj(U_v(k')_{mv'})."""
    return np.einsum("...mv,...mw->...vw", Uv_a, Uv_b.conj())


def overlap_c(Uc_a, Uc_b):
    """O^c(k, k')_{cc'} = sum_m conj(U_c(k)_{mc}) U_c(k')_{mc'}."""
    return np.einsum("...mc,...md->...cd", Uc_a.conj(), Uc_b)


def kernel_matrix(gm: GridModel) -> np.ndarray:
    """Explicit model kernel on one grid (N_g = number of grid points):

      K_{vck,v'c'k'} = (E_K / N_g) [ 2 sum_{G != 0} v(G) conj(M_vc(k,G)) M_v'c'(k',G)
                                     - (1/eps_inf) O^v_{vv'}(k,k') O^c_{cc'}(k,k') h(k - k') ]

    i.e. Eq. bse2 with the exchange of Eq. bse3a (v-bar, G = 0 removed) and
    the direct term of Eq. bse3b with a Yukawa-screened W (Eq. Wcoul
    replaced by the model).  Returned as a dense [N, N] matrix, N = t * N_g.
    """
    m = gm.model
    npts = gm.gint.shape[0]
    nv, nc = m.nv, m.nc
    t = nv * nc
    pref = m.e_k / npts
    Mflat = gm.M.transpose(0, 2, 3, 1).reshape(npts * t, 26)
    K = np.zeros((npts * t, npts * t), dtype=np.complex128)
    if m.exchange_on:
        K += 2 * pref * (Mflat.conj() * coulomb_bar()[None, :]) @ Mflat.T
    Ov = overlap_v(gm.Uv[:, None], gm.Uv[None, :])             # [k, k', v, v']
    Oc = overlap_c(gm.Uc[:, None], gm.Uc[None, :])             # [k, k', c, c']
    ht = h_table(gm.L, lambda d: h_full(d, gm.L, m))
    dg = np.mod(gm.gint[:, None, :] - gm.gint[None, :, :], gm.L)
    H = ht[dg[..., 0], dg[..., 1], dg[..., 2]]                 # [k, k']
    D = np.einsum("abvw,abcd,ab->avcbwd", Ov, Oc, H).reshape(npts * t, npts * t)
    K -= (pref / m.eps_inf) * D
    return K


def kernel_rows(gm: GridModel, pts: np.ndarray) -> np.ndarray:
    """Rows of the same kernel (kernel_matrix) for the grid points `pts`
    only: [len(pts) * t, N], computed pair by pair from the model, for grids
    whose full matrix is too large to store."""
    m = gm.model
    npts = gm.gint.shape[0]
    t = m.nv * m.nc
    pref = m.e_k / npts
    out = np.zeros((len(pts), t, npts, t), dtype=np.complex128)
    if m.exchange_on:
        Mflat = gm.M.transpose(0, 2, 3, 1)                                   # [p, v, c, G]
        rowsM = Mflat[pts].reshape(len(pts), t, 26)
        allM = Mflat.reshape(npts, t, 26)
        out += 2 * pref * np.einsum("avg,g,bwg->avbw", rowsM.conj(), coulomb_bar(), allM)
    Ov = overlap_v(gm.Uv[pts][:, None], gm.Uv[None, :])                    # [a, b, v, v']
    Oc = overlap_c(gm.Uc[pts][:, None], gm.Uc[None, :])
    ht = h_table(gm.L, lambda d: h_full(d, gm.L, m))
    dg = np.mod(gm.gint[pts][:, None, :] - gm.gint[None, :, :], gm.L)
    H = ht[dg[..., 0], dg[..., 1], dg[..., 2]]
    out -= (pref / m.eps_inf) * np.einsum("abvw,abcd,ab->avcbwd", Ov, Oc, H).reshape(len(pts), t, npts, t)
    return out.reshape(len(pts) * t, npts * t)


def head_matrix(gm: GridModel) -> tuple[np.ndarray, np.ndarray]:
    """Coarse head A (Eq. diverg, a-coefficients) and its divergent shape.

    A_{n1n2k~, n3n4k~'} = alpha O^v_{n1n3}(k~,k~') O^c_{n2n4}(k~,k~'),
    alpha = -(E_K / N_g)(4 pi lambda_0^2 / eps_inf), lambda_0 = 1: the G = 0
    term of the direct part, whose q-dependence is h_head(q) = 1/(|q|^2+kappa^2).
    Returns (A [N, N], Hhead [N_g, N_g]).
    """
    m = gm.model
    npts = gm.gint.shape[0]
    t = m.nv * m.nc
    alpha = -(m.e_k / npts) * 4 * np.pi / m.eps_inf
    Ov = overlap_v(gm.Uv[:, None], gm.Uv[None, :])
    Oc = overlap_c(gm.Uc[:, None], gm.Uc[None, :])
    A = alpha * np.einsum("abvw,abcd->avcbwd", Ov, Oc).reshape(npts * t, npts * t)
    ht = h_table(gm.L, lambda d: h_head(d, gm.L, m.kappa))
    dg = np.mod(gm.gint[:, None, :] - gm.gint[None, :, :], gm.L)
    return A, ht[dg[..., 0], dg[..., 1], dg[..., 2]]


def explicit_dense_hamiltonian(model: ModelParams, n: int, nd: int):
    """H = diag(Delta E) + K on the dense mesh (Eq. bse1), dense [N, N], with
    the dense grid model (dense order coarse-major)."""
    gm = GridModel(model, dense_global(n, nd), n * nd)
    K = kernel_matrix(gm)
    return np.diag(gm.dE.reshape(-1)).astype(np.complex128) + K, gm


def polarised_dipole(gm: GridModel, e: np.ndarray) -> np.ndarray:
    """P(q -> 0 along e)_vck = sum_alpha e_alpha P^alpha_vc(k), flattened [N]."""
    return np.einsum("a,pavc->pvc", np.asarray(e, dtype=np.float64), gm.P).reshape(-1)


class ExplicitOperator:
    """Matrix-free explicit dense H (Eq. bse1) for grids too large to store.

    Exchange: (2 E_K / N_k) conj(M) diag(v) (M^T psi), rank 26.
    Direct:   -(E_K / (N_k eps_inf)) U_v(k)^T [h (*) phi](k) conj(U_c(k)),
              phi(k') = conj(U_v(k')) psi(k') U_c(k')^T, where (*) is the periodic
              3-D convolution over the dense grid (exact: h depends only on the
              index difference), done with FFTs.
    This uses the model's own structure; it is a checking device, not the method.
    """

    def __init__(self, model: ModelParams, n: int, nd: int):
        self.gm = GridModel(model, dense_global(n, nd), n * nd)
        L = n * nd
        self.L = L
        m = model
        self.t = m.nv * m.nc
        npts = L ** 3
        self.pref = m.e_k / npts
        self.Mflat = self.gm.M.transpose(0, 2, 3, 1).reshape(npts * self.t, 26)
        self.vG = coulomb_bar()
        ht = h_table(L, lambda d: h_full(d, L, m))
        self.hk = np.fft.fftn(ht)
        g = self.gm.gint
        self.lin = (g[:, 0] * L + g[:, 1]) * L + g[:, 2]          # dense kd -> grid position

    def apply(self, psi: np.ndarray) -> np.ndarray:
        m = self.gm.model
        L = self.L
        out = self.gm.dE.reshape(-1) * psi
        if m.exchange_on:
            out = out + 2 * self.pref * (self.Mflat.conj() @ (self.vG * (self.Mflat.T @ psi)))
        P = psi.reshape(-1, m.nv, m.nc)
        phi = np.einsum("pmv,pvc,pnc->pmn", self.gm.Uv.conj(), P, self.gm.Uc)
        grid = np.zeros((L ** 3, m.nv, m.nc), dtype=np.complex128)
        grid[self.lin] = phi
        grid = grid.reshape(L, L, L, m.nv, m.nc)
        conv = np.fft.ifftn(np.fft.fftn(grid, axes=(0, 1, 2)) * self.hk[..., None, None], axes=(0, 1, 2))
        conv = conv.reshape(L ** 3, m.nv, m.nc)[self.lin]
        back = np.einsum("pmv,pmn,pnc->pvc", self.gm.Uv, conv, self.gm.Uc.conj())
        return out - (self.pref / m.eps_inf) * back.reshape(-1)
