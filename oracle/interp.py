"""Double-grid interpolation of the BSE kernel (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

  d tables   Eq. completeness: d_{nk}^{n'k~} = <u_{n'k~}|u_{nk}> = [U(k~)^H U(k)]_{n'n},
             kept block-diagonal in valence / conduction (Sec. 5.1: v-c mixing
             neglected).  Dv[kd, l] is nv x nv with Dv[n', n] = d_n^{n'}.
  F          Eq. interpwfn in matrix form: F_{(vc,k),(n1n2,k~)} =
             sum_{l: corner = k~} f(k, l) d_v^{n1} conj(d_c^{n2}).
  M1         Eq. interp1 = F K_c F^H, with the 1/N_div weight change from a
             coarse to a dense BZ sum:  K^{M1} = (1/N_div) F K_c F^H.
  matmul1-3  The same product without the dense matrix (Eqs. matmul1-3).
  M2         Sec. 4: every pair keeps the interpolated coefficients of Eq. diverg
             and divides the head by the dense q (dense matrix, small systems only).
  M3         Sec. 4: pairs with ||k - k'|| <= w d keep the interpolated
             divergent coefficient a (Eq. diverg) and divide by the dense q:
             K^{M3} = (1/N_div)[ (F A F^H) h_head(q_dense) + F (K_c - A h_head(q_coarse)) F^H ].
"""
from __future__ import annotations

import numpy as np

from paper_1602_01863_gb300.synth import ModelParams, System
from . import model as om


class Interp:
    """All interpolation data for one system (dense order coarse-major)."""

    def __init__(self, model: ModelParams, n: int, nd: int, scheme: str = "8nb", width: float = 1.0,
                 dense_gauge_twist: np.ndarray | None = None, build_dense_kc: bool = True):
        self.model = model
        self.n, self.nd = n, nd
        self.Ndiv = nd ** 3
        self.nv, self.nc = model.nv, model.nc
        self.t = model.nv * model.nc
        self.width = width
        self.coarse = om.GridModel(model, om.coarse_coords(n), n)
        self.dense = om.GridModel(model, om.dense_global(n, nd), n * nd, with_form_factors=False)
        if dense_gauge_twist is not None:
            # Gauge change of the dense states, U(k) -> U(k) Phi(k) (a phase per
            # band for non-degenerate bands).  P follows from the rotated
            # states; the spectrum must not move (Sec. 3, phase cancellation).
            Phv, Phc = dense_gauge_twist
            self.dense.Uv = self.dense.Uv @ Phv
            self.dense.Uc = self.dense.Uc @ Phc
            self.dense.P = om.dipoles(model, self.dense.Uv, self.dense.Uc, self.dense.kfrac)
        self.Nk = self.dense.gint.shape[0]
        self.Nkc = self.coarse.gint.shape[0]
        self.N = self.t * self.Nk
        self.Nc = self.t * self.Nkc
        self.corner, self.f = om.neighbour_tables(n, nd, scheme)
        Ucv = self.coarse.Uv[self.corner]                           # [Nk, 8, nv, nv]
        Ucc = self.coarse.Uc[self.corner]
        self.Dv = np.einsum("klmn,kmv->klnv", Ucv.conj(), self.dense.Uv)   # [Nk, 8, n', v]
        self.Dc = np.einsum("klmn,kmc->klnc", Ucc.conj(), self.dense.Uc)
        self.dE = self.dense.dE.reshape(-1)
        if build_dense_kc:
            self.Kc = om.kernel_matrix(self.coarse)
            self.A, self.Hhead_c = om.head_matrix(self.coarse)
        self._F = None

    # ------------------------------------------------------------ dense form
    def F(self) -> np.ndarray:
        """Dense interpolation matrix [N, N_c] (Eq. interpwfn)."""
        if self._F is None:
            F = np.zeros((self.N, self.Nc), dtype=np.complex128)
            for kd in range(self.Nk):
                for l in range(8):
                    if self.f[kd, l] == 0.0:
                        continue
                    blk = self.f[kd, l] * np.einsum("nv,mc->vcnm", self.Dv[kd, l], self.Dc[kd, l].conj())
                    ic = self.corner[kd, l]
                    F[kd * self.t:(kd + 1) * self.t, ic * self.t:(ic + 1) * self.t] += blk.reshape(self.t, self.t)
            self._F = F
        return self._F

    def K_m1_dense(self) -> np.ndarray:
        """K^{M1} = (1/N_div) F K_c F^H (Eq. interp1)."""
        F = self.F()
        return (F @ self.Kc @ F.conj().T) / self.Ndiv

    def dense_q_tables(self):
        """Dense pair data: near mask and h_head(q_dense) on [N_k, N_k]."""
        L = self.n * self.nd
        g = self.dense.gint
        dg = g[:, None, :] - g[None, :, :]
        dmin = np.mod(dg + L // 2, L) - L // 2          # a representative; near pairs are tie-free
        r2 = (dmin * dmin).sum(-1)
        near = r2 <= near_radius2(self.width, self.nd)
        ht = om.h_table(L, lambda d: om.h_head(d, L, self.model.kappa))
        dgm = np.mod(dg, L)
        return near, ht[dgm[..., 0], dgm[..., 1], dgm[..., 2]]

    def K_m3_dense(self) -> np.ndarray:
        """K^{M3}: M1 everywhere, the divergence-treated form on near pairs (Sec. 4)."""
        F = self.F()
        t = self.t
        near, hd = self.dense_q_tables()
        FA = F @ self.A @ F.conj().T
        Hc_blk = np.kron(self.Hhead_c, np.ones((t, t)))
        FAh = F @ (self.A * Hc_blk) @ F.conj().T
        near_blk = np.kron(near, np.ones((t, t))).astype(bool)
        hd_blk = np.kron(hd, np.ones((t, t)))
        delta = np.where(near_blk, (FA * hd_blk - FAh) / self.Ndiv, 0.0)
        return self.K_m1_dense() + delta

    def K_m2_dense(self) -> np.ndarray:
        """K^{M2} (Sec. 4, "Method 2"): the coefficients of Eq. diverg are
        interpolated for every dense pair and the divergent head is divided by
        the dense q everywhere (no width):
        (1/N_div)[(F A F^H) h_head(q_dense) + F (K_c - A h_head(q_coarse)) F^H].
        The model has no 1/q wing (b = 0), so a and c are the only terms."""
        F = self.F()
        t = self.t
        _, hd = self.dense_q_tables()
        FA = F @ self.A @ F.conj().T
        Hc_blk = np.kron(self.Hhead_c, np.ones((t, t)))
        FC = F @ (self.Kc - self.A * Hc_blk) @ F.conj().T
        return (FA * np.kron(hd, np.ones((t, t))) + FC) / self.Ndiv

    def H_dense(self, method: str = "m1") -> np.ndarray:
        K = {"m1": self.K_m1_dense, "m2": self.K_m2_dense, "m3": self.K_m3_dense}[method]()
        return np.diag(self.dE).astype(np.complex128) + K

    # ------------------------------------------------------- matrix-free form
    def restrict(self, psi: np.ndarray) -> np.ndarray:
        """Eq. matmul1 summed over the eight offsets: Q = F^H psi  -> [N_c]."""
        P = psi.reshape(self.Nk, self.nv, self.nc)
        x = np.einsum("klnv,kvc,klmc->klnm", self.Dv.conj(), P, self.Dc) * self.f[:, :, None, None]
        Q = np.zeros((self.Nkc, self.nv, self.nc), dtype=np.complex128)
        np.add.at(Q, self.corner.reshape(-1), x.reshape(-1, self.nv, self.nc))
        return Q.reshape(-1)

    def prolong(self, R: np.ndarray) -> np.ndarray:
        """Eq. matmul3: s = F R  -> [N]."""
        Rb = R.reshape(self.Nkc, self.nv, self.nc)[self.corner]          # [Nk, 8, n1, n2]
        s = np.einsum("klnv,klnm,klmc->kvc", self.Dv * self.f[:, :, None, None], Rb, self.Dc.conj())
        return s.reshape(-1)

    def apply_m1(self, psi: np.ndarray, Kc: np.ndarray | None = None) -> np.ndarray:
        """H^{M1} psi = Delta E psi + (1/N_div) F K_c (F^H psi) (Eqs. matmul1-3)."""
        Kc = self.Kc if Kc is None else Kc
        return self.dE * psi + self.prolong(Kc @ self.restrict(psi)) / self.Ndiv

    def apply_m1_rows(self, psi: np.ndarray, rows: np.ndarray) -> np.ndarray:
        """(H^{M1} psi) at the dense points `rows` (Eqs. matmul1-3) with only the
        K_c rows of their corners computed (for meshes whose K_c is too large
        to store): [len(rows), t]."""
        Q = self.restrict(psi)
        corners = np.unique(self.corner[rows][self.f[rows] != 0])
        Kr = om.kernel_rows(self.coarse, corners)
        Rc = (Kr @ Q).reshape(len(corners), self.nv, self.nc)
        pos = {int(c): i for i, c in enumerate(corners)}
        t = self.t
        out = np.zeros((len(rows), t), dtype=np.complex128)
        for r, kd in enumerate(rows):
            s = np.zeros((self.nv, self.nc), dtype=np.complex128)
            for l in range(8):
                if self.f[kd, l] == 0.0:
                    continue
                R = Rc[pos[int(self.corner[kd, l])]]
                s += self.f[kd, l] * (self.Dv[kd, l].T @ R @ self.Dc[kd, l].conj())
            out[r] = self.dE[kd * t:(kd + 1) * t] * psi[kd * t:(kd + 1) * t] + s.reshape(-1) / self.Ndiv
        return out

    def near_field_rows(self, psi: np.ndarray, rows: np.ndarray) -> np.ndarray:
        """(K^{M3} - K^{M1}) psi at the dense points `rows`, pair by pair.

        For every near pair (k, k') and every corner pair (k~ in N(k), k~' in N(k')):
        (1/N_div) f f' [h_head(q_dense) - h_head(q_coarse)] F-block A-block F^H-block.
        Slow; meant for a handful of sampled rows.
        """
        n, nd, L = self.n, self.nd, self.n * self.nd
        kap = self.model.kappa
        g = self.dense.gint
        lin = {tuple(x): i for i, x in enumerate(g)}
        R2 = near_radius2(self.width, nd)
        rad = int(np.floor(np.sqrt(R2)))
        offs = [np.array((a, b, c)) for a in range(-rad, rad + 1) for b in range(-rad, rad + 1)
                for c in range(-rad, rad + 1) if a * a + b * b + c * c <= R2]
        P = psi.reshape(self.Nk, self.nv, self.nc)
        cg = self.coarse.gint
        alpha = -(self.model.e_k / self.Nkc) * 4 * np.pi / self.model.eps_inf
        out = np.zeros((len(rows), self.nv, self.nc), dtype=np.complex128)
        for r, kd in enumerate(rows):
            for d in offs:
                kp = lin[tuple(np.mod(g[kd] + d, L))]
                hd = om.h_head(tuple(d), L, kap)
                for l in range(8):
                    if self.f[kd, l] == 0.0:
                        continue
                    a = self.corner[kd, l]
                    for lp in range(8):
                        if self.f[kp, lp] == 0.0:
                            continue
                        b = self.corner[kp, lp]
                        hc = om.h_head(tuple(cg[a] - cg[b]), n, kap)
                        Ov = om.overlap_v(self.coarse.Uv[a], self.coarse.Uv[b])
                        Oc = om.overlap_c(self.coarse.Uc[a], self.coarse.Uc[b])
                        x = self.f[kp, lp] * (self.Dv[kp, lp].conj() @ P[kp] @ self.Dc[kp, lp].T)
                        y = alpha * (hd - hc) * (Ov @ x @ Oc.T)
                        out[r] += self.f[kd, l] * (self.Dv[kd, l].T @ y @ self.Dc[kd, l].conj())
        return out.reshape(len(rows), -1) / self.Ndiv

    def dipole(self, e) -> np.ndarray:
        return om.polarised_dipole(self.dense, e)


def near_radius2(width: float, nd: int) -> int:
    """Near pairs: ||q_dense|| <= w d, d = one coarse spacing = n_div dense steps,
    tested on the integer offset: |delta|^2 <= floor(w^2 n_div^2 + 1e-9)."""
    return int(np.floor(width * width * nd * nd + 1e-9))


def interp_for(sys: System, **kw) -> Interp:
    return Interp(sys.model, sys.n_coarse, sys.n_div, **kw)
