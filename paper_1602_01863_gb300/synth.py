"""Seeded synthetic inputs for the model crystal.

This module only DRAWS random numbers and fixes the workload sizes. It holds
none of the method's arithmetic: no gauge matrices, no kernel elements, no
interpolation. Both the CUDA library (through the C-ABI `bse_model` struct)
and the CPU oracle consume the same arrays, each computing everything else
on its own.

The model stands in for the ab initio inputs of Sec. 2 (Eqs. bse1-bse3b):
band-energy offsets, Hermitian generators of the smooth band gauge, the
exchange form-factor coefficients mu and the dipole coefficients pi.
Array layouts (all complex128, C order):

  offsets [nv, nc]            real, eV, U(0, 0.5) per (v, c) pair
  gen_v   [3, 2, nv, nv]      Hermitian; [axis a, kind (sin, 1-cos)]
  gen_c   [3, 2, nc, nc]      Hermitian
  mu      [7, 26, nv, nc]     harmonic h in (1, cos k1, sin k1, cos k2, ...),
                              G index in gvectors_nonzero() order
  dip     [7, 3, nv, nc]      harmonic h, Cartesian direction alpha; pi[m, m']
                              pairs reference valence m with conduction m'
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Model constants (eV).  Fixed readings of quantities the paper leaves to the
# ab initio inputs; each one is listed with its reason in the design notes.
E_GAP = 1.1          # Delta E offset of the lowest transition at k = 0
BAND_WIDTH = 0.3     # Delta E_vc(k) = E_GAP + BAND_WIDTH * sum_i (1 - cos 2 pi k_i) + o_vc
E_K = 0.1            # overall kernel strength
A_X = 0.05           # exchange form-factor amplitude
THETA = 0.5          # gauge generator scale
HARM_MU = 0.5        # relative size of the k-harmonics of mu
HARM_DIP = 0.3       # relative size of the k-harmonics of the dipoles
S_EPS = 1.0          # epsilon prefactor s: eps = 1 - (s / N_k) |P|^2 g(z)
ETA = 0.1            # Lorentzian broadening (eV), Sec. 5.1


def gvectors_nonzero() -> np.ndarray:
    """The 26 non-zero G in {-1,0,1}^3, lexicographic (g1 slowest)."""
    g = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    return np.array([x for x in g if x != (0, 0, 0)], dtype=np.int64)


def gvectors_all() -> np.ndarray:
    """All 27 G in {-1,0,1}^3, lexicographic (g1 slowest)."""
    return np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1)
                     for c in (-1, 0, 1)], dtype=np.int64)


@dataclasses.dataclass
class ModelParams:
    nv: int
    nc: int
    eps_inf: float
    kappa: float
    offsets: np.ndarray
    gen_v: np.ndarray
    gen_c: np.ndarray
    mu: np.ndarray
    dip: np.ndarray
    e_k: float = E_K
    e_gap: float = E_GAP
    band_width: float = BAND_WIDTH
    direct_shells: int = 27      # 27: G in {-1,0,1}^3; 1: G = 0 only
    h_const: bool = False        # direct-term shape h(q) == h0 (constant model)
    h0: float = 40.0
    exchange_on: bool = True
    seed: int = 0


def _cnormal(rng: np.random.Generator, shape) -> np.ndarray:
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def _hermitian(rng: np.random.Generator, n: int) -> np.ndarray:
    x = _cnormal(rng, (n, n))
    return (x + x.conj().T) / 2.0


def draw_model(seed: int, nv: int, nc: int, *, eps_inf: float = 12.0,
               kappa: float = 0.3, const_mu: bool = False,
               direct_shells: int = 27, h_const: bool = False,
               exchange_on: bool = True) -> ModelParams:
    """Draw one model crystal's parameters from numpy's PCG64 stream.

    The draw order is fixed: offsets, gen_v, gen_c, mu, dip.  `const_mu`
    zeroes the k-harmonics of mu and the dipoles after the draw, so the
    stream position of every other number is unchanged.
    """
    rng = np.random.default_rng(seed)
    offsets = rng.uniform(0.0, 0.5, size=(nv, nc))
    gen_v = np.empty((3, 2, nv, nv), dtype=np.complex128)
    gen_c = np.empty((3, 2, nc, nc), dtype=np.complex128)
    for a in range(3):
        for kind in range(2):
            gen_v[a, kind] = THETA * _hermitian(rng, nv) / np.sqrt(nv)
    for a in range(3):
        for kind in range(2):
            gen_c[a, kind] = THETA * _hermitian(rng, nc) / np.sqrt(nc)
    g = gvectors_nonzero()
    gdamp = np.exp(-0.5 * (g * g).sum(axis=1))                    # [26]
    mu = _cnormal(rng, (7, 26, nv, nc)) * A_X * gdamp[None, :, None, None]
    mu[1:] *= HARM_MU
    dip = _cnormal(rng, (7, 3, nv, nc))
    dip[1:] *= HARM_DIP
    if const_mu:
        mu[1:] = 0.0
        dip[1:] = 0.0
    return ModelParams(nv=nv, nc=nc, eps_inf=float(eps_inf), kappa=float(kappa),
                       offsets=offsets, gen_v=gen_v, gen_c=gen_c, mu=mu, dip=dip,
                       direct_shells=direct_shells, h_const=h_const,
                       exchange_on=exchange_on, seed=seed)


@dataclasses.dataclass
class System:
    """One Haydock problem: model + coarse grid n^3 refined by n_div^3."""
    model: ModelParams
    n_coarse: int
    n_div: int
    npol: int
    pol_dirs: np.ndarray          # [npol, 3] unit vectors

    @property
    def t(self) -> int:
        return self.model.nv * self.model.nc

    @property
    def nk_coarse(self) -> int:
        return self.n_coarse ** 3

    @property
    def nk_dense(self) -> int:
        return (self.n_coarse * self.n_div) ** 3

    @property
    def n_coarse_dim(self) -> int:
        return self.t * self.nk_coarse

    @property
    def n_dense_dim(self) -> int:
        return self.t * self.nk_dense


POL3 = np.eye(3)


def small_system(seed: int = 1) -> System:
    """Coarse 4^3, 3v x 3c, n_div 2: 512 dense k, N = 4608; x polarisation."""
    return System(draw_model(seed, 3, 3, eps_inf=12.0, kappa=0.3), 4, 2, 1, POL3[:1].copy())


def single_system(seed: int = 2) -> System:
    """Coarse 8^3, 4v x 4c, n_div 4: 32768 dense k, N = 524288; 3 polarisations."""
    return System(draw_model(seed, 4, 4, eps_inf=12.0, kappa=0.3), 8, 4, 3, POL3.copy())


def largest_system(seed: int = 3) -> System:
    """Coarse 12^3, 4v x 6c, n_div 4: 110592 dense k, N = 2654208; 3 polarisations."""
    return System(draw_model(seed, 4, 6, eps_inf=12.0, kappa=0.3), 12, 4, 3, POL3.copy())


def batched_systems(first_seed: int = 100, count: int = 24) -> list[System]:
    """Uneven batch: per seed, coarse n in {4..8}, n_div in {2,3,4}, nv, nc in
    {2..6}, eps_inf ~ U(5, 15), kappa ~ U(0.2, 0.5); 3 polarisations each."""
    out = []
    for s in range(first_seed, first_seed + count):
        rng = np.random.default_rng(10_000 + s)
        n = int(rng.integers(4, 9))
        nd = int(rng.integers(2, 5))
        nv = int(rng.integers(2, 7))
        nc = int(rng.integers(2, 7))
        eps = float(rng.uniform(5.0, 15.0))
        kap = float(rng.uniform(0.2, 0.5))
        out.append(System(draw_model(s, nv, nc, eps_inf=eps, kappa=kap), n, nd, 3, POL3.copy()))
    return out


def frequency_grid(nw: int, wmax: float = 10.0) -> np.ndarray:
    """omega_j = j * wmax / (nw - 1), j = 0..nw-1 (eV)."""
    return np.linspace(0.0, wmax, nw)


def random_vectors(seed: int, shape, dtype=np.complex128) -> np.ndarray:
    """Seeded complex test vectors (unit-variance complex normal)."""
    rng = np.random.default_rng(seed)
    return _cnormal(rng, shape).astype(dtype)
