"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than itself: a
closed form, an identity the paper derives, an exact special case, or a
brute-force computation on a tiny input.  A plausible mistake (a dropped
term, a wrong sign, a misplaced conjugate, a transposed operand, a missing
1/N_div) fails at least one of them.
"""
import functools
import json
import os

import numpy as np
import pytest

from paper_1602_01863_gb300 import synth
from oracle import haydock as oh
from oracle import interp as oi
from oracle import model as om

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@functools.lru_cache(maxsize=None)
def tiny_interp(seed=7, n=2, nd=2, nv=2, nc=2, const_mu=False, shells=27, h_const=False,
                scheme="8nb", width=0.5):
    m = synth.draw_model(seed, nv, nc, const_mu=const_mu, direct_shells=shells, h_const=h_const)
    return oi.Interp(m, n, nd, scheme=scheme, width=width)


# ------------------------------------------------------------------ grids
@pytest.mark.parametrize("nd", [1, 2, 3, 4, 5])
def test_trilinear_partition_of_unity_and_affine(nd):
    """Sec. 3, f^{lmn} = f^l f^m f^n: weights sum to 1 and reproduce affine
    functions of k inside a cell (what trilinear interpolation means)."""
    n = 3
    corner, f = om.neighbour_tables(n, nd)
    assert np.allclose(f.sum(1), 1.0, atol=1e-15)
    i, j = om.dense_coords(n, nd)
    rng = np.random.default_rng(0)
    A, c = rng.standard_normal(3), rng.standard_normal()
    x_dense = (i + j / nd) @ A + c                                     # affine, no wrap
    x_corner = (i[:, None, :] + om.CORNERS[None]) @ A + c
    assert np.allclose((f * x_corner).sum(1), x_dense, atol=1e-12)


def test_trilinear_weights_exact_values():
    """f^0_j = 1 - j/n_div, f^1_j = j/n_div: n_div = 4, j = (1, 2, 3) gives
    f^{lmn} = prod over axes, e.g. f^{000} = 3/4 * 1/2 * 1/4."""
    j = np.array([1, 2, 3])
    assert om.trilinear_weight(j, np.array([0, 0, 0]), 4) == pytest.approx(0.75 * 0.5 * 0.25)
    assert om.trilinear_weight(j, np.array([1, 1, 1]), 4) == pytest.approx(0.25 * 0.5 * 0.75)
    assert om.trilinear_weight(j, np.array([1, 0, 1]), 4) == pytest.approx(0.25 * 0.5 * 0.75)


def test_one_neighbour_scheme_picks_nearest_corner():
    """Eq. eqRL: f = 1 on one neighbour.  Reading: the nearest corner, with
    j/n_div = 1/2 going to l = 0."""
    corner, f = om.neighbour_tables(2, 4, "1nb")
    assert np.all(f.sum(1) == 1.0) and np.all((f == 0) | (f == 1))
    i, j = om.dense_coords(2, 4)
    l = om.CORNERS[np.argmax(f, axis=1)]
    assert np.all(l == (2 * j > 4))


def test_sum_reordering_identity():
    """Eq. ordersums: sum_k sum_{k~ in N(k)} f = sum_{k~'} sum_{k~ in N(k~')} sum_{k in S(k~')} f,
    checked by brute force with an arbitrary function in place of f."""
    n, nd = 3, 2
    corner, _ = om.neighbour_tables(n, nd)
    rng = np.random.default_rng(1)
    g = rng.standard_normal((n ** 3 * nd ** 3, n ** 3))       # arbitrary g(k, k~)
    lhs = sum(g[k, corner[k, l]] for k in range(g.shape[0]) for l in range(8))
    rhs = 0.0
    ci = om.coarse_coords(n)
    for kp in range(n ** 3):                                   # k~'
        for l in range(8):                                     # k~ in N(k~')
            kt = om.coarse_index(ci[kp] + om.CORNERS[l], n)
            for js in range(nd ** 3):                          # k in S(k~')
                rhs += g[kp * nd ** 3 + js, kt]
    assert np.isclose(lhs, rhs, rtol=1e-13)


def test_min_image_and_tie_symmetry():
    """Minimum image on a periodic axis; ties (difference exactly L/2) are
    averaged so h(q) = h(-q) holds on even grids (H stays Hermitian)."""
    assert om.min_image_candidates(3, 8) == [3]
    assert om.min_image_candidates(5, 8) == [-3]
    assert om.min_image_candidates(4, 8) == [4, -4]
    m = synth.draw_model(0, 1, 1)
    for d in [(4, 0, 0), (4, 4, 1), (1, 2, 3), (0, 0, 4)]:
        dm = tuple(-x for x in d)
        assert om.h_full(d, 8, m) == pytest.approx(om.h_full(dm, 8, m), rel=1e-15)
        assert om.h_head(d, 8, 0.3) == pytest.approx(om.h_head(dm, 8, 0.3), rel=1e-15)


def test_paper_sizes_golden():
    """Sec. 2: N = N_v N_c N_k and the dense-matrix storage it quotes;
    Sec. 3: N_k = N~_k N_div with N_div = n_div^3."""
    g = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))
    for ex in g["matrix_examples"]:
        N = ex["nv"] * ex["nc"] * ex["k_per_dim"] ** 3
        assert N == ex["N"]
    gb = ex_bytes = g["matrix_examples"][0]["N"] ** 2 * 16 / 2 ** 30
    assert 15 < gb < 17                                         # "ca. 16 GB"
    tb = g["matrix_examples"][1]["N"] ** 2 * 16 / 2 ** 40
    assert 33 < tb < 35                                         # "ca. 34 TB"
    for dg in g["double_grids"]:
        s = synth.System(synth.draw_model(0, 3, 4), dg["coarse"], dg["n_div"], 1, synth.POL3[:1])
        assert s.nk_dense == dg["dense"] ** 3 == s.nk_coarse * dg["N_div"]
    del ex_bytes


# ------------------------------------------------------------------ model
def test_single_k_point_closed_form():
    """One k point, one valence and one conduction band: H is the scalar
    Delta E + E_K [2 sum_G v(G) |mu(G)|^2 - h(0)/eps_inf] (Eqs. bse1-bse3b in
    the model), written out here without the oracle's matrix routines."""
    m = synth.draw_model(3, 1, 1)
    gm = om.GridModel(m, np.zeros((1, 3), dtype=np.int64), 1)
    K = om.kernel_matrix(gm)
    mu0 = m.mu[0] + m.mu[1] + m.mu[3] + m.mu[5]               # harmonics at k = 0
    G = synth.gvectors_nonzero()
    ex = 2 * np.sum(4 * np.pi / (G * G).sum(1) * np.abs(mu0[:, 0, 0]) ** 2)
    Gall = synth.gvectors_all()
    h0 = np.sum(np.exp(-(Gall * Gall).sum(1)) * 4 * np.pi / ((Gall * Gall).sum(1) + m.kappa ** 2))
    expect = m.e_k * (ex - h0 / m.eps_inf)
    assert K.shape == (1, 1)
    assert K[0, 0] == pytest.approx(expect, rel=1e-13)
    assert gm.dE[0, 0, 0] == pytest.approx(m.e_gap + m.offsets[0, 0], rel=1e-15)


def test_kernel_and_head_hermitian():
    I = tiny_interp()
    Hx, _ = om.explicit_dense_hamiltonian(I.model, 2, 2)
    for M in (I.Kc, I.A, Hx):
        assert np.abs(M - M.conj().T).max() < 1e-15 * max(1.0, np.abs(M).max()) * 10


def test_overlaps_unitary_and_consistent():
    """d = U(k~)^H U(k) is unitary, and d at k = k~ is the identity."""
    I = tiny_interp()
    for D in (I.Dv, I.Dc):
        eye = np.einsum("klnv,klnw->klvw", D.conj(), D)
        assert np.abs(eye - np.eye(D.shape[-1])).max() < 1e-13
    I1 = tiny_interp(nd=1)
    assert np.abs(I1.Dv[:, 0] - np.eye(I1.nv)).max() < 1e-13


def test_fft_explicit_operator_matches_dense():
    I = tiny_interp(n=3, nd=2)
    Hx, _ = om.explicit_dense_hamiltonian(I.model, 3, 2)
    op = om.ExplicitOperator(I.model, 3, 2)
    v = synth.random_vectors(11, I.N)
    assert np.abs(op.apply(v) - Hx @ v).max() < 1e-12


# ---------------------------------------------------------- interpolation
def test_restrict_is_adjoint_of_prolong_and_matches_dense_F():
    """Eqs. matmul1 / matmul3 are F^H and F of Eq. interpwfn."""
    I = tiny_interp(n=3, nd=2, nv=2, nc=3)
    F = I.F()
    s = synth.random_vectors(1, I.N)
    r = synth.random_vectors(2, I.Nc)
    assert np.abs(I.restrict(s) - F.conj().T @ s).max() < 1e-13
    assert np.abs(I.prolong(r) - F @ r).max() < 1e-13
    assert np.vdot(I.restrict(s), r) == pytest.approx(np.vdot(s, I.prolong(r)), rel=1e-13)


def test_ndiv1_interpolation_is_identity():
    """Dense mesh = coarse mesh: the interpolated H (M1 and M3) equals the explicit H."""
    I = tiny_interp(n=3, nd=1, nv=2, nc=2, width=1.0)
    Hx, _ = om.explicit_dense_hamiltonian(I.model, 3, 1)
    assert np.abs(I.H_dense("m1") - Hx).max() < 1e-13
    assert np.abs(I.H_dense("m3") - Hx).max() < 1e-13


@pytest.mark.parametrize("nd,scheme", [(2, "8nb"), (3, "8nb"), (2, "1nb"), (3, "1nb")])
def test_constant_model_m1_exact(nd, scheme):
    """mu k-independent and h constant: the model kernel is a fixed
    reference-basis tensor sandwiched between U(k)'s, so the expansion of
    Eq. expansion is exact and Eq. interp1 (with 1/N_div) reproduces the
    explicit dense kernel for any n_div and any neighbour weights."""
    I = tiny_interp(n=2, nd=nd, nv=2, nc=3, const_mu=True, h_const=True, scheme=scheme)
    Hx, _ = om.explicit_dense_hamiltonian(I.model, 2, nd)
    assert np.abs(I.H_dense("m1") - Hx).max() < 1e-13


def test_m1_not_exact_for_varying_model():
    """Control for the test above: with k-dependent mu and h the M1 kernel differs."""
    I = tiny_interp(n=2, nd=2)
    Hx, _ = om.explicit_dense_hamiltonian(I.model, 2, 2)
    assert np.abs(I.H_dense("m1") - Hx).max() > 1e-4


def test_m3_exact_on_near_pairs_for_head_only_model():
    """G = 0 shell only and constant mu: the head A is interpolated exactly
    and K_c - A h_head(q) is the (exactly interpolated) exchange, so M3 equals
    the explicit kernel on every near pair, and M1 on every far pair."""
    I = tiny_interp(n=4, nd=2, nv=2, nc=2, const_mu=True, shells=1, width=1.0)
    Hx, _ = om.explicit_dense_hamiltonian(I.model, 4, 2)
    H3, H1 = I.H_dense("m3"), I.H_dense("m1")
    near, _ = I.dense_q_tables()
    nb = np.kron(near, np.ones((I.t, I.t))).astype(bool)
    assert np.abs((H3 - Hx)[nb]).max() < 1e-13
    assert np.abs((H3 - H1)[~nb]).max() == 0.0
    assert np.abs((H1 - Hx)[nb]).max() > 1e-4                  # M1 alone is not exact there
    assert np.abs(H3 - H3.conj().T).max() < 1e-15


def test_matrix_free_m1_and_near_field_match_dense():
    I = tiny_interp(n=4, nd=2, nv=2, nc=2, width=1.0)
    v = synth.random_vectors(3, I.N)
    H1 = I.H_dense("m1")
    assert np.abs(I.apply_m1(v) - H1 @ v).max() < 1e-13
    rows = np.array([0, 5, 77, I.Nk - 1])
    d = ((I.H_dense("m3") - H1) @ v).reshape(I.Nk, -1)[rows]
    assert np.abs(I.near_field_rows(v, rows) - d).max() < 1e-14


def test_gauge_covariance_of_interpolated_spectrum():
    """Sec. 3: the phases carried by d cancel against P computed with the
    dense states.  A random phase on every dense band state (the gauge
    freedom of non-degenerate bands) leaves the M1 and M3 spectra unchanged;
    a conjugate in the wrong place in F, d or P breaks this."""
    base = tiny_interp(n=2, nd=2, nv=2, nc=2, width=0.5)
    rng = np.random.default_rng(5)
    Phv = np.stack([np.diag(np.exp(2j * np.pi * rng.random(2))) for _ in range(base.Nk)])
    Phc = np.stack([np.diag(np.exp(2j * np.pi * rng.random(2))) for _ in range(base.Nk)])
    tw = oi.Interp(base.model, 2, 2, width=0.5, dense_gauge_twist=(Phv, Phc))
    w = np.linspace(0, 5, 200)
    for meth in ("m1", "m3"):
        e0 = oh.epsilon_brute(base.H_dense(meth), base.dipole([1, 0, 0]), 1.0 / base.Nk, 0.1, w)
        e1 = oh.epsilon_brute(tw.H_dense(meth), tw.dipole([1, 0, 0]), 1.0 / base.Nk, 0.1, w)
        assert np.abs(e0 - e1).max() < 1e-11


def test_m3_closer_to_explicit_than_m1():
    """Sec. 5.1 trend (not a number): M3 beats M1 near the first peak on a held-out seed."""
    m = synth.draw_model(299, 2, 2)
    I = oi.Interp(m, 4, 2, width=1.0)
    Hx, _ = om.explicit_dense_hamiltonian(m, 4, 2)
    w = synth.frequency_grid(400)
    P = I.dipole([1, 0, 0])
    ex = oh.epsilon_brute(Hx, P, 1.0 / I.Nk, 0.1, w)
    e1 = oh.epsilon_brute(I.H_dense("m1"), P, 1.0 / I.Nk, 0.1, w)
    e3 = oh.epsilon_brute(I.H_dense("m3"), P, 1.0 / I.Nk, 0.1, w)
    assert oh.spectrum_error(e3.imag, ex.imag) < oh.spectrum_error(e1.imag, ex.imag)


# ----------------------------------------------------- Lanczos / fraction
def test_two_level_closed_form():
    """N = 2: the two-step fraction equals the exact resolvent element
    <P|(z - H)^-1|P> of a 2x2 Hermitian H, written with its adjugate."""
    e1, e2, v = 1.3, 2.1, 0.4 - 0.25j
    H = np.array([[e1, v], [np.conj(v), e2]])
    p = np.array([0.7 + 0.2j, -0.3 + 0.5j])
    a, b, pn2, _ = oh.haydock(lambda x: H @ x, p, 2)
    z = np.array([0.5 + 0.1j, 1.7 + 0.1j, 3.0 + 0.05j])
    det = (z - e1) * (z - e2) - abs(v) ** 2
    res = (abs(p[0]) ** 2 * (z - e2) + abs(p[1]) ** 2 * (z - e1)
           + np.conj(p[0]) * v * p[1] + np.conj(p[1]) * np.conj(v) * p[0]) / det
    assert np.allclose(pn2 * oh.continued_fraction(a, b, z), res, rtol=1e-13)
    assert a[0] == pytest.approx((np.vdot(p, H @ p) / pn2).real, rel=1e-14)


def test_lanczos_fraction_equals_brute_force_tiny():
    """N = 16 (coarse 2^3, n_div 1, 1v x 2c): m = N steps with full
    reorthogonalisation reproduce the diagonalisation spectrum."""
    m = synth.draw_model(21, 1, 2)
    I = oi.Interp(m, 2, 1)
    H = I.H_dense("m1")
    P = I.dipole([0.6, 0.8, 0.0])
    a, b, pn2, ima = oh.haydock(lambda x: H @ x, P, I.N, "cgs2")
    w = np.linspace(0, 6, 300)
    e = oh.epsilon(a, b, pn2, 1.0 / I.Nk, 0.1, w)
    eb = oh.epsilon_brute(H, P, 1.0 / I.Nk, 0.1, w)
    assert np.abs(e - eb).max() / np.abs(eb.imag).max() < 1e-10
    assert np.abs(ima).max() < 1e-13                            # a_i real for Hermitian H


def test_lanczos_fraction_equals_brute_force_medium():
    I = tiny_interp(n=2, nd=2, nv=2, nc=2)
    H = I.H_dense("m3")
    P = I.dipole([1, 0, 0])
    a, b, pn2, _ = oh.haydock(lambda x: H @ x, P, I.N, "cgs2")
    w = synth.frequency_grid(500)
    e = oh.epsilon(a, b, pn2, 1.0 / I.Nk, 0.1, w)
    eb = oh.epsilon_brute(H, P, 1.0 / I.Nk, 0.1, w)
    assert np.abs(e - eb).max() / np.abs(eb.imag).max() < 1e-10


def test_gauss_quadrature_moments():
    """T_m reproduces the moments <P|H^j|P> for j <= 2m - 1."""
    I = tiny_interp(n=2, nd=2, nv=2, nc=2)
    H = I.H_dense("m1")
    P = I.dipole([0, 1, 0])
    m = 6
    a, b, pn2, _ = oh.haydock(lambda x: H @ x, P, m, "cgs2")
    E, wts = oh.gauss_nodes(a, b, pn2)
    v = P.copy()
    for j in range(2 * m):
        mom = np.vdot(P, v).real
        assert np.sum(wts * E ** j) == pytest.approx(mom, rel=1e-10)
        v = H @ v


def test_independent_particle_limit():
    """K = 0: eps = 1 - (s/N_k) sum_vck |P_vck|^2 / (omega + i eta - Delta E_vck)."""
    m = synth.draw_model(4, 2, 2)
    m.e_k = 0.0
    I = oi.Interp(m, 2, 2, build_dense_kc=True)
    H = I.H_dense("m1")
    assert np.abs(H - np.diag(I.dE)).max() == 0.0
    P = I.dipole([0, 0, 1])
    a, b, pn2, _ = oh.haydock(lambda x: H @ x, P, I.N, "cgs2")
    w = synth.frequency_grid(300)
    e = oh.epsilon(a, b, pn2, 1.0 / I.Nk, 0.1, w)
    closed = 1 - (1.0 / I.Nk) * np.sum(np.abs(P)[None] ** 2 / (w[:, None] + 0.1j - I.dE[None]), axis=1)
    assert np.abs(e - closed).max() / np.abs(closed.imag).max() < 1e-10


def test_sum_rules():
    """Zeroth moment: (1/pi) int Im eps = (s/N_k) ||P||^2 (numerical integral
    of the fraction over a wide window plus analytic Lorentzian tails).
    First moment (TDA f-sum): sum_j w_j E_j = <P|H|P> = ||P||^2 a_1."""
    I = tiny_interp(n=2, nd=2, nv=2, nc=2)
    H = I.H_dense("m1")
    P = I.dipole([1, 1, 0])
    a, b, pn2, _ = oh.haydock(lambda x: H @ x, P, 40, "cgs2")
    E, wts = oh.gauss_nodes(a, b, pn2)
    pref, eta = 1.0 / I.Nk, 0.1
    lo, hi = -40.0, 45.0
    w = np.linspace(lo, hi, 400001)
    im = oh.epsilon(a, b, pn2, pref, eta, w).imag
    integral = np.sum((im[1:] + im[:-1]) / 2 * np.diff(w))
    tails = pref * np.sum(wts * (np.pi - (np.arctan((hi - E) / eta) - np.arctan((lo - E) / eta))))
    assert (integral + tails) / np.pi == pytest.approx(pref * pn2, rel=1e-6)
    assert np.sum(wts) == pytest.approx(pn2, rel=1e-12)
    assert np.sum(wts * E) == pytest.approx(np.vdot(P, H @ P).real, rel=1e-12)
    assert np.sum(wts * E) == pytest.approx(pn2 * a[0], rel=1e-12)


def test_sampled_rows_match_matrix_free_apply():
    """apply_m1_rows (K_c rows built on demand) equals the full matrix-free M1."""
    I = tiny_interp(n=3, nd=2, nv=2, nc=3)
    v = synth.random_vectors(12, I.N)
    rows = np.array([0, 7, 100, I.Nk - 1])
    full = I.apply_m1(v).reshape(I.Nk, I.t)[rows]
    assert np.abs(I.apply_m1_rows(v, rows) - full).max() < 1e-13
    Kr = om.kernel_rows(I.coarse, np.array([1, 5]))
    assert np.abs(Kr - I.Kc[np.r_[I.t:2 * I.t, 5 * I.t:6 * I.t]]).max() < 1e-15


# ------------------------------------------------------------------- Method 2
def test_m2_exact_on_every_pair_for_head_only_model():
    """Method 2 (Sec. 4) interpolates a and c for every pair and divides by the
    dense q.  G = 0 shell only and constant mu: a and c are interpolated
    exactly, so M2 equals the explicit kernel on every pair (near and far),
    where M3 is exact only on near pairs; M2 = M3 on near pairs in general."""
    I = tiny_interp(n=4, nd=2, nv=2, nc=2, const_mu=True, shells=1, width=1.0)
    Hx, _ = om.explicit_dense_hamiltonian(I.model, 4, 2)
    H2, H3 = I.H_dense("m2"), I.H_dense("m3")
    assert np.abs(H2 - Hx).max() < 1e-13
    near, _ = I.dense_q_tables()
    nb = np.kron(near, np.ones((I.t, I.t))).astype(bool)
    assert np.abs((H3 - Hx)[~nb]).max() > 1e-5                 # M3 is M1 (inexact) on far pairs
    J = tiny_interp(n=4, nd=2, nv=2, nc=2, width=1.0)          # varying model
    assert np.abs((J.H_dense("m2") - J.H_dense("m3"))[nb]).max() < 1e-15
    assert np.abs(J.H_dense("m2") - J.H_dense("m2").conj().T).max() < 1e-15


def test_m2_with_ndiv1_is_explicit():
    """Dense mesh = coarse mesh: M2 reduces to the explicit kernel too."""
    I = tiny_interp(n=3, nd=1, nv=2, nc=2, width=1.0)
    Hx, _ = om.explicit_dense_hamiltonian(I.model, 3, 1)
    assert np.abs(I.H_dense("m2") - Hx).max() < 1e-13


# ------------------------------------------------- adaptive stop (Sec. 5.1)
def test_converged_stop_rule():
    """Sec. 5.1 stops a chain once the spectrum changes by less than 1 % (real
    and imaginary parts).  The oracle's stop step must be a check point, the
    change at it must be within the tolerance and the change at every earlier
    check above it; the stopped spectrum must then be close to the exact one
    (brute-force diagonalisation of the same H)."""
    I = tiny_interp(n=4, nd=2, nv=2, nc=2, width=1.0)
    H = I.H_dense("m3")
    P = I.dipole([1, 0, 0])
    w = synth.frequency_grid(500)
    pref, eta, c, tol = 1.0 / I.Nk, 0.1, 5, 0.01
    a, b, pn2, _ = oh.haydock_until_converged(lambda v: H @ v, P, 400, c, tol, pref, eta, w, "cgs2")
    m = len(a)
    assert m % c == 0 and 2 * c <= m < 400
    changes = []
    for j in range(c, m + 1, c):
        changes.append(oh.epsilon(a[:j], b[:j + 1], pn2, pref, eta, w))
    d = [max(oh.spectrum_change(changes[i], changes[i - 1])) for i in range(1, len(changes))]
    assert d[-1] <= tol and all(x > tol for x in d[:-1])
    exact = oh.epsilon_brute(H, P, pref, eta, w)
    assert oh.spectrum_error(changes[-1].imag, exact.imag) < 5 * tol
