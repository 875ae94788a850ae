"""Pins of the model's k dependence away from k = 0.

At k = 0 every sine harmonic vanishes and 1 - cos 2 pi k = 0, so the k = 0
closed form cannot see a wrong slot order, a missing 2 pi, a wrong band-width
factor or a conjugate on the wrong gauge matrix.  These tests evaluate the
model at k = (1/4, 1/8, 3/8) and k = (1/4, 0, 0), where the trigonometric
values are exact (0, 1, 1/sqrt 2), and compare with the values written out by
hand from the model's definition (energies, harmonics, band gauge, exchange
form factors M = U_v^H mu U_c, dipoles P = U_v^T pi conj U_c).
"""
import numpy as np
import pytest

from oracle import model as om
from paper_1602_01863_gb300 import synth

R = 1.0 / np.sqrt(2.0)
K1 = np.array([0.25, 0.125, 0.375])          # 2 pi k = (pi/2, pi/4, 3 pi/4)
# (1, cos 2pi k1, sin 2pi k1, cos 2pi k2, sin 2pi k2, cos 2pi k3, sin 2pi k3) at K1
HARM_K1 = np.array([1.0, 0.0, 1.0, R, R, -R, R])


def _model(nv, nc, gen_v, gen_c, seed=17):
    base = synth.draw_model(seed, nv, nc)
    return synth.ModelParams(nv=nv, nc=nc, eps_inf=base.eps_inf, kappa=base.kappa, offsets=base.offsets,
                             gen_v=gen_v, gen_c=gen_c, mu=base.mu, dip=base.dip)


def test_harmonics_at_k_nonzero():
    got = om.harmonics(K1[None])[0]
    assert np.abs(got - HARM_K1).max() < 1e-15


def test_energies_at_k_nonzero():
    """Delta E = 1.1 + 0.3 sum_i (1 - cos 2 pi k_i) + o: at K1 the cosines are
    0, 1/sqrt 2, -1/sqrt 2, so the sum is 3 and Delta E = 2.0 + o exactly; at
    (1/4, 0, 0) it is 1.4 + o."""
    m = synth.draw_model(5, 2, 3)
    e = om.energies(m, np.stack([K1, [0.25, 0.0, 0.0]]))
    assert np.abs(e[0] - (2.0 + m.offsets)).max() < 1e-14
    assert np.abs(e[1] - (1.4 + m.offsets)).max() < 1e-14


def test_one_band_gauge_form_factor_dipole_at_k_nonzero():
    """One valence and one conduction band: the generators are real numbers,
    U(k) = exp(i a(k)) with a = sum_a sin(2 pi k_a) g_a0 + (1 - cos 2 pi k_a) g_a1,
    M(k, G) = conj(u_v) mu(k, G) u_c and P^alpha = u_v pi^alpha(k) conj(u_c)."""
    gv = np.array([0.3, -0.2, 0.5, 0.1, -0.4, 0.25]).reshape(3, 2, 1, 1).astype(np.complex128)
    gc = np.array([-0.15, 0.35, 0.2, -0.3, 0.45, 0.05]).reshape(3, 2, 1, 1).astype(np.complex128)
    m = _model(1, 1, gv, gc)
    # sin(2 pi k) = (1, R, R), 1 - cos(2 pi k) = (1, 1 - R, 1 + R) at K1
    s, omc = np.array([1.0, R, R]), np.array([1.0, 1.0 - R, 1.0 + R])
    av = float(np.sum(s * gv[:, 0, 0, 0].real + omc * gv[:, 1, 0, 0].real))
    ac = float(np.sum(s * gc[:, 0, 0, 0].real + omc * gc[:, 1, 0, 0].real))
    uv, uc = np.exp(1j * av), np.exp(1j * ac)
    Uv = om.gauge(m.gen_v, K1[None])
    Uc = om.gauge(m.gen_c, K1[None])
    assert abs(Uv[0, 0, 0] - uv) < 1e-14 and abs(Uc[0, 0, 0] - uc) < 1e-14
    mu_k = (m.mu[0] + m.mu[2] + R * m.mu[3] + R * m.mu[4] - R * m.mu[5] + R * m.mu[6])[:, 0, 0]   # [26]
    M = om.form_factors(m, Uv, Uc, K1[None])[0, :, 0, 0]
    assert np.abs(M - np.conj(uv) * mu_k * uc).max() < 1e-14
    pi_k = (m.dip[0] + m.dip[2] + R * m.dip[3] + R * m.dip[4] - R * m.dip[5] + R * m.dip[6])[:, 0, 0]  # [3]
    P = om.dipoles(m, Uv, Uc, K1[None])[0, :, 0, 0]
    assert np.abs(P - uv * pi_k * np.conj(uc)).max() < 1e-14


def test_two_band_gauge_placement_at_k_nonzero():
    """Two valence bands whose generators are multiples of sigma_x: at
    k = (1/4, 0, 0) the exponent is (pi/8 + pi/8) sigma_x, so
    U_v = (I + i sigma_x) / sqrt 2.  With one conduction band (gauge 1):
      M_0 = (mu_0 - i mu_1) / sqrt 2,  M_1 = (-i mu_0 + mu_1) / sqrt 2   (U_v^H mu)
      P_0 = (pi_0 + i pi_1) / sqrt 2,  P_1 = (i pi_0 + pi_1) / sqrt 2    (U_v^T pi)
    with mu, pi at the harmonics (1, 0, 1, 1, 0, 1, 0) of that k."""
    sx = np.array([[0.0, 1.0], [1.0, 0.0]], dtype=np.complex128)
    gv = np.zeros((3, 2, 2, 2), dtype=np.complex128)
    gv[0, 0] = np.pi / 8 * sx
    gv[0, 1] = np.pi / 8 * sx
    gv[1, 0] = 0.7 * sx                        # axes 2 and 3 do not enter at k2 = k3 = 0
    gv[2, 1] = -0.4 * sx
    gc = np.zeros((3, 2, 1, 1), dtype=np.complex128)
    m = _model(2, 1, gv, gc)
    k = np.array([[0.25, 0.0, 0.0]])
    Uv = om.gauge(m.gen_v, k)
    Uc = om.gauge(m.gen_c, k)
    assert np.abs(Uv[0] - R * np.array([[1, 1j], [1j, 1]])).max() < 1e-14
    assert np.abs(Uc[0] - 1.0).max() < 1e-15
    mu_k = m.mu[0] + m.mu[2] + m.mu[3] + m.mu[5]          # [26, 2, 1]
    M = om.form_factors(m, Uv, Uc, k)[0]                   # [26, 2, 1]
    assert np.abs(M[:, 0, 0] - R * (mu_k[:, 0, 0] - 1j * mu_k[:, 1, 0])).max() < 1e-14
    assert np.abs(M[:, 1, 0] - R * (-1j * mu_k[:, 0, 0] + mu_k[:, 1, 0])).max() < 1e-14
    pi_k = m.dip[0] + m.dip[2] + m.dip[3] + m.dip[5]      # [3, 2, 1]
    P = om.dipoles(m, Uv, Uc, k)[0]                        # [3, 2, 1]
    assert np.abs(P[:, 0, 0] - R * (pi_k[:, 0, 0] + 1j * pi_k[:, 1, 0])).max() < 1e-14
    assert np.abs(P[:, 1, 0] - R * (1j * pi_k[:, 0, 0] + pi_k[:, 1, 0])).max() < 1e-14


def test_single_point_kernel_at_k_nonzero():
    """One k point at K1 (grid L = 8, integer coordinate (2, 1, 3)), one band each:
    K = E_K [2 sum_G v(G) |mu(K1, G)|^2 - h(0) / eps_inf], the gauge phases
    cancelling in |M|^2 and in O^v O^c = 1."""
    m = synth.draw_model(8, 1, 1)
    gm = om.GridModel(m, np.array([[2, 1, 3]]), 8)
    assert np.abs(gm.kfrac[0] - K1).max() == 0.0
    K = om.kernel_matrix(gm)
    mu_k = (m.mu[0] + m.mu[2] + R * m.mu[3] + R * m.mu[4] - R * m.mu[5] + R * m.mu[6])[:, 0, 0]
    G = synth.gvectors_nonzero()
    ex = 2 * np.sum(4 * np.pi / (G * G).sum(1) * np.abs(mu_k) ** 2)
    Gall = synth.gvectors_all()
    h0 = np.sum(np.exp(-(Gall * Gall).sum(1)) * 4 * np.pi / ((Gall * Gall).sum(1) + m.kappa ** 2))
    assert K[0, 0] == pytest.approx(m.e_k * (ex - h0 / m.eps_inf), rel=1e-13)
    assert gm.dE[0, 0, 0] == pytest.approx(2.0 + m.offsets[0, 0], rel=1e-15)
