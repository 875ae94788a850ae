"""Pins of the learned-residual oracle (MLP, Adam, pair data, stencil)."""
import numpy as np
import pytest
from scipy.stats import norm

from oracle import interp as oi
from oracle import learned as ol
from oracle import model as om
from paper_1602_01863_gb300 import synth


def test_gelu_exact_values():
    """gelu(z) = z Phi(z) with the normal CDF (exact, erf form)."""
    z = np.array([-2.0, -1.0, 0.0, 0.5, 1.0, 3.0])
    assert np.allclose(ol.gelu(z), z * norm.cdf(z), rtol=1e-14, atol=1e-16)
    h = 1e-6
    assert np.allclose(ol.gelu_grad(z), (ol.gelu(z + h) - ol.gelu(z - h)) / (2 * h), rtol=1e-8)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    params = ol.init_params(10, seed=1, width=8)
    X = rng.standard_normal((5, 10))
    Y = rng.standard_normal((5, 2))
    out, cache = ol.forward(params, X)
    _, dout = ol.loss_and_grad_out(out, Y)
    grads = ol.backward(params, cache, dout)
    h = 1e-6
    for layer in range(ol.LAYERS):
        for j in range(2):
            p = params[layer][j]
            flat = p.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp, _ = ol.loss_and_grad_out(ol.forward(params, X)[0], Y)
                flat[idx] = old - h
                lm, _ = ol.loss_and_grad_out(ol.forward(params, X)[0], Y)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                assert grads[layer][j].reshape(-1)[idx] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_adam_first_step_is_signed_learning_rate():
    """With m = v = 0 the bias-corrected first step is lr g / (|g| + eps)."""
    params = ol.init_params(4, seed=2, width=3)
    grads = [[np.full_like(W, 0.3), np.full_like(b, -2.0)] for W, b in params]
    m = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
    v = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
    before = [[W.copy(), b.copy()] for W, b in params]
    ol.adam_update(params, grads, m, v, step=1, lr=0.01)
    for layer in range(ol.LAYERS):
        assert np.allclose(before[layer][0] - params[layer][0], 0.01 * 0.3 / (0.3 + 1e-8))
        assert np.allclose(before[layer][1] - params[layer][1], -0.01 * 2.0 / (2.0 + 1e-8))


def _tiny(seed=3, const=False):
    m = synth.draw_model(seed, 2, 2, const_mu=const, h_const=const)
    I = oi.Interp(m, 2, 4)
    Hx, _ = om.explicit_dense_hamiltonian(m, 2, 4)
    return I, Hx, I.H_dense("m1")


def test_residual_vanishes_where_interpolation_is_exact():
    """Constant model: M1 is exact (Eq. interp1), so every residual target is 0."""
    I, Hx, H1 = _tiny(const=True)
    rng = np.random.default_rng(4)
    kd = rng.integers(0, I.Nk, 50)
    kd2 = rng.integers(0, I.Nk, 50)
    tr = rng.integers(0, I.t, 50)
    X, Y = ol.residual_samples(I, Hx, H1, kd, kd2, tr, tr[::-1].copy())
    assert np.abs(Y).max() < 1e-10
    assert X.shape == (50, 6 + 2 * I.t)
    assert np.all(X[np.arange(50), 4 + tr] == 1.0)


def test_stencil_hermitian_and_convolutions_agree():
    I, _, _ = _tiny()
    params = ol.init_params(6 + 2 * I.t, seed=5)
    offs, T = ol.stencil(params, I, 3, ol.mean_dE(I))
    idx = {tuple(o): i for i, o in enumerate(offs)}
    for i, o in enumerate(offs):
        assert np.allclose(T[idx[tuple(-o)]], T[i].conj().T, atol=1e-15)
    psi = synth.random_vectors(6, I.N)
    a = ol.apply_stencil_direct(I, offs, T, psi)
    b = ol.apply_stencil_fft(I, offs, T, psi)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
    # Hermitian operator: <x, T y> = <T x, y>
    x = synth.random_vectors(7, I.N)
    assert np.vdot(x, ol.apply_stencil_direct(I, offs, T, psi)) == pytest.approx(
        np.vdot(ol.apply_stencil_direct(I, offs, T, x), psi), rel=1e-12)
