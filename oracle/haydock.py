"""Lanczos-Haydock recursion, continued fraction and brute force (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Index convention: a[i] = a_{i+1} (i = 0..m-1), b[i] = b_{i+1} (i = 0..m),
so b[0] = b_1 = 0 and b[i] for i >= 1 is the norm produced by step i.
"""
from __future__ import annotations

import numpy as np


def haydock(apply_h, p: np.ndarray, m: int, reorth: str = "none", breakdown_tol: float = 1e-12, stop=None):
    """Eqs. ai, bi, ci.

      b_1 = 0, psi_1 = P / ||P||
      a_i = <psi_i|H|psi_i>                       (real part; H is Hermitian)
      w   = H psi_i - a_i psi_i - b_i psi_{i-1}
      [reorth = "cgs2": classical Gram-Schmidt of w against psi_1..psi_i, twice]
      b_{i+1} = ||w||,  psi_{i+1} = w / b_{i+1}

    Stops early when b_{i+1} < breakdown_tol * max_j |a_j| (invariant subspace),
    or when stop(a, b, ||P||^2) returns True after a step (the coefficients of
    the steps done so far).
    Returns (a [steps], b [steps + 1], ||P||^2, imag_a [steps]).
    """
    pn2 = float(np.vdot(p, p).real)
    psi = p / np.sqrt(pn2)
    psi_prev = np.zeros_like(psi)
    a, b, ima = [], [0.0], []
    basis = [psi]
    for _ in range(m):
        w = apply_h(psi)
        ai = np.vdot(psi, w)
        a.append(float(ai.real))
        ima.append(float(ai.imag))
        w = w - ai.real * psi - b[-1] * psi_prev
        if reorth == "cgs2":
            V = np.array(basis)
            for _ in range(2):
                w = w - V.T @ (V.conj() @ w)
        elif reorth != "none":
            raise ValueError(reorth)
        bn = float(np.sqrt(np.vdot(w, w).real))
        b.append(bn)
        if bn < breakdown_tol * max(abs(x) for x in a):
            break
        if stop is not None and stop(np.array(a), np.array(b), pn2):
            break
        psi_prev, psi = psi, w / bn
        basis.append(psi)
    return np.array(a), np.array(b), pn2, np.array(ima)


def continued_fraction(a: np.ndarray, b: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Eq. fraccont, evaluated bottom-up and truncated (no terminator):
    g_m = 1/(z - a_m), g_i = 1/(z - a_i - b_{i+1}^2 g_{i+1}); returns g_1."""
    z = np.asarray(z, dtype=np.complex128)
    m = len(a)
    g = 1.0 / (z - a[m - 1])
    for i in range(m - 2, -1, -1):
        g = 1.0 / (z - a[i] - b[i + 1] ** 2 * g)
    return g


def epsilon(a, b, pn2, prefactor, eta, omega) -> np.ndarray:
    """eps_M(omega) = 1 - prefactor ||P||^2 g_1(omega + i eta)  (Eqs. epsmacro, fraccont);
    prefactor stands for the v(q) q->0 limit times the BZ weight (s / N_k)."""
    return 1.0 - prefactor * pn2 * continued_fraction(a, b, np.asarray(omega) + 1j * eta)


def epsilon_brute(H: np.ndarray, p: np.ndarray, prefactor, eta, omega) -> np.ndarray:
    """Eq. epsmacro by diagonalisation: 1 - prefactor sum_l |<l|P>|^2 / (omega + i eta - E_l)."""
    E, V = np.linalg.eigh(H)
    w = np.abs(V.conj().T @ p) ** 2
    z = np.asarray(omega)[:, None] + 1j * eta
    return 1.0 - prefactor * np.sum(w[None, :] / (z - E[None, :]), axis=1)


def tridiagonal(a, b) -> np.ndarray:
    m = len(a)
    T = np.diag(np.asarray(a, dtype=np.float64))
    for i in range(m - 1):
        T[i, i + 1] = T[i + 1, i] = b[i + 1]
    return T


def gauss_nodes(a, b, pn2):
    """Poles E_j and weights w_j of the truncated fraction: eig(T_m),
    w_j = ||P||^2 |first component|^2."""
    E, V = np.linalg.eigh(tridiagonal(a, b))
    return E, pn2 * V[0, :] ** 2


def spectrum_error(eps_im: np.ndarray, ref_im: np.ndarray) -> float:
    """max_w |Im eps - Im eps_ref| / max_w |Im eps_ref| (peak-normalised)."""
    return float(np.max(np.abs(eps_im - ref_im)) / np.max(np.abs(ref_im)))


def spectrum_change(eps_new: np.ndarray, eps_old: np.ndarray) -> tuple[float, float]:
    """Largest change of the real and of the imaginary part of eps over the
    frequency window, each relative to the largest |part| of the new spectrum."""
    d_re = float(np.max(np.abs(eps_new.real - eps_old.real)) / np.max(np.abs(eps_new.real)))
    d_im = float(np.max(np.abs(eps_new.imag - eps_old.imag)) / np.max(np.abs(eps_new.imag)))
    return d_re, d_im


def haydock_until_converged(apply_h, p: np.ndarray, max_steps: int, check_every: int, tol: float, prefactor,
                            eta, omega, reorth: str = "none"):
    """The stopping rule of Sec. 5.1: the chain runs until the whole dielectric
    spectrum changes by less than `tol` (1 %) in both its real and imaginary
    part.  Reading: eps is evaluated (Eq. fraccont) after every `check_every`
    steps, compared with the previous evaluation by spectrum_change, and the
    chain stops at the first check where both changes are <= tol.
    Returns haydock()'s tuple; len(a) is the number of steps done."""
    prev = {}

    def stop(a, b, pn2):
        j = len(a)
        if j % check_every:
            return False
        eps = epsilon(a, b, pn2, prefactor, eta, omega)
        old = prev.get("eps")
        prev["eps"] = eps
        if old is None:
            return False
        d_re, d_im = spectrum_change(eps, old)
        return d_re <= tol and d_im <= tol

    return haydock(apply_h, p, max_steps, reorth, stop=stop)
