"""FP64 kernel mathematics of the paper, written from its definitions (test infrastructure).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``); shares no code with the product.

  phi(x)        modified exponential-of-semicircle kernel, Sec. 3.2 Eq. (semicircle2):
                phi(x) = exp(alpha beta [(1 - (2x/alpha)^2)^mu - 1]) on [-alpha/2, alpha/2],
                zero outside; mu = 1/2 gives the ES kernel of Eq. (semicircle).
  psi(k)        its Fourier transform, Sec. 2 below Eq. (rime3d), read as
                psi(k) = int phi(x) exp(2 pi i k x) dx  (x in grid cells, k in cycles per
                cell; the 2 pi is our reading of the garbled definition).
  map_error(k)  l(k) of Sec. 3.2 Eq. (maperror):
                l(k)^2 = int_0^1 | 1 - sum_j phi(j - nu) exp(2 pi i (j - nu) k) / psi(k) |^2 d nu
                evaluated literally (integral over the fractional visibility position nu).
  kernel_eps    sup of l(k) over the retained image |k| <= 1/(2 sigma) (Sec. 3.2: the
                supremum norm of the map error is the kernel's accuracy epsilon, App. A).

Integrals use tanh-sinh (double-exponential) quadrature, whose nodes cluster at the
interval ends, because phi has an algebraic (1 - s^2)^mu branch point at its support edge.
"""
from __future__ import annotations

import numpy as np


def phi(x, alpha, beta, mu):
    """Modified ES kernel (Eq. semicircle2), zero outside [-alpha/2, alpha/2]."""
    x = np.asarray(x, dtype=np.float64)
    s = 2.0 * x / alpha
    inside = np.abs(s) <= 1.0
    t = np.where(inside, 1.0 - s * s, 0.0)
    val = np.exp(alpha * beta * (t ** mu - 1.0))
    return np.where(inside, val, 0.0)


def _tanh_sinh(level=7, jmax_factor=4.0):
    """Nodes s in (-1, 1), 1 - s^2 and weights of tanh-sinh quadrature on [-1, 1]."""
    h = 2.0 ** (-level)
    j = np.arange(-int(jmax_factor / h), int(jmax_factor / h) + 1)
    t = j * h
    q = 0.5 * np.pi * np.sinh(t)
    s = np.tanh(q)
    one_minus_s2 = 1.0 / np.cosh(q) ** 2          # exact form of 1 - s^2, no cancellation
    w = h * 0.5 * np.pi * np.cosh(t) * one_minus_s2
    keep = w > 1e-300
    return s[keep], one_minus_s2[keep], w[keep]


_TS = _tanh_sinh()


def psi(k, alpha, beta, mu):
    """Fourier transform of phi at k (cycles per cell): int phi(x) cos(2 pi k x) dx."""
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    s, oms2, w = _TS
    # x = alpha s / 2; phi(x) = exp(alpha beta ((1 - s^2)^mu - 1))
    ph = np.exp(alpha * beta * (oms2 ** mu - 1.0))
    x = 0.5 * alpha * s
    return 0.5 * alpha * (np.cos(2.0 * np.pi * np.outer(k, x)) * (ph * w)).sum(axis=1)


def map_error(k, alpha, beta, mu):
    """l(k) of Eq. (maperror), by literal quadrature over nu in [0, 1)."""
    return map_error_of(k, alpha, lambda x: phi(x, alpha, beta, mu),
                        lambda kk: psi(kk, alpha, beta, mu))


def map_error_of(k, alpha, phi_fn, psi_fn):
    """l(k) of Eq. (maperror) for any kernel of support alpha given as callables
    phi_fn(x) (x in cells) and psi_fn(k) (its Fourier transform), by literal quadrature:
    l(k)^2 = int_0^1 | 1 - sum_j phi(j - nu) e^{2 pi i (j - nu) k} / psi(k) |^2 d nu."""
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    ps = np.asarray(psi_fn(k), dtype=np.float64)
    s, oms2, w = _TS
    # cells j with |j - nu| <= alpha/2 change only where nu - alpha/2 crosses an integer:
    # at nu = 0 (even alpha) or nu = 1/2 (odd alpha); integrate piecewise between them.
    if alpha % 2 == 0:
        pieces = [(0.0, 1.0)]
    else:
        pieces = [(0.0, 0.5), (0.5, 1.0)]
    out = np.zeros(k.size)
    for a, b in pieces:
        nu = 0.5 * (a + b) + 0.5 * (b - a) * s
        wn = 0.5 * (b - a) * w
        numid = 0.5 * (a + b)
        jlo = int(np.ceil(numid - alpha / 2.0)) - 1
        jhi = int(np.floor(numid + alpha / 2.0)) + 1
        acc = np.zeros((k.size, nu.size), dtype=np.complex128)
        for j in range(jlo, jhi + 1):
            x = j - nu
            f = np.asarray(phi_fn(x), dtype=np.float64)
            acc += f[None, :] * np.exp(2j * np.pi * np.outer(k, x))
        err = np.abs(1.0 - acc / ps[:, None]) ** 2
        out += (err * wn[None, :]).sum(axis=1)
    return np.sqrt(out)


def map_error_aliasing(k, alpha, beta, mu, mmax=40):
    """Closed form of l(k) by Poisson summation + Parseval (an independent route):
    l(k)^2 = sum_{m != 0} psi(k + m)^2 / psi(k)^2."""
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    num = np.zeros(k.size)
    for m in range(-mmax, mmax + 1):
        if m != 0:
            num += psi(k + m, alpha, beta, mu) ** 2
    return np.sqrt(num) / np.abs(psi(k, alpha, beta, mu))


def kernel_eps(alpha, beta, mu, sigma, nk=96):
    """sup_{|k| <= 1/(2 sigma)} l(k): the accuracy of a (alpha, sigma, beta, mu) kernel."""
    kmax = 0.5 / sigma
    k = np.linspace(0.0, kmax, nk)
    l = map_error(k, alpha, beta, mu)
    i = int(np.argmax(l))
    # refine around the maximum (l is smooth in k)
    lo, hi = k[max(i - 1, 0)], k[min(i + 1, nk - 1)]
    kk = np.linspace(lo, hi, 33)
    return float(max(l.max(), map_error(kk, alpha, beta, mu).max()))
