"""Pins of the kernel mathematics in oracle/kernel_math.py against the paper's App. A.

The kernel-parameter table of App. A (tests/golden/kernel_table_appA.txt, values as printed)
lists, for each (alpha, sigma), the parameters (beta, mu) of the modified ES kernel and the
accuracy epsilon it reaches.  epsilon is the supremum over the retained image of the map
error function l(x) of Eq. (maperror).  Recomputing it from (alpha, sigma, beta, mu) pins at
once: the kernel formula (Eq. semicircle2), the reading psi(k) = int phi(x) e^{2 pi i k x} dx
(with the 2 pi), and the retained range |k| <= 1/(2 sigma).
"""
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import kernel_math as km

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "kernel_table_appA.txt")


def table_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            a, s, e, b, m = line.split()
            rows.append((int(a), float(s), float(e), float(b), float(m)))
    return rows


def test_table_shape():
    rows = table_rows()
    assert len(rows) == 86
    assert sorted({r[0] for r in rows}) == [4, 7, 8, 12, 16]


@pytest.mark.parametrize("row", table_rows(), ids=lambda r: f"a{r[0]}-s{r[1]}")
def test_map_error_reproduces_table_epsilon(row):
    alpha, sigma, eps, beta, mu = row
    got = km.kernel_eps(alpha, beta, mu, sigma)
    # below ~1e-12 the literal |1 - sum/psi|^2 sits at the FP64 cancellation floor
    tol = 0.03 if eps >= 1e-12 else 0.25
    assert abs(got / eps - 1) < tol, (got, eps)


def test_two_routes_to_the_map_error_agree():
    """Literal Eq. (maperror) integral over nu vs its Poisson/Parseval closed form
    l(k)^2 = sum_{m != 0} psi(k + m)^2 / psi(k)^2 (tail beyond |m| = 80 ~ 1e-4 relative)."""
    alpha, beta, mu = 8, 1.7876782642, 0.5176319503
    k = np.array([0.0, 0.17, 0.33])
    saved = km._TS
    try:
        km._TS = km._tanh_sinh(level=11)      # resolve psi(k + m) oscillations up to m = 80
        ali = km.map_error_aliasing(k, alpha, beta, mu, mmax=80)
    finally:
        km._TS = saved
    lit = km.map_error(k, alpha, beta, mu)
    np.testing.assert_allclose(ali, lit, rtol=2e-3)


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
def test_psi_against_scipy_quad():
    """psi by tanh-sinh vs scipy.integrate.quad with the algebraic end-point weight."""
    alpha, beta, mu = 7, 1.868082272, 0.5206277502
    for k in [0.0, 0.21, 0.5, 1.3]:
        ref, _ = integrate.quad(lambda x: km.phi(x, alpha, beta, mu) * np.cos(2 * np.pi * k * x),
                                -alpha / 2, alpha / 2, limit=400, epsabs=1e-15, epsrel=1e-13)
        assert abs(km.psi(k, alpha, beta, mu)[0] - ref) < 1e-11


def test_mu_half_is_the_es_kernel():
    """Eq. (semicircle2) with mu = 1/2 is the ES kernel of Eq. (semicircle)."""
    x = np.linspace(-3.0, 3.0, 41)
    es = np.exp(6 * 2.1 * (np.sqrt(np.clip(1 - (2 * x / 6) ** 2, 0, None)) - 1))
    np.testing.assert_allclose(km.phi(x, 6, 2.1, 0.5), es, rtol=1e-15)
    assert km.phi(3.01, 6, 2.1, 0.5) == 0.0
