"""Pins of the direct-sum oracle (oracle/direct.c) against facts other than itself.

Each test fixes a property the paper's Eq. (rime) and its adjoint must have, chosen so a
plausible slip in the oracle (a sign, the pixel offset -n/2, a transposed axis, the 1/n
factor, the frequency scaling, the real part of the adjoint) fails at least one of them:

  * w = 0 and u, v on the image's Fourier lattice reduce Eq. (rime) to a 2-D DFT, which
    numpy.fft computes independently (library reduction);
  * the phase of a point source moves with u and w at the rates -2 pi l and +2 pi (n - 1)
    that Eq. (rime) prescribes (sign pins, measured by finite differences of the output);
  * degrid and grid are adjoint (Sec. 5.1, Eq. adjointness) to FP64 rounding;
  * the Hermitian transformation (u, v, w, d) -> (-u, -v, -w, d*) leaves Eq. (rime)
    invariant (Sec. 2, Eq. Hermitian-symmetry);
  * mask / weight / do_wstacking behave as App. B describes.
"""
import numpy as np
import pytest

C = 299792458.0


def _ncoord(nx, ny, psx, psy):
    l = (np.arange(nx) - nx // 2) * psx
    m = (np.arange(ny) - ny // 2) * psy
    L, M = np.meshgrid(l, m, indexing="ij")
    return L, M, np.sqrt(1.0 - L**2 - M**2)


def test_fft_lattice_reduction(oracle_lib):
    """w = 0, u = p / (nx dl), v = q / (ny dm): degrid = (-1)^(p+q) FFT2(I/n)[p, q]."""
    rng = np.random.default_rng(1)
    nx, ny = 32, 40                       # unequal sides catch a transposed axis
    psx, psy = np.deg2rad(0.7), np.deg2rad(0.45)
    I = rng.standard_normal((nx, ny))
    _, _, n = _ncoord(nx, ny, psx, psy)
    F = np.fft.fft2(I / n)
    freq = np.array([0.7e9, 1.3e9])        # two channels: u = u~ f / c
    p = rng.integers(-nx // 2, nx // 2, size=12)
    q = rng.integers(-ny // 2, ny // 2, size=12)
    # rows chosen so that channel 0 lands on (p, q); channel 1 is a scaled copy
    uvw = np.stack([p / (nx * psx) * C / freq[0], q / (ny * psy) * C / freq[0],
                    np.zeros(12)], axis=1)
    vis = oracle_lib.degrid(uvw, freq, I, psx, psy)
    expect = ((-1.0) ** (p + q)) * F[p % nx, q % ny]
    np.testing.assert_allclose(vis[:, 0], expect, rtol=0, atol=1e-11 * np.abs(F).max())
    # the adjoint on the same lattice: grid(delta_k) = Re((-1)^(p+q) e^{+2 pi i(...)}) / n
    d = np.zeros((12, 2), dtype=complex)
    d[3, 0] = 0.6 - 0.8j
    img = oracle_lib.grid(uvw, freq, d, nx, ny, psx, psy)
    jx = np.arange(nx)[:, None]; jy = np.arange(ny)[None, :]
    ph = np.exp(2j * np.pi * (p[3] * jx / nx + q[3] * jy / ny)) * (-1.0) ** (p[3] + q[3])
    np.testing.assert_allclose(img, np.real(ph * d[3, 0]) / n, rtol=0, atol=1e-13)


def test_phase_rates_pin_signs(oracle_lib):
    """d(arg d)/du = -2 pi l0 and d(arg d)/dw = +2 pi (n0 - 1) for a point source (Eq. rime)."""
    nx = ny = 32
    ps = np.deg2rad(1.5)
    I = np.zeros((nx, ny)); j0, k0 = 7, 25                 # off-centre, both axes
    I[j0, k0] = 1.0
    l0, m0 = (j0 - nx // 2) * ps, (k0 - ny // 2) * ps
    n0 = np.sqrt(1 - l0**2 - m0**2)
    freq = np.array([C])                                   # lambda = 1 m: uvw in wavelengths
    base = np.array([[13.0, -4.0, 21.0]])
    h = 1e-3
    rows = np.concatenate([base, base + [h, 0, 0], base + [0, h, 0], base + [0, 0, h]])
    vis = oracle_lib.degrid(rows, freq, I, ps, ps)[:, 0]
    rate = np.angle(vis[1:] / vis[0]) / h
    np.testing.assert_allclose(rate, [-2 * np.pi * l0, -2 * np.pi * m0, 2 * np.pi * (n0 - 1)],
                               rtol=1e-6)
    np.testing.assert_allclose(np.abs(vis), 1.0 / n0, rtol=1e-14)
    assert n0 - 1 < 0 and rate[2] < 0                      # w-phase falls off-centre


def _wide_case(rng, nrows=60, nchan=3, nx=48, ny=36, fov_deg=20.0):
    psx = np.deg2rad(fov_deg) / nx
    psy = np.deg2rad(fov_deg * 0.8) / ny
    freq = np.linspace(0.9e9, 1.4e9, nchan)
    umax = 0.45 / psx * C / freq[-1]
    uvw = np.stack([rng.uniform(-umax, umax, nrows), rng.uniform(-umax, umax, nrows),
                    rng.uniform(-umax, umax, nrows)], axis=1)
    return uvw, freq, nx, ny, psx, psy


def test_adjointness(oracle_lib):
    """Sec. 5.1 Eq. (adjointness): Re<R0 I, d> = <I, R0^dagger d>, to FP64 rounding."""
    rng = np.random.default_rng(2)
    uvw, freq, nx, ny, psx, psy = _wide_case(rng)
    I = rng.uniform(-0.5, 0.5, (nx, ny))
    d = rng.uniform(-0.5, 0.5, (uvw.shape[0], freq.size)) + 1j * rng.uniform(-0.5, 0.5, (uvw.shape[0], freq.size))
    wgt = rng.uniform(0.5, 2.0, d.shape)
    mask = (rng.uniform(size=d.shape) > 0.2).astype(np.uint8)
    RI = oracle_lib.degrid(uvw, freq, I, psx, psy, wgt=wgt, mask=mask)
    Rd = oracle_lib.grid(uvw, freq, d, nx, ny, psx, psy, wgt=wgt, mask=mask)
    assert oracle_lib.adjointness_error(I, RI, d, Rd) < 1e-14


def test_hermitian_fold_invariance(oracle_lib):
    """(u, v, w, d) -> (-u, -v, -w, d*) leaves Eq. (rime) invariant (Sec. 2)."""
    rng = np.random.default_rng(3)
    uvw, freq, nx, ny, psx, psy = _wide_case(rng, nrows=20)
    I = rng.standard_normal((nx, ny))
    a = oracle_lib.degrid(uvw, freq, I, psx, psy)
    b = oracle_lib.degrid(-uvw, freq, I, psx, psy)
    np.testing.assert_allclose(b, np.conj(a), rtol=0, atol=1e-12 * np.abs(a).max())
    d = rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)
    g1 = oracle_lib.grid(uvw, freq, d, nx, ny, psx, psy)
    g2 = oracle_lib.grid(-uvw, freq, np.conj(d), nx, ny, psx, psy)
    np.testing.assert_allclose(g1, g2, rtol=0, atol=1e-12 * np.abs(g1).max())


def test_mask_weights_and_no_wstacking(oracle_lib):
    """App. B: wgt scales, mask == 0 removes a visibility, do_wstacking=False sets w = 0."""
    rng = np.random.default_rng(4)
    uvw, freq, nx, ny, psx, psy = _wide_case(rng, nrows=15, nchan=2)
    I = rng.standard_normal((nx, ny))
    full = oracle_lib.degrid(uvw, freq, I, psx, psy)
    wgt = rng.uniform(0.1, 3, full.shape)
    mask = np.ones(full.shape, np.uint8); mask[2, 1] = 0; mask[7, 0] = 0
    out = oracle_lib.degrid(uvw, freq, I, psx, psy, wgt=wgt, mask=mask)
    np.testing.assert_allclose(out, full * wgt * mask, rtol=1e-14, atol=1e-14)
    flat = uvw.copy(); flat[:, 2] = 0.0
    np.testing.assert_allclose(oracle_lib.degrid(uvw, freq, I, psx, psy, do_wstacking=False),
                               oracle_lib.degrid(flat, freq, I, psx, psy), rtol=1e-15, atol=1e-15)
    d = rng.standard_normal(full.shape) + 1j * rng.standard_normal(full.shape)
    g = oracle_lib.grid(uvw, freq, d, nx, ny, psx, psy, wgt=wgt, mask=mask)
    np.testing.assert_allclose(g, oracle_lib.grid(uvw, freq, d * wgt * mask, nx, ny, psx, psy),
                               rtol=1e-12, atol=1e-12)


def test_subsets_match_full(oracle_lib):
    rng = np.random.default_rng(5)
    uvw, freq, nx, ny, psx, psy = _wide_case(rng, nrows=10, nchan=2)
    I = rng.standard_normal((nx, ny))
    full = oracle_lib.degrid(uvw, freq, I, psx, psy)
    sel = np.array([3, 0, 19, 7])
    np.testing.assert_array_equal(oracle_lib.degrid(uvw, freq, I, psx, psy, vis_index=sel),
                                  full.reshape(-1)[sel])
    d = rng.standard_normal(full.shape) + 1j * rng.standard_normal(full.shape)
    g = oracle_lib.grid(uvw, freq, d, nx, ny, psx, psy)
    psel = np.array([0, 5, nx * ny - 1, 777])
    np.testing.assert_array_equal(oracle_lib.grid(uvw, freq, d, nx, ny, psx, psy, pixel_index=psel),
                                  g.reshape(-1)[psel])


def test_brute_force_matrix_tiny(oracle_lib):
    """n = 32, 10 visibilities: the oracle equals an explicit dense matrix built by numpy
    in long double from Eq. (rime)'s definition (a different summation route)."""
    rng = np.random.default_rng(6)
    uvw, freq, nx, ny, psx, psy = _wide_case(rng, nrows=10, nchan=1, nx=32, ny=32)
    L, M, n = _ncoord(nx, ny, psx, psy)
    u, v, w = (uvw * freq[0] / C).T
    ph = (u[:, None, None] * L + v[:, None, None] * M - w[:, None, None] * (n - 1)).reshape(10, -1)
    A = np.exp(-2j * np.pi * ph) / n.reshape(1, -1)
    I = rng.standard_normal((nx, ny))
    np.testing.assert_allclose(oracle_lib.degrid(uvw, freq, I, psx, psy)[:, 0], A @ I.reshape(-1),
                               rtol=0, atol=1e-10)
    d = rng.standard_normal(10) + 1j * rng.standard_normal(10)
    np.testing.assert_allclose(oracle_lib.grid(uvw, freq, d[:, None], nx, ny, psx, psy).reshape(-1),
                               np.real(A.conj().T @ d), rtol=0, atol=1e-10)


def test_rejects_fov_beyond_unit_disc(oracle_lib):
    with pytest.raises(ValueError):
        oracle_lib.degrid(np.zeros((1, 3)), np.array([1e9]), np.ones((32, 32)), 0.1, 0.1)
