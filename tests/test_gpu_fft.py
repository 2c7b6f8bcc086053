"""The double-float (df64) plane FFT against cuFFT's double-precision transform.

Both are unnormalised 2-D transforms of complex128 planes (forward e^{-2 pi i}); the df64
transform carries each value as a pair of floats (48-bit significand), so it is expected to
agree with the FP64 transform to ~1e-14 relative L2 (normwise), far below the eps >= 1e-12
the FP64 mode serves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wg():
    from paper_2010_10122_gb300 import _build
    _build.build()
    import paper_2010_10122_gb300 as wg
    assert torch.cuda.is_available()
    return wg


@pytest.mark.parametrize("shape", [(1, 32, 48), (3, 96, 160), (2, 224, 352), (1, 3200, 3200),
                                   (1, 2816, 2304), (2, 1344, 1760), (1, 704, 6400)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_df64_matches_cufft_z2z(wg, shape, sign):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    a = torch.from_numpy(x).cuda()
    b = a.clone()
    wg.wgrid.fft2d(a, sign=sign, impl=2)
    wg.wgrid.fft2d(b, sign=sign, impl=1)
    err = ((a - b).abs().pow(2).sum() / b.abs().pow(2).sum()).sqrt().item()
    assert err < 5e-14, err


def test_df64_against_numpy_small(wg):
    rng = np.random.default_rng(7)
    x = rng.standard_normal((2, 40, 56)) + 1j * rng.standard_normal((2, 40, 56))
    a = torch.from_numpy(x).cuda()
    wg.wgrid.fft2d(a, sign=-1, impl=2)
    ref = np.fft.fft2(x)
    assert np.linalg.norm(a.cpu().numpy() - ref) / np.linalg.norm(ref) < 5e-14


@pytest.mark.parametrize("shape", [(2, 12, 7040), (1, 16, 13824), (1, 13824, 16), (1, 6912, 40),
                                   (1, 24, 25600)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_df64_split_lines_against_numpy(wg, shape, sign):
    """Sides above 6400 run each line on 2 CTAs (7040, 6912) or 4 CTAs (13824, 25600), one
    radix-2 / radix-4 decimation-in-frequency step folded into the loads; both passes (rows and
    the strided columns) against numpy's FFT."""
    rng = np.random.default_rng(sum(shape) + sign)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    a = torch.from_numpy(x).cuda()
    wg.wgrid.fft2d(a, sign=sign, impl=2)
    ref = np.fft.fft2(x) if sign < 0 else np.fft.ifft2(x) * (shape[1] * shape[2])
    assert np.linalg.norm(a.cpu().numpy() - ref) / np.linalg.norm(ref) < 5e-14


@pytest.mark.parametrize("shape", [(1, 32, 48), (3, 96, 160), (2, 224, 352), (1, 2816, 2304),
                                   (2, 1344, 1760), (1, 5632, 64), (1, 64, 11264), (1, 11264, 32),
                                   (1, 6000, 40), (1, 40, 7056)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_f32_fft_matches_cufft_c2c(wg, shape, sign):
    """The library's FP32 plane FFT (impl 4; long lines on clusters of 2, 4 or 8 CTAs) against
    cuFFT's C2C on the same complex64 planes: both round in FP32, so they agree to a few 1e-7
    (normwise)."""
    rng = np.random.default_rng(sum(shape) + 7 * sign)
    x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    a = torch.from_numpy(x).cuda()
    b = a.clone()
    wg.wgrid.fft2d(a, sign=sign, impl=4)
    wg.wgrid.fft2d(b, sign=sign, impl=1)
    err = ((a - b).abs().pow(2).sum() / b.abs().pow(2).sum()).sqrt().item()
    assert err < 2e-6, err
    ref = np.fft.fft2(x.astype(np.complex128)) if sign < 0 else \
        np.fft.ifft2(x.astype(np.complex128)) * (shape[1] * shape[2])
    assert np.linalg.norm(a.cpu().numpy() - ref) / np.linalg.norm(ref) < 2e-6


@pytest.mark.parametrize("tune", [(4, 256, 8), (2, 64, 2), (8, 12800, 16), (1, 1024, 4),
                                  (4, 12800, 8)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_f32_fft_shapes(wg, tune, sign):
    """Every shape of the FP32 line kernels gives the same transform: columns per CTA 1, 2, 4, 8,
    lines on one CTA or split over clusters of 2, 4, 8 CTAs (small part sizes force the splits
    on small planes), against numpy in FP64."""
    try:
        wg.wgrid.fft_f32_tune(*tune)
        for shape in [(2, 512, 448), (1, 176, 1056), (3, 96, 120)]:
            rng = np.random.default_rng(sum(shape) + sign)
            x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
            a = torch.from_numpy(x).cuda()
            wg.wgrid.fft2d(a, sign=sign, impl=4)
            ref = np.fft.fft2(x.astype(np.complex128)) if sign < 0 else \
                np.fft.ifft2(x.astype(np.complex128)) * (shape[1] * shape[2])
            err = np.linalg.norm(a.cpu().numpy() - ref) / np.linalg.norm(ref)
            assert err < 2e-6, (tune, shape, err)
    finally:
        wg.wgrid.fft_f32_tune(0, 0, 0)


def test_df64_rejects_unsupported(wg):
    a = torch.zeros((1, 64, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(wg.WgridError):
        wg.wgrid.fft2d(a, impl=2)           # single precision
    b = torch.zeros((1, 13 * 8, 64), dtype=torch.complex128, device="cuda")
    with pytest.raises(wg.WgridError):
        wg.wgrid.fft2d(b, impl=2)           # factor 13
    c = torch.zeros((1, 8, 25856), dtype=torch.complex128, device="cuda")
    with pytest.raises(wg.WgridError):
        wg.wgrid.fft2d(c, impl=2)           # beyond 4 x 6400
