"""The benchmark's roofline accounting (host arithmetic, no GPU): the double-float FFT's radix
plan and FP32 instruction count, its algorithmic bytes in the pruned form, and the (de)gridding
flop count per visibility.  The roofline fractions the benchmark reports rest on these."""
import bench


def test_df64_radix_plan_matches_the_library_rule():
    # powers of two as radix 8 and 4 (2 only for n = 2 * odd), then 5, 3, 7, 11
    assert bench.df64_radices(3456) == [8, 4, 4, 3, 3, 3]
    assert bench.df64_radices(2048) == [8, 8, 8, 4]
    assert bench.df64_radices(2 * 27) == [2, 3, 3, 3]


def test_df64_line_ops_per_element():
    # 456 FP32 instructions per element of a 3456-point transform on one CTA (radix-8 butterfly
    # 600, radix 4 176, radix 3 160, 38 per non-trivial twiddle product)
    assert bench.df64_part_ops(3456) == 456 * 3456
    # the symmetric odd radices: (R - 1) + P complex adds (22 each), then per output pair 4 P
    # fused multiply-adds (15) and 2 complex adds, P = (R - 1) / 2
    for r, p in ((7, 3), (11, 5)):
        assert bench.DF64_BUTTERFLY[r] == 22 * (r - 1 + p) + p * (4 * p * 15 + 44)
    # a single radix-8 stage has no twiddles: one butterfly per 8 elements
    assert bench.df64_part_ops(8) == 600
    assert bench.df64_line_ops(8) == 600
    # a 3456-point line runs as two 1728-point halves (radices 8, 8, 3, 3, 3: 419.25 per element)
    # after one radix-2 decimation step (butterfly 44 and one twiddle product per pair)
    assert bench.df64_part_ops(1728) == 724464
    assert bench.df64_line_ops(3456) == 1728 * (44 + 38) + 2 * 724464
    # 13824: four 3456-point parts after a radix-4 decimation step (butterfly 176 and three
    # twiddle products per group of four)
    assert bench.df64_line_ops(13824) == 3456 * (176 + 3 * 38) + 4 * 456 * 3456


def test_df64_line_split_rule():
    # two halves above 2048 points when the half needs only the radices 8, 4, 5, 3
    assert bench.df64_line_split(3456) == 2 and bench.df64_line_split(4096) == 2
    assert bench.df64_line_split(6400) == 2
    assert bench.df64_line_split(2048) == 1           # not above 2048
    assert bench.df64_line_split(2816) == 1           # half 1408 = 2^7 x 11: generic radix 11
    assert bench.df64_line_split(3360) == 1           # half 1680 has a factor 7
    # longer lines: 2 or 4 CTAs of at most 6400 points
    assert bench.df64_line_split(6912) == 2 and bench.df64_line_split(12800) == 2
    assert bench.df64_line_split(13824) == 4 and bench.df64_line_split(25600) == 4


def test_df64_fft_bytes_pruned_and_full():
    nx = ny = 2048
    nu = nv = 3456
    # full transform: one 16-byte read and one write per cell and pass
    assert bench.df64_fft_bytes(nu, nv, nu, nv, "degrid") == 2 * 32 * nu * nv
    assert bench.df64_fft_bytes(nu, nv, nu, nv, "grid") == 2 * 32 * nu * nv
    # pruned: both directions move the same bytes (loads pruned forward, stores pruned inverse)
    d = bench.df64_fft_bytes(nx, ny, nu, nv, "degrid")
    assert d == bench.df64_fft_bytes(nx, ny, nu, nv, "grid")
    assert d == 16 * (nx * ny + nu * ny) + 16 * (nu * ny + nu * nv)
    assert d < 2 * 32 * nu * nv


def test_gridding_flops_per_visibility():
    # alpha^3 complex-by-real multiply-adds (4 flops) plus 3 alpha Horner evaluations of degree
    # alpha + 3 (2 flops per step)
    for a in (4, 8, 15, 16):
        assert bench.algorithmic_flops_per_vis(a) == 4 * a ** 3 + 6 * a * (a + 3)


def test_stratified_pixel_sample():
    """The stratified image-error estimate: the edge stratum first, then the interior; with every
    pixel of both strata in the sample it is exactly the image's relative L2 error."""
    import numpy as np
    nx, ny, band = 40, 24, 5
    psel, nb, share = bench.stratified_pixels(nx, ny, seed=3, band=band, nb=50, ni=30)
    jx, jy = psel // ny, psel % ny
    edge = np.minimum(np.minimum(jx, nx - 1 - jx), np.minimum(jy, ny - 1 - jy))
    assert len(psel) == 80 and nb == 50 and len(set(psel.tolist())) == 80
    assert (edge[:nb] < band).all() and (edge[nb:] >= band).all()
    n_band = nx * ny - (nx - 2 * band) * (ny - 2 * band)
    assert share == n_band / (nx * ny)
    # every pixel sampled: the estimate is the plain relative L2 over the image
    all_idx, nb_all, share_all = bench.stratified_pixels(nx, ny, seed=0, band=band, nb=10 ** 6, ni=10 ** 6)
    assert nb_all == n_band and len(all_idx) == nx * ny
    rng = np.random.default_rng(1)
    ref = rng.standard_normal(nx * ny)
    x = ref + 1e-3 * rng.standard_normal(nx * ny) * (1 + 9 * (np.arange(nx * ny) % 7 == 0))
    est = bench.stratified_rel_l2(x[all_idx], ref[all_idx], nb_all, share_all)
    assert abs(est - np.linalg.norm(x - ref) / np.linalg.norm(ref)) < 1e-12 * est
