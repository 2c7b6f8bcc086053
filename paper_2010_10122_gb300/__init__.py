"""GB300-native w-gridding: the wide-field radio-interferometric response operator of
Arras et al. (degrid = R, grid = R^dagger) as hand-written sm_103a CUDA behind a C ABI
(include/wgrid.h, libwgrid.so), with a thin Python binding, an autograd Function and a
continuous-batching server on top."""
from .wgrid import (Plan, WgridError, dirty2ms, ms2dirty, kernel_table, kernel_phi,  # noqa: F401
                    kernel_poly, kernel_psi, kernel_design_table, kernel_eps, kernel_search,
                    plan_params, fft_time, fma_peak, version, wait, lib)
