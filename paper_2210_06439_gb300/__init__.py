"""GB300-native batched hydro right-hand side (Octo-Tiger hydro solver,
arXiv 2210.06439): PPM reconstruction to 26 points per cell, Kurganov-Tadmor
flux with Simpson face quadrature, flux divergence, SSP-RK3 update and the
CFL time-step reduction, as sm_103a CUDA kernels behind a C ABI.

The CUDA library is loaded on first use by ``paper_2210_06439_gb300.binding``;
importing this package alone loads nothing.
"""

__all__ = ["binding", "inputs"]
