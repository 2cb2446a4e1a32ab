"""B300-native scalar-diffraction simulation of diffractive optical elements (DOEs).

Implements the forward model of Wei et al., "Large-Area Fabrication-Aware Computational
Diffractive Optics" (ACM TOG 2025), Sec. 3.1, Eq. 1-4: height map -> transmittance ->
band-limited angular-spectrum propagation -> PSF per wavelength, its adjoint (height-map
gradient), and PSF convolution of images.  All arithmetic runs in the hand-written CUDA
kernels of libdoe.so (C ABI in include/doe.h); this package marshals PyTorch tensors.
"""
from .api import (  # noqa: F401
    PSF,
    Geometry,
    band_limits,
    debug_band_mask,
    grad,
    init,
    propagate,
    psf,
    psf_autograd,
    psf_many,
    launch_count,
    render,
    trace_enable,
    trace_read,
    workspace,
    workspace_bytes,
)
from ._lib import DoeError  # noqa: F401
