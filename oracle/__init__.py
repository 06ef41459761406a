"""FP64 CPU oracle for CFOG matching (arXiv 1808.06194).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA path.  See ``cfog_oracle.c`` for the step-by-step
definitions and the paper passages they follow.

Pins (tests/test_oracle_*.py, run without a GPU):
  * gradients, Z smoothing and the spatial Gaussian against scipy.ndimage
    routines with the same taps and border rule;
  * CFOG invariants: D >= 0, unit L2 norm, constant image -> 0, invariance to
    a*I + b (including a < 0), the horizontal-flip channel permutation, the
    transpose permutation for even m, and the closed form on a linear ramp;
  * brute-force SSD against an independent numpy FFT correlation (Eq. 5, 8, 9);
  * exact recovery of a known integer shift with S(v*) = 0;
  * the quadratic sub-pixel fit on exactly quadratic surfaces;
  * Harris against a scipy.ndimage statement and a single-corner image;
  * affine least squares against numpy.linalg.lstsq and exact data;
  * pixel-wise HOG (Sec. III-C): a separable triangular-kernel statement of
    the trilinear interpolation, the ramp closed form, invariances and the
    flip permutation of cells and bins;
  * TIN rectification (Sec. IV): identity maps, exact resampling of a linear
    image under a global affine map, the hull against scipy's Delaunay point
    location, and agreement of neighbouring triangles on shared edges;
  * outlier rejection (Sec. IV): exact polynomial data, a step-by-step replay
    of every removal with numpy.linalg.lstsq in another basis, the stop rule,
    planted outliers, the min_keep floor, degenerate sets, translation
    invariance, and agreement of the degree-1 model with affine LS.
"""
from .oracle import (  # noqa: F401
    build,
    lib,
    gradients,
    channels,
    channels_binned,
    gauss_taps,
    smooth_xy,
    smooth_z,
    normalize,
    cfog,
    fhog,
    tin_rectify,
    ssd_surface,
    subpixel,
    match_one,
    match_many,
    harris,
    detect,
    cell_chip,
    affine_ls,
    poly_terms,
    reject_outliers,
    poly_predict,
    DEFAULTS,
)
