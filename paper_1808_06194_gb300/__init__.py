"""GB300 (sm_103a) CFOG matching: CFOG and pixel-wise HOG extraction, block-based Harris CPs,
FFT SSD template matching with sub-pixel refinement, an FP64 affine fit and
iterative outlier rejection with a polynomial model (Ye et al., arXiv
1808.06194).  The kernels live in libcfog.so (csrc/); this
package is its thin Python binding."""
from . import _lib  # noqa: F401
from ._lib import CfogError, lib  # noqa: F401
from .api import (  # noqa: F401
    Features,
    alloc_features,
    cfog_detect_cps,
    cfog_extract,
    cfog_extract_fhog,
    cfog_extract_rows,
    cfog_fit_affine,
    cfog_match,
    cfog_match_batched,
    job_table,
    match_workspace,
    cfog_plan_info,
    cfog_reject_outliers,
    cfog_tin_rectify,
    tin_delaunay,
    tin_workspace,
    reject_workspace,
    unpack_models,
    default_params,
    feature_layout,
    params,
    resolve_variant,
    unpack_results,
)
