"""Seeded synthetic image pairs for CFOG matching.

These generators stand in for the multimodal image pairs of the paper
(Table I, Table IV), which are not available.  They produce the reference
image A, the sensed image B and the ground-truth displacement field.  They
contain none of the matching method's arithmetic (no gradients, no CFOG,
no SSD): only texture synthesis, intensity remapping, speckle and warping.
Both the oracle and the CUDA path take their inputs from here.
"""
from .pairs import (  # noqa: F401
    Pair,
    make_pair,
    rect_texture,
    tiny_pair,
    batched_pair,
    precision_pair,
    serving_jobs,
    large_scene_pair,
    random_cp_params,
    job_pair,
)
from .cpsets import RESULT_DTYPE, cp_set  # noqa: F401
