"""GB300 spline x-ray projector.

The x-ray transform of an image written as a sum of shifted tensor-product
B-splines (degree 0-3) over any list of lines, and its exact adjoint
(arXiv 2503.20907).  The work runs in hand-written sm_103a CUDA kernels behind
the C ABI of include/spline_project.h; this package is a thin ctypes binding
(`_lib`) plus the differentiable operator built on it.
"""
from ._lib import (BASIS_BOX3, BASIS_BSPLINE, Batch, Grid, Lines, Plan, SplineError, fp32_peak, load,
                   sp_release_workspace, sp_version,
                   spline_footprint_eval, spline_lines_expand, spline_project_adj,
                   spline_project_fwd, spline_visited)
from .autograd import backproject, project

__all__ = ["BASIS_BOX3", "BASIS_BSPLINE", "Batch", "Grid", "Lines", "Plan", "SplineError", "backproject", "fp32_peak",
           "load", "project",
           "sp_release_workspace", "sp_version",
           "spline_footprint_eval", "spline_lines_expand", "spline_project_adj",
           "spline_project_fwd", "spline_visited"]
