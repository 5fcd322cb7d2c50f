"""Seeded synthetic stereo scenes (inputs only).

This package renders piecewise-smooth scenes through a rectified pinhole
stereo pair and returns the left-view disparity map together with the
generator's ground truth (surface normals, primitive ids).  It holds none of
the estimator's arithmetic: the normals it returns come from the analytic
primitives, never from disparities.  Both the CUDA path's tests and the CPU
oracle's tests draw their inputs from here.
"""
from .generator import (  # noqa: F401
    Camera,
    Scene,
    CONFIGS,
    make_scene,
    config_scene,
    plane_disparity,
)
