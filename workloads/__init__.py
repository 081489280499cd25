"""Seeded synthetic inputs for the adaptive-heightfield renderer.

This package only *generates inputs*: fBm terrain, quadtree leaf layouts and
camera poses.  It contains none of the method's arithmetic (no RBF weights,
no cascade fitting, no mip reduction, no ray casting), so both the CUDA
library and the CPU oracle can draw their inputs from it without sharing any
part of the computation they are compared on.

The inputs stand in for the paper's DEM / flood-simulation scenarios
(Section 6, Table 1), whose data are not available: terrain is fractional
Brownian motion with Hurst exponent 0.8, and quadtrees are refined either at
random or where the terrain's curvature is high, with cell sizes spanning
several levels as in Table 1.
"""

from .fbm import FBm
from .quadtree import Quadtree, random_split_quadtree, curvature_quadtree
from .cameras import Camera, fixed_camera, flight_path
from .configs import (tiny_config, dem_config, precision_config, batch_config, serve_config,
                      tiny_flood_config, flood_config, flood_depths, Request)

__all__ = [
    "FBm", "Quadtree", "random_split_quadtree", "curvature_quadtree",
    "Camera", "fixed_camera", "flight_path",
    "tiny_config", "dem_config", "precision_config", "batch_config", "serve_config", "Request",
    "tiny_flood_config", "flood_config", "flood_depths",
]
