"""Seeded synthetic inputs for ROSAR imaging: scenes, raw IF cubes, windows, offsets, weights.

Shared by the tests, the benchmark and the smoke check.  This package holds the
sensor simulation (the paper's signal model, used only to make inputs) and the
offline default-weight design; it holds none of the imaging arithmetic (range
compression, azimuth filtering, back-projection), and imports neither the CUDA
library nor the oracle.
"""

from .configs import (CONFIGS, HIGHRES, INDOOR, TINY, RadarParams, ScanConfig,  # noqa: F401
                      batched_configs, diff_configs, max_range)
from .scene import Scene, draw_offsets, draw_scene, hann_window, make_scene, synth_if  # noqa: F401
from .weights import default_weights, migration_offsets  # noqa: F401
