"""Offline weight design for the sparse aperture (CPU): the FPP-SCA robust sparse array synthesis of
Sec. III (Algorithm 1) and the second-order cone solver it needs.  Its output (per-row offsets and
weights) feeds the imaging entry points unchanged."""

from . import fpp_sca, socp  # noqa: F401
