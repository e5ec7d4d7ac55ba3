"""GB300-native ROSAR imaging by sparse-aperture azimuth filtering (arXiv 2309.08038).

The compute path is librosar.so (hand-written CUDA for sm_103a, C ABI declared in
include/rosar.h); this package is its thin Python binding.  Build it with
``python -m paper_2309_08038_gb300.build``.
"""

from ._lib import LIB_PATH, RosarError, load  # noqa: F401
from .ops import (Radar, azimuth_fft_supported, azimuth_plan, bpa, image, image_fft, image_noalloc,  # noqa: F401
                  range_compress, sparse_azimuth, sparse_azimuth_fft)
from .ops import azimuth_weight_grad_fft, bpa_time, image_fft_host, sas_time, sparse_azimuth_fft_scans  # noqa: F401
from .ops import image_fft_scans, image_fft_scans_pipelined, image_l2_loss, image_l2_loss_grad  # noqa: F401
from .ops import (image_migrating, phase_apply, phase_grad, range_compress_adjoint,  # noqa: F401
                  sparse_azimuth_adjoint, sparse_azimuth_migrating, sparse_azimuth_scans)
from .ops import (MigratingPlan, azimuth_plan_migrating, image_migrating_fft,  # noqa: F401
                  sparse_azimuth_migrating_fft)
from .ops import (azimuth_weight_grad_fft_phase, azimuth_weight_grad_spectra, phase_grad_phasor,  # noqa: F401
                  phasors, sparse_azimuth_fft_scans_ex)
from .ops import TimeDomainPlan, bpa_time_plan, bpa_time_planned, sas_time_plan, sas_time_planned  # noqa: F401
from .batch import Batch, Tuning  # noqa: F401
from . import autograd, autotune  # noqa: F401

__version__ = "0.1.0"
