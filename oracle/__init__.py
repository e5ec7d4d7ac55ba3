"""FP64 CPU oracle for ROSAR sparse-aperture imaging (arXiv 2309.08038).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import anything from
this package.  The CUDA library and its Python binding never import it, and it
imports neither of them: the two share no code.

Everything here is a plain, slow, obviously-correct restatement of the paper's
definitions in complex FP64 (numpy), with each function citing the section and
equation it follows.  Pins that tie it to something other than itself live in
``tests/test_oracle_*.py``.

Parity status per function (see the module docstrings):
  geometry, signal model, range compression, sparse azimuth filter, BPA,
  default weights, adjoints: pinned.
  image metrics (entropy, PISR): pinned by hand-computed cases only; the paper's
  printed values need its measured data and are not reproducible here.
"""

from .rosar_oracle import *  # noqa: F401,F403
