"""rosar_image_noalloc against rosar_image, through the C ABI (GPU).

The no-allocation variant serves callers that own only their input and output
device buffers and may not allocate scratch (e.g. a plugin handed buffers by a
host framework, or a real-time loop that must not call cudaMalloc after start-up).
It must produce the same image as rosar_image, call after call, even though
every call reuses the same library-owned scratch array.  This file is named to be
collected last.
"""

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL_IMAGE = 1e-4     # the relative-L2 bar of the parity tests


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def rosar():
    from paper_2309_08038_gb300 import build
    build.build()
    import paper_2309_08038_gb300 as r
    return r


def test_noalloc_matches_image_on_consecutive_calls(rosar):
    import torch
    cfg = synth.TINY
    sc = synth.make_scene(cfg)
    o = torch.from_numpy(synth.draw_offsets(cfg)).cuda()
    w = torch.from_numpy(synth.default_weights(cfg, synth.draw_offsets(cfg))).cuda()
    win = torch.from_numpy(synth.hann_window(cfg.L)).cuda()
    rng = np.random.default_rng(21)
    second = (rng.standard_normal(sc.raw.shape) + 1j * rng.standard_normal(sc.raw.shape)).astype(np.complex64)
    for raw_np in (sc.raw, second):                       # two calls in a row share the scratch array
        raw = torch.from_numpy(raw_np).cuda()
        ref = rosar.image(raw, win, w, o).cpu().numpy().astype(np.complex128)
        got = rosar.image_noalloc(raw, win, w, o).cpu().numpy().astype(np.complex128)
        assert _rel(got, ref) <= TOL_IMAGE
        oracle = O.sparse_azimuth(O.range_compress(raw_np, synth.hann_window(cfg.L)), w.cpu().numpy(),
                                  o.cpu().numpy())
        assert _rel(got, oracle) <= TOL_IMAGE


def test_noalloc_indoor_size_and_limit(rosar):
    import torch
    from paper_2309_08038_gb300 import _lib
    cfg = synth.INDOOR                                    # 256 x 3600 = 921600 elements, inside the limit
    rng = np.random.default_rng(22)
    raw = torch.from_numpy((rng.standard_normal((cfg.n_az, cfg.L)) +
                            1j * rng.standard_normal((cfg.n_az, cfg.L))).astype(np.complex64)).cuda()
    o_np = synth.draw_offsets(cfg)
    o = torch.from_numpy(o_np).cuda()
    w = torch.from_numpy(synth.default_weights(cfg, o_np)).cuda()
    win = torch.from_numpy(synth.hann_window(cfg.L)).cuda()
    for _ in range(2):
        ref = rosar.image(raw, win, w, o).cpu().numpy().astype(np.complex128)
        got = rosar.image_noalloc(raw, win, w, o).cpu().numpy().astype(np.complex128)
        assert _rel(got, ref) <= TOL_IMAGE
    # beyond the built-in scratch: refused on the host before any launch
    n_az = _lib.NOALLOC_MAX_ELEMS // 1024 + 8
    big = torch.zeros((n_az, 1024), dtype=torch.complex64, device="cuda")
    wb = torch.zeros((1024, 4), dtype=torch.complex64, device="cuda")
    ob = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(rosar.RosarError, match="UNSUPPORTED"):
        rosar.image_noalloc(big, None, wb, ob)
