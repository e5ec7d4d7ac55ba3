"""Range-migration-aware taps (Eq. (43) with per-pulse peak bins, Eq. (40)) against the FP64 oracle (GPU)."""

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rosar():
    from paper_2309_08038_gb300 import build
    build.build()
    import paper_2309_08038_gb300 as r
    return r


def _c(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", ["two_rows", "edges", "wide_spread", "wide_span", "ragged"])
def test_migrating_filter_matches_oracle(rosar, case):
    import torch
    rng = np.random.default_rng(abs(hash(case)) % 2 ** 32)
    n_bins, n_rng, n_az, K, M = 12, 10, 1031, 40, 300
    if case == "wide_span":
        n_az, M = 9000, 8000                   # span beyond the staged window: direct gathers
    if case == "ragged":
        n_az = 37
        K, M = 7, 30
    o = (np.sort(rng.choice(M, K, replace=False)) - M // 2).astype(np.int32)
    if case in ("two_rows", "wide_span", "ragged"):
        dl = rng.integers(0, 2, (n_rng, K)).astype(np.int32)
    elif case == "edges":
        dl = rng.integers(-3, 4, (n_rng, K)).astype(np.int32)      # rows below 0 / above n_bins read zero
    else:
        dl = rng.integers(-6, 7, (n_rng, K)).astype(np.int32)      # more rows than a tile stages
    S, w = _c(rng, n_bins, n_az), _c(rng, n_rng, K)
    got = rosar.sparse_azimuth_migrating(torch.from_numpy(S).cuda(), torch.from_numpy(w).cuda(),
                                         torch.from_numpy(o).cuda(), torch.from_numpy(dl).cuda()).cpu().numpy()
    assert _rel(got, O.sparse_azimuth_migrating(S, w, o, dl)) < 2e-6, case


def test_zero_offsets_equal_fixed_row_bit_exact(rosar):
    import torch
    rng = np.random.default_rng(3)
    S, w = _c(rng, 16, 3600), _c(rng, 16, 64)
    o = torch.from_numpy((np.sort(rng.choice(600, 64, replace=False)) - 300).astype(np.int32)).cuda()
    a = rosar.sparse_azimuth(torch.from_numpy(S).cuda(), torch.from_numpy(w).cuda(), o)
    b = rosar.sparse_azimuth_migrating(torch.from_numpy(S).cuda(), torch.from_numpy(w).cuda(), o,
                                       torch.zeros((16, 64), dtype=torch.int32, device="cuda"))
    assert torch.equal(a, b)


@pytest.mark.parametrize("name", ["tiny", "indoor"])
def test_image_migrating_matches_oracle_chain(rosar, name):
    import torch
    cfg = synth.CONFIGS[name]
    sc = synth.make_scene(cfg)
    o = synth.draw_offsets(cfg)
    w = synth.default_weights(cfg, o)
    dl = synth.migration_offsets(cfg, o)
    win = synth.hann_window(cfg.L)
    got = rosar.image_migrating(*(torch.from_numpy(x).cuda() for x in (sc.raw, win, w, o, dl))).cpu().numpy()
    ref = O.sparse_azimuth_migrating(O.range_compress(sc.raw, win), w, o, dl)
    assert _rel(got, ref) < 1e-4
    a = np.abs(ref) ** 2
    p = np.unravel_index(np.argmax(a), a.shape)
    assert np.unravel_index(np.argmax(np.abs(got)), got.shape) == p
