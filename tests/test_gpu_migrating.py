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


# ------------------------------------------- the migrating filter in the frequency domain --

TOL_FFT_FILTER = 5e-6     # as the fixed-row FFT filter: float32 transforms of length n_az


@pytest.mark.parametrize("n_az,per_row,dl_range,n_bins,n_rng", [
    (3600, False, (0, 2), 12, 10),      # compile-time plan, offsets 0 / 1
    (1800, True, (-1, 2), 9, 9),        # compile-time plan, per-row offsets, a row below 0
    (7200, False, (-3, 4), 8, 7),       # compile-time plan (512 threads), rows outside 0 .. n_bins-1 read zero
    (360, False, (0, 1), 5, 5),         # compile-time plan, one plane: the fixed-row filter
    (1000, True, (-2, 3), 11, 6),       # run-time plan (power-of-two factors and 5^3)
    (48, False, (0, 2), 4, 4),          # short row, run-time plan
    (4096, False, (1, 3), 7, 7),        # power of two (padded layout), no tap reads its own row
])
def test_migrating_fft_matches_oracle(rosar, n_az, per_row, dl_range, n_bins, n_rng):
    """rosar_azimuth_plan_migrating + rosar_sparse_azimuth_migrating_fft against the oracle's migrating filter
    (Eq. (43) with per-tap rows): planes per row offset, wrapping offsets, rows outside read zero."""
    import torch
    rng = np.random.default_rng(n_az + n_bins)
    K = min(24, n_az)
    M = min(n_az, 600)
    if per_row:
        o = np.stack([np.sort(rng.choice(M, K, replace=False)) - M // 2 for _ in range(n_rng)]).astype(np.int32)
        o[0, 0] -= 2 * n_az
    else:
        o = (np.sort(rng.choice(M, K, replace=False)) - M // 2).astype(np.int32)
    dl = rng.integers(dl_range[0], dl_range[1], (n_rng, K)).astype(np.int32)
    S, w = _c(rng, n_bins, n_az), _c(rng, n_rng, K)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    plan = rosar.azimuth_plan_migrating(t(w), t(o), t(dl), n_az)
    assert plan.n_d == int(dl.max() - dl.min() + 1)
    got = rosar.sparse_azimuth_migrating_fft(t(S), plan).cpu().numpy()
    ref = O.sparse_azimuth_migrating(S, w, o, dl)
    assert _rel(got, ref) < TOL_FFT_FILTER, (n_az, per_row, dl_range)
    gather = rosar.sparse_azimuth_migrating(t(S), t(w), t(o), t(dl), n_rng=n_rng).cpu().numpy()
    assert _rel(got, gather) < TOL_FFT_FILTER


def test_migrating_fft_one_plane_equals_fixed_row_fft(rosar):
    """dl = 0 everywhere: one plane, the same plan and sums as rosar_sparse_azimuth_fft (bit for bit)."""
    import torch
    rng = np.random.default_rng(11)
    S, w = _c(rng, 16, 3600), _c(rng, 16, 64)
    o = torch.from_numpy((np.sort(rng.choice(600, 64, replace=False)) - 300).astype(np.int32)).cuda()
    Sd, wd = torch.from_numpy(S).cuda(), torch.from_numpy(w).cuda()
    plan = rosar.azimuth_plan_migrating(wd, o, torch.zeros((16, 64), dtype=torch.int32, device="cuda"), 3600)
    H = rosar.azimuth_plan(wd, o, 3600)
    assert torch.equal(plan.H[0], H)
    a = rosar.sparse_azimuth_fft(Sd, H)
    b = rosar.sparse_azimuth_migrating_fft(Sd, plan)
    assert _rel(b.cpu().numpy(), a.cpu().numpy()) < 1e-6


@pytest.mark.parametrize("name", ["tiny", "indoor"])
def test_image_migrating_fft_matches_oracle_chain(rosar, name):
    """The paper's FFT+SAS with per-pulse peak bins (l*_n of Eq. (40) in Eq. (43)) through the frequency-domain
    filter, in the launch configuration the benchmark times, against the oracle chain; peak position exact."""
    import torch
    cfg = synth.CONFIGS[name]
    sc = synth.make_scene(cfg)
    o = synth.draw_offsets(cfg)
    w = synth.default_weights(cfg, o)
    dl = synth.migration_offsets(cfg, o)
    win = synth.hann_window(cfg.L)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    plan = rosar.azimuth_plan_migrating(t(w), t(o), t(dl), cfg.n_az)
    got = rosar.image_migrating_fft(t(sc.raw), t(win), plan).cpu().numpy()
    ref = O.sparse_azimuth_migrating(O.range_compress(sc.raw, win), w, o, dl)
    assert _rel(got, ref) < 1e-4
    a = np.abs(ref) ** 2
    assert np.unravel_index(np.argmax(np.abs(got)), got.shape) == np.unravel_index(np.argmax(a), a.shape)


def test_migrating_fft_refuses_bad_arguments(rosar):
    import torch
    S = torch.zeros((4, 1031), dtype=torch.complex64, device="cuda")      # 1031 is prime: no FFT plan
    w = torch.zeros((4, 3), dtype=torch.complex64, device="cuda")
    o = torch.zeros(3, dtype=torch.int32, device="cuda")
    dl = torch.zeros((4, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(rosar.RosarError, match="UNSUPPORTED"):
        rosar.azimuth_plan_migrating(w, o, dl, 1031)
    plan = rosar.MigratingPlan(torch.zeros((1, 4, 1031), dtype=torch.complex64, device="cuda"), 0, 1)
    with pytest.raises(rosar.RosarError, match="UNSUPPORTED"):
        rosar.sparse_azimuth_migrating_fft(S, plan)
    dl[0, 0] = 40                                                          # 41 planes: more than 16
    with pytest.raises(rosar.RosarError, match="INVALID"):
        rosar.azimuth_plan_migrating(w, o, dl, 3600)
