"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

Bar (per image, complex64 result vs FP64 oracle): relative L2 <= 1e-4; point-target
peak indices identical.  Integer-exact properties (identity, circular shift) are
checked bit for bit.  Sizes span several tiles and a ragged tail; the full-size
workloads are checked on sampled rows the oracle computes one by one.
"""

import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL_IMAGE = 1e-4     # relative L2 per image
TOL_FFT = 2e-6       # range compression alone: float32 FFT error ~ 1e-7 * log2(L)
TOL_MAC = 2e-6       # azimuth filter alone: float32 sums of <= a few hundred taps


@pytest.fixture(scope="module")
def rosar():
    from paper_2309_08038_gb300 import build
    build.build()
    import paper_2309_08038_gb300 as r
    return r


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def dev(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.cpu().numpy().astype(np.complex128)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def crand(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def oracle_radar(cfg):
    r = cfg.radar
    return O.Radar(fc=r.fc, slope=r.slope, t_s=r.t_sample(cfg.L), t_start=r.t_start, r0=r.r0, c=r.c)


def api_radar(rosar, cfg):
    r = cfg.radar
    return rosar.Radar(r.fc, r.slope, r.t_sample(cfg.L), r.t_start, r.r0, r.c)


_SCENES = {}


def scene(name):
    if name not in _SCENES:
        _SCENES[name] = synth.make_scene(synth.CONFIGS[name])
    return _SCENES[name]


# --------------------------------------------------------- range compression --

@pytest.mark.parametrize("L", [8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("n_az", [37, 64])
def test_range_compress_every_length(rosar, torch, L, n_az):
    rng = np.random.default_rng(L + n_az)
    raw = crand(rng, n_az, L)
    win = synth.hann_window(L)
    for centred in (True, False):
        got = host(rosar.range_compress(dev(torch, raw), dev(torch, win), centred=centred))
        ref = O.range_compress(raw, win, centred=centred)
        assert got.shape == (L, n_az)
        assert rel_l2(got, ref) < TOL_FFT, (L, n_az, centred)


def test_range_compress_rectangular_window_and_scene(rosar, torch):
    sc = scene("tiny")
    got = host(rosar.range_compress(dev(torch, sc.raw), None))
    assert rel_l2(got, O.range_compress(sc.raw, None)) < TOL_FFT


# ------------------------------------------------------ sparse azimuth filter --

def _offsets_case(kind, rng):
    if kind == "tiny":
        cfg = synth.TINY
        return cfg.L, cfg.n_az, synth.draw_offsets(cfg)
    if kind == "many_taps_ragged":                 # K > one staged chunk, n_az not a tile multiple
        return 8, 1031, (np.sort(rng.choice(800, 300, replace=False)) - 400).astype(np.int32)
    if kind == "wide_span":                        # span > staged window: direct-gather path
        return 4, 9000, np.sort(rng.choice(np.arange(-4400, 4400), 20, replace=False)).astype(np.int32)
    if kind == "wild_ints":                        # any int32 is valid: non-negative modulo
        return 5, 100, np.array([123456789, -987654321, 0, 99, -1, 2 ** 31 - 1, -2 ** 31], dtype=np.int32)
    if kind == "per_row":
        o = np.stack([np.sort(rng.choice(600, 64, replace=False)) - 300 for _ in range(16)]).astype(np.int32)
        return 16, 3600, o
    if kind == "short_row":                        # n_az smaller than the offsets' span
        return 3, 40, np.array([-30, -7, 0, 5, 33], dtype=np.int32)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["tiny", "many_taps_ragged", "wide_span", "wild_ints", "per_row", "short_row"])
def test_sparse_azimuth_matches_oracle(rosar, torch, kind):
    rng = np.random.default_rng(abs(hash(kind)) % 2 ** 32)
    n_rng, n_az, o = _offsets_case(kind, rng)
    K = o.shape[-1]
    S = crand(rng, n_rng, n_az)
    w = crand(rng, n_rng, K)
    got = host(rosar.sparse_azimuth(dev(torch, S), dev(torch, w), dev(torch, o)))
    ref = O.sparse_azimuth(S, w, o.astype(np.int64))
    assert rel_l2(got, ref) < TOL_MAC, kind


def test_sparse_azimuth_identity_is_bit_exact(rosar, torch):
    rng = np.random.default_rng(5)
    S = crand(rng, 7, 2100)
    got = rosar.sparse_azimuth(dev(torch, S), dev(torch, np.ones((7, 1), np.complex64)),
                               dev(torch, np.zeros(1, np.int32)))
    assert np.array_equal(got.cpu().numpy(), S)


def test_circular_shift_is_bit_exact(rosar, torch):
    """T6: rolling the pulses by s rolls the image by s, bit for bit (fixed tap order)."""
    cfg = synth.TINY
    sc = scene("tiny")
    o = synth.draw_offsets(cfg)
    w = dev(torch, synth.default_weights(cfg, o))
    win = dev(torch, synth.hann_window(cfg.L))
    base = rosar.image(dev(torch, sc.raw), win, w, dev(torch, o)).cpu().numpy()
    for s in (1, 77, 359):
        rolled = rosar.image(dev(torch, np.roll(sc.raw, s, axis=0)), win, w, dev(torch, o)).cpu().numpy()
        assert np.array_equal(rolled, np.roll(base, s, axis=1)), s


# ------------------------------------------------------------- whole image --

def _peaks_with_margin(img, count):
    """Up to `count` local peaks of |img|^2, strongest first, each unique by the 1e-3 margin."""
    a = np.abs(img) ** 2
    peaks = []
    b = a.copy()
    for _ in range(count):
        idx = np.unravel_index(np.argmax(b), b.shape)
        r, t = idx
        nb = b.copy()
        nb[max(r - 1, 0):r + 2][:, [(t + j) % a.shape[1] for j in (-1, 0, 1)]] = 0
        if nb.max() < (1 - 1e-3) * b[idx]:
            peaks.append((int(r), int(t)))
        b[max(r - 3, 0):r + 4][:, [(t + j) % a.shape[1] for j in range(-6, 7)]] = 0
    return peaks


@pytest.mark.parametrize("name", ["tiny", "indoor"])
def test_image_matches_oracle_chain(rosar, torch, name):
    cfg = synth.CONFIGS[name]
    sc = scene(name)
    o = synth.draw_offsets(cfg)
    w = synth.default_weights(cfg, o)
    win = synth.hann_window(cfg.L)
    got = host(rosar.image(dev(torch, sc.raw), dev(torch, win), dev(torch, w), dev(torch, o)))
    ref = O.sparse_azimuth(O.range_compress(sc.raw, win), w, o)
    assert rel_l2(got, ref) < TOL_IMAGE
    pk_ref = _peaks_with_margin(ref, 3)
    assert pk_ref, "no unambiguous peak in the reference image"
    for p in pk_ref:
        a = np.abs(got) ** 2
        r, t = p
        win3 = a[max(r - 1, 0):r + 2][:, [(t + j) % a.shape[1] for j in (-1, 0, 1)]]
        assert a[p] == win3.max(), p


def test_image_equals_the_two_calls(rosar, torch):
    cfg = synth.TINY
    sc = scene("tiny")
    o = dev(torch, synth.draw_offsets(cfg))
    w = dev(torch, synth.default_weights(cfg, synth.draw_offsets(cfg)))
    win = dev(torch, synth.hann_window(cfg.L))
    raw = dev(torch, sc.raw)
    a = rosar.image(raw, win, w, o).cpu().numpy()
    b = rosar.sparse_azimuth(rosar.range_compress(raw, win), w, o).cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("pix", [(20, 90), (35, 200), (12, 359), (50, 0)])
def test_point_target_peak_is_bit_exact(rosar, torch, pix):
    """A noise-free target at the centre of pixel (r*, theta*) peaks there on the GPU and in the oracle."""
    cfg = synth.TINY
    rad = cfg.radar
    dR = rad.bin_spacing(cfg.L)
    r_s, t_s = pix
    raw = synth.synth_if(cfg, [rad.r0 + r_s * dR], [2 * math.pi * t_s / cfg.n_az], [1.0]).astype(np.complex64)
    o = synth.draw_offsets(cfg)
    w = synth.default_weights(cfg, o)
    win = synth.hann_window(cfg.L)
    got = host(rosar.image(dev(torch, raw), dev(torch, win), dev(torch, w), dev(torch, o)))
    ref = O.sparse_azimuth(O.range_compress(raw, win), w, o)
    assert _peaks_with_margin(ref, 1) == [pix]
    assert np.unravel_index(np.argmax(np.abs(got)), got.shape) == pix
    assert rel_l2(got, ref) < TOL_IMAGE


# -------------------------------------------------------------------- BPA --

def _unambiguous_rows(cfg, rows, M):
    """Rows whose nearest-bin choice is not within 1e-4 bin of a rounding tie for any tap (nominal geometry)."""
    rad = oracle_radar(cfg)
    dR = O.range_bin_spacing(rad, cfg.L)
    d = np.arange(-(M // 2), M - M // 2)
    keep = []
    for r in rows:
        x = O.slant_range(rad.r0 + r * dR, 0.0, rad.r0, O.phase_centre_angle(d, cfg.n_az)) / dR
        if np.all(np.abs(x - np.floor(x) - 0.5) > 1e-4):
            keep.append(r)
    return keep


@pytest.mark.parametrize("interp", ["linear", "nearest"])
def test_bpa_nominal_matches_oracle(rosar, torch, interp):
    cfg = synth.TINY
    sc = scene("tiny")
    win = synth.hann_window(cfg.L)
    S = O.range_compress(sc.raw, win).astype(np.complex64)
    got = host(rosar.bpa(dev(torch, S), api_radar(rosar, cfg), cfg.L, cfg.M_ap, interp=interp))
    ref = O.bpa(S, oracle_radar(cfg), cfg.L, cfg.M_ap, interp=interp)
    rows = list(range(cfg.L)) if interp == "linear" else _unambiguous_rows(cfg, range(cfg.L), cfg.M_ap)
    assert len(rows) > cfg.L // 2
    assert rel_l2(got[rows], ref[rows]) < TOL_IMAGE
    assert _peaks_with_margin(ref, 1)[0] == np.unravel_index(np.argmax(np.abs(got)), got.shape)


def test_bpa_with_pulse_errors_matches_oracle(rosar, torch):
    """Per-pixel-pulse geometry with supplied rotation errors (Eq. (37)), linear interpolation."""
    cfg = synth.INDOOR
    sc = scene("indoor")
    win = synth.hann_window(cfg.L)
    S = O.range_compress(sc.raw, win).astype(np.complex64)
    dphi = sc.dphi.astype(np.float32)
    dr = sc.dr.astype(np.float32)
    got = host(rosar.bpa(dev(torch, S), api_radar(rosar, cfg), cfg.L, cfg.M_ap, dphi=dev(torch, dphi),
                         dr=dev(torch, dr)))
    rad = oracle_radar(cfg)
    for r in (0, 1, 17, 100, 255):
        ref = O.bpa_pixels(S, rad, cfg.n_az, cfg.M_ap, np.full(cfg.n_az, r), np.arange(cfg.n_az),
                           dphi=dphi.astype(np.float64), dr=dr.astype(np.float64))
        assert rel_l2(got[r], ref) < TOL_IMAGE, r


@pytest.mark.parametrize("interp", ["linear", "nearest"])
def test_bpa_large_pulse_errors_mixed_windows(rosar, torch, interp):
    """Supplied positions several range bins off on a few pulses (Eq. (37)): the azimuth tile whose pulses include
    them (pixels 0..255 read pulses -30..285; pixels 256..359 read 226..359 and 0..180, so pulses 190..199 are
    the first tile's alone) cannot bound its bins by the staged window and reads those samples through L2, the
    other tile reads the window unchecked.  With a moderate error everywhere nearly every window is bounded (the
    first rows, where x spans most bins, are not)."""
    cfg = synth.TINY
    rng = np.random.default_rng(21)
    S = crand(rng, cfg.L, cfg.n_az)
    rad = oracle_radar(cfg)
    dR = O.range_bin_spacing(rad, cfg.L)
    for big in (True, False):
        dr = (0.3 * dR * rng.uniform(-1, 1, cfg.n_az)).astype(np.float32)
        dphi = np.deg2rad(0.2 * rng.uniform(-1, 1, cfg.n_az)).astype(np.float32)
        if big:        # pulses 190..199: 3.5 bins out and 4 degrees off
            dr[190:200] = np.float32(3.5 * dR)
            dphi[190:200] = np.float32(np.deg2rad(4.0))
        got = host(rosar.bpa(dev(torch, S), api_radar(rosar, cfg), cfg.L, cfg.M_ap, interp=interp,
                             dphi=dev(torch, dphi), dr=dev(torch, dr)))
        rows = np.arange(cfg.L)
        ref = np.stack([O.bpa_pixels(S, rad, cfg.n_az, cfg.M_ap, np.full(cfg.n_az, r), np.arange(cfg.n_az),
                                     interp=interp, dphi=dphi.astype(np.float64), dr=dr.astype(np.float64))
                        for r in rows])
        if interp == "nearest":      # rounding at a bin's midpoint may pick either bin: compare the pixels
            # whose every sample lies clear of a midpoint in the oracle's own geometry
            keep = _clear_of_midpoints(rad, cfg, dR, dphi, dr)
            assert keep.mean() > 0.3
            assert rel_l2(got[keep], ref[keep]) < TOL_IMAGE, big
        else:
            assert rel_l2(got, ref) < TOL_IMAGE, big


def _clear_of_midpoints(rad, cfg, dR, dphi, dr):
    """Pixels of the tiny grid whose every (pixel, pulse) bin position lies more than 1e-3 of a bin from a
    midpoint between bins (nearest-bin reads agree there whatever the float rounding)."""
    M = cfg.M_ap
    d = np.arange(-(M // 2), M - M // 2)
    keep = np.zeros((cfg.L, cfg.n_az), dtype=bool)
    th = np.arange(cfg.n_az)
    n = (th[:, None] + d[None, :]) % cfg.n_az
    phi_n = O.phase_centre_angle(d, cfg.n_az)[None, :] + dphi.astype(np.float64)[n]
    for r in range(cfg.L):
        x = O.slant_range(rad.r0 + r * dR, 0.0, rad.r0 + dr.astype(np.float64)[n], phi_n) / dR
        keep[r] = np.all(np.abs(x - np.floor(x) - 0.5) > 1e-3, axis=1)
    return keep


def test_bpa_row_subset_and_ragged_azimuth(rosar, torch):
    rng = np.random.default_rng(9)
    cfg = synth.TINY
    n_az, L = 301, 64
    S = crand(rng, L, n_az)
    rad = oracle_radar(cfg)
    got = host(rosar.bpa(dev(torch, S), api_radar(rosar, cfg), 20, 41))
    ref = np.stack([O.bpa_pixels(S, rad, n_az, 41, np.full(n_az, r), np.arange(n_az)) for r in range(20)])
    assert rel_l2(got, ref) < TOL_IMAGE


# ------------------------------------------------- full sizes, sampled rows --

def test_highres_full_size_sampled_rows(rosar, torch):
    """1024 x 14400, K = 128 per-row taps over M = 2400 (the high-resolution workload's launch shapes):
    the GPU image through rosar_image against the oracle on sampled rows."""
    cfg = synth.HIGHRES
    rng = np.random.default_rng(77)
    raw = crand(rng, cfg.n_az, cfg.L)
    o = synth.draw_offsets(cfg)
    w = synth.default_weights(cfg, o)
    win = synth.hann_window(cfg.L)
    got = rosar.image(dev(torch, raw), dev(torch, win), dev(torch, w), dev(torch, o))
    torch.cuda.synchronize()
    rows = [0, 1, 333, 512, 1000, 1023]
    S_rows = O.range_compress(raw, win, bins=rows)
    ref = O.sparse_azimuth(S_rows, w[rows], o[rows])
    got_rows = host(got[rows])
    for i, r in enumerate(rows):
        if not np.any(w[r]):      # row 0 without a tap facing the rotation circle: all-zero weights
            assert not np.any(got_rows[i]), r
            continue
        assert rel_l2(got_rows[i], ref[i]) < TOL_IMAGE, r
    # FFT+BPA (Sec. III-D, w_BP) on sampled pixels: the GPU chain (range compression, then BPA) against
    # the oracle chain on the same raw cube; the oracle's range bins come from its own DFT, and only the
    # bins the sampled rows' interpolation can touch are evaluated
    S = rosar.range_compress(dev(torch, raw), dev(torch, win))
    b = host(rosar.bpa(S, api_radar(rosar, cfg), cfg.L, cfg.M_ap)[[5, 700]])
    need = sorted({l for r in (5, 700) for l in range(r - 2, r + 12) if 0 <= l < cfg.L})
    Sh = np.zeros((cfg.L, cfg.n_az), dtype=np.complex128)
    Sh[need] = O.range_compress(raw, win, bins=need)
    assert rel_l2(host(S[need]), Sh[need]) < TOL_FFT
    th = np.arange(0, cfg.n_az, 97)
    for i, r in enumerate((5, 700)):
        ref_b = O.bpa_pixels(Sh, oracle_radar(cfg), cfg.n_az, cfg.M_ap, np.full(th.size, r), th)
        assert rel_l2(b[i, th], ref_b) < TOL_IMAGE, r


# ------------------------------------------------------------------ errors --

def test_errors_are_raised_before_launch(rosar, torch):
    raw = torch.zeros((10, 48), dtype=torch.complex64, device="cuda")
    with pytest.raises(rosar.RosarError, match="UNSUPPORTED"):
        rosar.range_compress(raw)
    with pytest.raises(TypeError):
        rosar.range_compress(torch.zeros((10, 64), dtype=torch.complex128, device="cuda"))
