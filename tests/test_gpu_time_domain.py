"""Parity of the time-domain comparison paths (Eq. (14) BPA, Algorithm 2 SAS) with the FP64 oracle.

Bar: relative L2 <= 1e-4 per image (float32 sums of K*L terms per pixel); full-size workloads on
pixels the oracle evaluates one by one; point-target peak at the target's pixel.
"""

import numpy as np
import pytest

import oracle as O
import synth

from test_gpu_parity import api_radar, crand, dev, host, oracle_radar, rel_l2, scene  # noqa: F401
from test_gpu_parity import rosar, torch  # noqa: F401  (fixtures)

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _weights(cfg):
    o = synth.draw_offsets(cfg)
    return synth.default_weights(cfg, o), o


def _radar_pair(rosar, L):
    rad = synth.RadarParams()
    o_rad = O.Radar(fc=rad.fc, slope=rad.slope, t_s=rad.t_sample(L), t_start=rad.t_start, r0=rad.r0, c=rad.c)
    a_rad = rosar.Radar(rad.fc, rad.slope, rad.t_sample(L), rad.t_start, rad.r0, rad.c)
    return o_rad, a_rad


def test_bpa_time_tiny_full_image(rosar, torch):
    cfg = synth.TINY
    sc = scene("tiny")
    win = synth.hann_window(cfg.L)
    got = host(rosar.bpa_time(dev(torch, sc.raw), dev(torch, win), api_radar(rosar, cfg), cfg.L, cfg.M_ap))
    ref = O.bpa_time(sc.raw, win, oracle_radar(cfg), cfg.L, cfg.M_ap)
    assert rel_l2(got, ref) <= TOL


@pytest.mark.parametrize("centred", [True, False])
@pytest.mark.parametrize("use_win", [True, False])
def test_sas_time_tiny_full_image(rosar, torch, centred, use_win):
    cfg = synth.TINY
    sc = scene("tiny")
    w, o = _weights(cfg)
    win = synth.hann_window(cfg.L) if use_win else None
    got = host(rosar.sas_time(dev(torch, sc.raw), None if win is None else dev(torch, win), dev(torch, w),
                              dev(torch, o), api_radar(rosar, cfg), centred=centred))
    ref = O.sas_time(sc.raw, win, w, o, oracle_radar(cfg), cfg.L, centred=centred)
    assert rel_l2(got, ref) <= TOL


@pytest.mark.parametrize("n_az,L,n_rng,M_ap", [(200, 48, 45, 13), (129, 16, 33, 1), (97, 32, 1, 97)])
def test_bpa_time_ragged(rosar, torch, n_az, L, n_rng, M_ap):
    """Azimuth and row counts off the 128 x 32 tile, L a multiple of 16 but not a power of two, odd
    and extreme apertures (one pulse; the whole ring)."""
    o_rad, a_rad = _radar_pair(rosar, L)
    rng = np.random.default_rng(n_az + L)
    raw = crand(rng, n_az, L)
    win = rng.uniform(0.1, 1.0, L).astype(np.float32)
    got = host(rosar.bpa_time(dev(torch, raw), dev(torch, win), a_rad, n_rng, M_ap))
    ref = O.bpa_time(raw, win, o_rad, n_rng, M_ap)
    assert rel_l2(got, ref) <= TOL


@pytest.mark.parametrize("n_az,M_ap", [(4200, 4200), (3000, 2600)])
def test_bpa_time_wide_aperture(rosar, torch, n_az, M_ap):
    """Apertures of thousands of pulses: 2600 taps run as ~40 groups of sorted taps per CTA in the window
    kernel, 4200 taps exceed the taps one CTA of it holds (more than 512 per cluster rank) and take the per-tap
    kernel; sampled pixels against the oracle."""
    L, n_rng = 16, 3
    o_rad, a_rad = _radar_pair(rosar, L)
    rng = np.random.default_rng(n_az + M_ap)
    raw = crand(rng, n_az, L)
    win = rng.uniform(0.1, 1.0, L).astype(np.float32)
    got = host(rosar.bpa_time(dev(torch, raw), dev(torch, win), a_rad, n_rng, M_ap))
    rows = np.array([0, 1, 2, 1, 2, 2])
    thetas = np.array([0, 1, n_az // 2, n_az - 1, 777, 2999])
    ref = O.bpa_time_pixels(raw, win, o_rad, n_az, M_ap, rows, thetas)
    assert rel_l2(got[rows, thetas], ref) <= TOL


@pytest.mark.parametrize("per_row", [False, True])
def test_sas_time_ragged_and_wrapping_offsets(rosar, torch, per_row):
    """Offsets anywhere in int32 range (taken modulo n_az, including beyond +-n_az), ragged tiles,
    shared and per-row offset tables (the per-row path is a different kernel)."""
    n_az, L, n_rng, K = 300, 64, 45, 9
    o_rad, a_rad = _radar_pair(rosar, L)
    rng = np.random.default_rng(31)
    raw = crand(rng, n_az, L)
    win = synth.hann_window(L)
    w = crand(rng, n_rng, K)
    if per_row:
        o = rng.integers(-700, 700, (n_rng, K)).astype(np.int32)
    else:
        o = np.array([-299, -150, -7, 0, 3, 151, 299, 612, -1000], dtype=np.int32)
    got = host(rosar.sas_time(dev(torch, raw), dev(torch, win), dev(torch, w), dev(torch, o), a_rad))
    ref = O.sas_time(raw, win, w, o, o_rad, n_rng)
    assert rel_l2(got, ref) <= TOL


def test_sas_time_per_row_equals_shared_when_rows_agree(rosar, torch):
    """The per-row kernel and the tiled kernel compute the same sums when every row holds the same
    offsets (different summation order: compared to the oracle's tolerance)."""
    cfg = synth.TINY
    sc = scene("tiny")
    w_np, o = _weights(cfg)
    win = dev(torch, synth.hann_window(cfg.L))
    raw, w = dev(torch, sc.raw), dev(torch, w_np)
    a = host(rosar.sas_time(raw, win, w, dev(torch, o), api_radar(rosar, cfg)))
    b = host(rosar.sas_time(raw, win, w, dev(torch, np.tile(o, (cfg.L, 1))), api_radar(rosar, cfg)))
    assert rel_l2(b, a) <= TOL


def test_time_domain_point_target_peaks_at_its_pixel(rosar, torch):
    cfg = synth.TINY
    L, n_az = cfg.L, cfg.n_az
    o_rad = oracle_radar(cfg)
    dR = O.range_bin_spacing(o_rad, L)
    r_t, th_t = 27, 301
    raw = O.if_cube(o_rad, n_az, L, [o_rad.r0 + r_t * dR], [O.phase_centre_angle(th_t, n_az)], [1.0])
    raw = raw.astype(np.complex64)
    win = synth.hann_window(L)
    w, o = _weights(cfg)
    for img in (rosar.bpa_time(dev(torch, raw), dev(torch, win), api_radar(rosar, cfg), L, cfg.M_ap),
                rosar.sas_time(dev(torch, raw), dev(torch, win), dev(torch, w), dev(torch, o),
                               api_radar(rosar, cfg))):
        a = np.abs(host(img)) ** 2
        assert np.unravel_index(np.argmax(a), a.shape) == (r_t, th_t)


@pytest.mark.parametrize("name", ["indoor"])
def test_time_domain_full_size_sampled_pixels(rosar, torch, name):
    """The indoor workload at full size in the benchmark's launch configuration, checked on sampled
    pixels (all rows' tiles, ragged azimuth tail included) against the oracle's per-pixel forms."""
    cfg = synth.CONFIGS[name]
    sc = scene(name)
    w, o = _weights(cfg)
    win = synth.hann_window(cfg.L)
    o_rad = oracle_radar(cfg)
    rng = np.random.default_rng(41)
    rows = np.concatenate([rng.integers(1, cfg.L, 28), [cfg.L - 1, 255 if cfg.L > 255 else cfg.L - 1]])
    thetas = np.concatenate([rng.integers(0, cfg.n_az, 28), [cfg.n_az - 1, 0]])
    sas = host(rosar.sas_time(dev(torch, sc.raw), dev(torch, win), dev(torch, w), dev(torch, o),
                              api_radar(rosar, cfg)))
    ref = O.sas_time_pixels(sc.raw, win, w, o, o_rad, cfg.n_az, rows, thetas)
    assert rel_l2(sas[rows, thetas], ref) <= TOL
    bpa = host(rosar.bpa_time(dev(torch, sc.raw), dev(torch, win), api_radar(rosar, cfg), cfg.L, cfg.M_ap))
    sel = slice(0, 12)
    ref = O.bpa_time_pixels(sc.raw, win, o_rad, cfg.n_az, cfg.M_ap, rows[sel], thetas[sel])
    assert rel_l2(bpa[rows[sel], thetas[sel]], ref) <= TOL


# ------------------------------------------------------ planned forms (B operand precomputed) --

@pytest.mark.parametrize("centred", [True, False])
def test_sas_time_planned_matches_oracle_and_unplanned(rosar, torch, centred):
    """The plan (coefficient x window x phasor of every tap, sample and row, split into bf16 pairs) fed to the
    tensor-core kernel: the tiny image against the oracle, and equal to the unplanned call within the
    tolerance; a second scan through the same plan."""
    cfg = synth.TINY
    sc = scene("tiny")
    w, o = _weights(cfg)
    win = dev(torch, synth.hann_window(cfg.L))
    plan = rosar.sas_time_plan(win, dev(torch, w), dev(torch, o), api_radar(rosar, cfg), cfg.n_az, cfg.L,
                               centred=centred)
    assert plan.data.numel() == 16384 * (cfg.L // 64) * cfg.K * (cfg.L // 16) + 8 * cfg.K
    ref = O.sas_time(sc.raw, synth.hann_window(cfg.L), w, o, oracle_radar(cfg), cfg.L, centred=centred)
    got = host(rosar.sas_time_planned(dev(torch, sc.raw), plan))
    assert rel_l2(got, ref) <= TOL
    unplanned = host(rosar.sas_time(dev(torch, sc.raw), win, dev(torch, w), dev(torch, o), api_radar(rosar, cfg),
                                    centred=centred))
    assert rel_l2(got, unplanned) <= TOL
    raw2 = np.roll(sc.raw, 41, axis=0)
    got2 = host(rosar.sas_time_planned(dev(torch, raw2), plan))
    assert rel_l2(got2, np.roll(ref, 41, axis=1)) <= TOL


@pytest.mark.parametrize("n_az,K,spread", [(1200, 16, 500), (300, 24, 900), (640, 40, 150)])
def test_sas_time_planned_wide_unsorted_offsets(rosar, torch, n_az, K, spread):
    """Shared offsets in no order, spread wider than one staged window of pulses (several windows per chunk),
    with repeats, values past n_az and below -n_az (taken modulo n_az): the planned SAS against the oracle and
    the unplanned tensor-core call."""
    L, n_rng = 48, 70
    o_rad, a_rad = _radar_pair(rosar, L)
    rng = np.random.default_rng(n_az + K)
    o = rng.integers(-spread, spread, K).astype(np.int32)
    o[1] = o[0]                                          # a repeated offset
    o[2] += 3 * n_az                                     # the same pulse as o[2] - 3 n_az
    o[3] -= 2 * n_az
    w = crand(rng, n_rng, K)
    raw = crand(rng, n_az, L)
    win = rng.uniform(0.1, 1.0, L).astype(np.float32)
    plan = rosar.sas_time_plan(dev(torch, win), dev(torch, w), dev(torch, o), a_rad, n_az, L)
    got = host(rosar.sas_time_planned(dev(torch, raw), plan))
    assert rel_l2(got, O.sas_time(raw, win, w, o, o_rad, n_rng)) <= TOL
    unplanned = host(rosar.sas_time(dev(torch, raw), dev(torch, win), dev(torch, w), dev(torch, o), a_rad))
    assert rel_l2(got, unplanned) <= TOL


@pytest.mark.parametrize("n_az,L,n_rng,M_ap", [(200, 48, 45, 13), (97, 32, 1, 97), (360, 64, 64, 60),
                                               (1000, 32, 64, 400)])
def test_bpa_time_planned_ragged(rosar, torch, n_az, L, n_rng, M_ap):
    """Planned time-domain BPA on ragged tiles (rows and azimuth off the tile, L a multiple of 16 but not a
    power of two, one row, the whole ring, a tap range wider than one staged window) against the oracle."""
    o_rad, a_rad = _radar_pair(rosar, L)
    rng = np.random.default_rng(n_az + 3 * L)
    raw = crand(rng, n_az, L)
    win = rng.uniform(0.1, 1.0, L).astype(np.float32)
    plan = rosar.bpa_time_plan(dev(torch, win), a_rad, n_az, L, n_rng, M_ap)
    got = host(rosar.bpa_time_planned(dev(torch, raw), plan))
    assert rel_l2(got, O.bpa_time(raw, win, o_rad, n_rng, M_ap)) <= TOL


def test_time_domain_planned_full_size_sampled_pixels(rosar, torch):
    """The indoor workload through the planned kernels in the benchmark's launch configuration, sampled pixels
    against the oracle."""
    cfg = synth.INDOOR
    sc = scene("indoor")
    w, o = _weights(cfg)
    win = synth.hann_window(cfg.L)
    o_rad = oracle_radar(cfg)
    rng = np.random.default_rng(43)
    rows = np.concatenate([rng.integers(1, cfg.L, 20), [cfg.L - 1]])
    thetas = np.concatenate([rng.integers(0, cfg.n_az, 20), [cfg.n_az - 1]])
    plan = rosar.sas_time_plan(dev(torch, win), dev(torch, w), dev(torch, o), api_radar(rosar, cfg), cfg.n_az, cfg.L)
    sas = host(rosar.sas_time_planned(dev(torch, sc.raw), plan))
    assert rel_l2(sas[rows, thetas], O.sas_time_pixels(sc.raw, win, w, o, o_rad, cfg.n_az, rows, thetas)) <= TOL
    bplan = rosar.bpa_time_plan(dev(torch, win), api_radar(rosar, cfg), cfg.n_az, cfg.L, cfg.L, cfg.M_ap)
    bpa = host(rosar.bpa_time_planned(dev(torch, sc.raw), bplan))
    sel = slice(0, 10)
    ref = O.bpa_time_pixels(sc.raw, win, o_rad, cfg.n_az, cfg.M_ap, rows[sel], thetas[sel])
    assert rel_l2(bpa[rows[sel], thetas[sel]], ref) <= TOL
