"""The seeded input generators agree with the oracle's signal model and weight design (CPU only)."""

import math

import numpy as np
import pytest

import oracle as O
import synth


def _oracle_radar(cfg):
    r = cfg.radar
    return O.Radar(fc=r.fc, slope=r.slope, t_s=r.t_sample(cfg.L), t_start=r.t_start, r0=r.r0, c=r.c)


def test_raw_cube_matches_oracle_signal_model_with_jitter():
    cfg = synth.TINY
    rng = np.random.default_rng(11)
    R = rng.uniform(0.4, 3.0, 5)
    phi = rng.uniform(0, 2 * math.pi, 5)
    A = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    dphi = rng.standard_normal(cfg.n_az) * math.radians(0.3)
    dr = rng.standard_normal(cfg.n_az) * 2e-3
    got = synth.synth_if(cfg, R, phi, A, dphi, dr)
    n = np.arange(cfg.n_az)
    ref = O.if_cube(_oracle_radar(cfg), cfg.n_az, cfg.L, R, phi, A,
                    O.phase_centre_angle(n, cfg.n_az) + dphi, cfg.radar.r0 + dr)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("name", ["tiny", "indoor"])
def test_default_weights_match_oracle(name):
    cfg = synth.CONFIGS[name]
    o = synth.draw_offsets(cfg)
    w = synth.default_weights(cfg, o)
    ref = O.default_weights(_oracle_radar(cfg), cfg.L, cfg.n_az, cfg.L, o, cfg.M_ap)
    assert w.dtype == np.complex64 and w.shape == (cfg.L, cfg.K)
    np.testing.assert_allclose(w, ref, rtol=0, atol=2e-7)


def test_offsets_are_sorted_unique_in_range():
    for cfg in (synth.TINY, synth.INDOOR):
        o = synth.draw_offsets(cfg)
        assert o.dtype == np.int32 and o.shape == (cfg.K,)
        assert np.all(np.diff(o) > 0) and o.min() >= -cfg.M_ap // 2 and o.max() < cfg.M_ap - cfg.M_ap // 2
    o = synth.draw_offsets(synth.HIGHRES)
    assert o.shape == (synth.HIGHRES.L, synth.HIGHRES.K) and np.all(np.diff(o, axis=1) > 0)


def test_scene_draws_are_reproducible():
    a = synth.make_scene(synth.TINY)
    b = synth.make_scene(synth.TINY)
    assert a.raw.dtype == np.complex64 and a.raw.shape == (360, 64)
    assert np.array_equal(a.raw, b.raw)


def test_hann_window():
    np.testing.assert_allclose(synth.hann_window(64), O.hann_symmetric(64), atol=1e-7)


def test_migration_offsets_match_oracle():
    for cfg in (synth.TINY, synth.INDOOR):
        o = synth.draw_offsets(cfg)
        got = synth.migration_offsets(cfg, o)
        ref = O.migration_offsets(_oracle_radar(cfg), cfg.L, cfg.n_az, cfg.L, o)
        assert got.dtype == np.int32 and np.array_equal(got, ref)
