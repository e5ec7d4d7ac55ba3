"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test ties an oracle function to something other than itself: the paper's
printed numbers (tests/golden/paper_geometry.json), closed forms, a library
routine for a textbook special case, or an invariant that a dropped term, a
wrong sign or a transposed index would break.
"""

import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _paper():
    with open(os.path.join(GOLD, "paper_geometry.json")) as f:
        return json.load(f)


def _radar77(L):
    # 77 GHz, 4 GHz over 40 us, ADC window = central 60 % of the ramp, r0 = 0.25 m
    slope = 4e9 / 40e-6
    return O.Radar(fc=77e9, slope=slope, t_s=0.6 * 40e-6 / L, t_start=8e-6, r0=0.25)


# ----------------------------------------------------------------- geometry --

def test_effective_aperture_matches_paper():
    """Sec. IV-D-1: a target at (pi/2, 2 m) with r = 0.145 m, N = 800 sees 381 phase centres (Eq. (5))."""
    p = _paper()
    n_min, n_max = O.visible_pulses(p["target_R_m"], p["r_m"], p["N"])
    assert n_max - n_min + 1 == p["effective_phase_centres"]


def test_visibility_equals_antenna_pattern_support():
    """Eq. (5)'s index range is exactly where p(theta_n) of Eqs. (3), (8) is non-zero."""
    p = _paper()
    n = np.arange(p["N"])
    theta = O.off_boresight_angle(p["target_R_m"], math.pi / 2, p["r_m"], O.phase_centre_angle(n, p["N"]))
    vis = np.nonzero(O.antenna_pattern(theta) > 0)[0]
    n_min, n_max = O.visible_pulses(p["target_R_m"], p["r_m"], p["N"])
    assert vis[0] == n_min and vis[-1] == n_max and vis.size == n_max - n_min + 1


def test_range_resolution_matches_paper():
    """Sec. IV-B: R_delta = c/2B = 0.0435 m with B the sampled sweep; bin spacing of Eq. (40) equals c/2B."""
    p = _paper()
    ts = 1.0 / p["fs_hz"]
    rad = O.Radar(fc=p["f_start_hz"], slope=p["slope_hz_per_s"], t_s=ts, t_start=p["t_start_s"], r0=p["r_m"])
    B = p["slope_hz_per_s"] * (p["t_sample_end_s"] - p["t_start_s"])
    dR = O.range_bin_spacing(rad, p["M"])
    assert dR == pytest.approx(O.C_LIGHT / (2 * B), rel=1e-12)
    assert dR == pytest.approx(p["range_resolution_m"], rel=0.02)
    # maximum unambiguous range c*Fs/(4K) (real sampling keeps half the bins)
    assert p["M"] * dR / 2 == pytest.approx(p["max_unambiguous_range_m"], rel=0.02)


# --------------------------------------------------------- range compression --

@pytest.mark.parametrize("L", [8, 64, 1024])
def test_dft_matrix_is_the_textbook_dft(L):
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    np.testing.assert_allclose(O.dft_matrix(L) @ x, np.fft.fft(x), rtol=0, atol=1e-10 * np.sqrt(L))


@pytest.mark.parametrize("centred", [False, True])
def test_integer_tone_lands_in_one_bin(centred):
    L, b, n_az = 64, 11, 3
    m = np.arange(L)
    raw = np.tile(np.exp(2j * math.pi * b * m / L), (n_az, 1))
    S = O.range_compress(raw, np.ones(L), centred=centred)
    expect = L * (np.exp(1j * math.pi * b * (L - 1) / L) if centred else 1.0)
    np.testing.assert_allclose(S[b], expect, rtol=1e-12)
    others = np.delete(S, b, axis=0)
    assert np.abs(others).max() < 1e-10


def test_centred_peak_phase_is_two_k_mid_R():
    """A boresight target whose slant range is a whole number of bins: the centred spectrum at
    l* is A * p * sum(win) * exp(j*2*k_mid*R) (derivation of Eqs. (38)-(39) about the window centre)."""
    L, n_az = 64, 360
    rad = _radar77(L)
    dR = O.range_bin_spacing(rad, L)
    n0, l_star = 90, 20
    R_t = rad.r0 + l_star * dR
    A = 0.7 * np.exp(0.3j)
    raw = O.if_cube(rad, n_az, L, [R_t], [O.phase_centre_angle(n0, n_az)], [A])
    win = O.hann_symmetric(L)
    S = O.range_compress(raw, win, centred=True)
    expect = A * win.sum() * np.exp(2j * O.wavenumber_centred(rad, L) * l_star * dR)
    assert abs(S[l_star, n0] - expect) < 1e-9 * abs(expect)
    # without centring the phase is off by the Dirichlet term of Remark 1
    S0 = O.range_compress(raw, win, centred=False)
    assert abs(np.angle(S0[l_star, n0] / expect)) > 1e-3


def test_peak_bin_matches_eq40():
    """T3: the peak of every visible range profile is round(2 R_n K t_s L / c) (Eq. (40))."""
    L, n_az = 64, 360
    rad = _radar77(L)
    R_t, phi_t = 2.13, 1.1
    raw = O.if_cube(rad, n_az, L, [R_t], [phi_t], [1.0])
    S = O.range_compress(raw, O.hann_symmetric(L))
    n = np.arange(n_az)
    R_n = O.slant_range(R_t, phi_t, rad.r0, O.phase_centre_angle(n, n_az))
    x = 2 * R_n * rad.slope * rad.t_s * L / rad.c
    vis = O.antenna_pattern(O.off_boresight_angle(R_t, phi_t, rad.r0, O.phase_centre_angle(n, n_az))) > 0.05
    ok = vis & (np.abs(x - np.floor(x) - 0.5) > 0.15)
    assert ok.sum() > 50
    assert np.array_equal(np.argmax(np.abs(S[:, ok]), axis=0), O.peak_range_bin(R_n[ok], rad, L))


# ----------------------------------------------------- sparse azimuth filter --

def test_sparse_azimuth_identity():
    rng = np.random.default_rng(1)
    S = rng.standard_normal((5, 17)) + 1j * rng.standard_normal((5, 17))
    out = O.sparse_azimuth(S, np.ones((5, 1)), np.array([0]))
    assert np.array_equal(out, S)


def test_full_aperture_is_circular_correlation():
    """K = M_ap with every offset: out_r = IFFT(FFT(S_r) * N*IFFT(h_r)), h_r[d mod N] = w[r, d]."""
    rng = np.random.default_rng(2)
    n_rng, N, M = 4, 50, 12
    S = rng.standard_normal((n_rng, N)) + 1j * rng.standard_normal((n_rng, N))
    o = np.arange(-M // 2, M - M // 2)
    w = rng.standard_normal((n_rng, M)) + 1j * rng.standard_normal((n_rng, M))
    out = O.sparse_azimuth(S, w, o)
    for r in range(n_rng):
        h = np.zeros(N, dtype=np.complex128)
        h[o % N] = w[r]
        ref = np.fft.ifft(np.fft.fft(S[r]) * N * np.fft.ifft(h))
        np.testing.assert_allclose(out[r], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_shift_equivariance_is_exact():
    """T6: rolling the pulses by s rolls the image by s (same taps, same k order: bit-exact in FP64)."""
    rng = np.random.default_rng(3)
    S = rng.standard_normal((6, 40)) + 1j * rng.standard_normal((6, 40))
    o = np.array([-7, -2, 0, 3, 9])
    w = rng.standard_normal((6, 5)) + 1j * rng.standard_normal((6, 5))
    for s in (1, 13, 39):
        assert np.array_equal(O.sparse_azimuth(np.roll(S, s, axis=1), w, o),
                              np.roll(O.sparse_azimuth(S, w, o), s, axis=1))


def test_per_row_offsets_equal_shared_when_identical():
    rng = np.random.default_rng(4)
    S = rng.standard_normal((3, 30)) + 1j * rng.standard_normal((3, 30))
    o = np.array([-5, 1, 4])
    w = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    assert np.array_equal(O.sparse_azimuth(S, w, o), O.sparse_azimuth(S, w, np.tile(o, (3, 1))))


def _peak_with_margin(img):
    a = np.abs(img) ** 2
    idx = np.unravel_index(np.argmax(a), a.shape)
    b = a.copy()
    r, t = idx
    b[max(r - 1, 0):r + 2][:, [(t + j) % a.shape[1] for j in (-1, 0, 1)]] = 0
    assert b.max() < (1 - 1e-3) * a[idx]
    return tuple(int(i) for i in idx)


@pytest.mark.parametrize("pix", [(20, 90), (35, 200), (12, 359)])
def test_point_target_focuses_at_its_pixel(pix):
    """A noise-free point target at the centre of pixel (r*, theta*) peaks at (r*, theta*) in both the
    sparse-aperture image (Eq. (43) with the default weights) and the BPA image."""
    L, n_az, K, M = 64, 360, 16, 60
    rad = _radar77(L)
    dR = O.range_bin_spacing(rad, L)
    r_s, t_s = pix
    raw = O.if_cube(rad, n_az, L, [rad.r0 + r_s * dR], [O.phase_centre_angle(t_s, n_az)], [1.0])
    S = O.range_compress(raw, O.hann_symmetric(L))
    o = np.sort(np.random.default_rng(100).choice(M, K, replace=False)) - M // 2
    w = O.default_weights(rad, L, n_az, L, o, M)
    assert _peak_with_margin(O.sparse_azimuth(S, w, o)) == pix
    for interp in ("linear", "nearest"):
        assert _peak_with_margin(O.bpa(S, rad, L, M, interp=interp)) == pix


# ------------------------------------------------------------------- BPA --

def test_nearest_bpa_equals_full_aperture_matched_filter():
    """T5: when every tap's nearest bin is the pixel's row, nearest-bin BPA is Eq. (43) with
    w_BP[d] = alpha_d exp(-j 2 k_mid R_d) over all M_ap pulses (the weight of Sec. III-D)."""
    L, n_az, M = 64, 360, 20
    rad = _radar77(L)
    dR = O.range_bin_spacing(rad, L)
    rng = np.random.default_rng(5)
    S = rng.standard_normal((L, n_az)) + 1j * rng.standard_normal((L, n_az))
    d = np.arange(-M // 2, M - M // 2)
    k_mid = O.wavenumber_centred(rad, L)
    checked = 0
    for r in (8, 20, 40):
        R = rad.r0 + r * dR
        R_d = O.slant_range(R, 0.0, rad.r0, O.phase_centre_angle(d, n_az))
        assert np.all(np.floor(R_d / dR + 0.5) == r)
        a = O.antenna_pattern(O.off_boresight_angle(R, 0.0, rad.r0, O.phase_centre_angle(d, n_az)))
        w_bp = (a * np.exp(-2j * k_mid * R_d))[None, :]
        ref = O.sparse_azimuth(S[r:r + 1], w_bp, d)[0]
        got = O.bpa_pixels(S, rad, n_az, M, np.full(n_az, r), np.arange(n_az), interp="nearest")
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        checked += 1
    assert checked == 3


@pytest.mark.parametrize("errors", [False, True])
def test_linear_bpa_is_exact_on_range_profiles_affine_in_the_bin(errors):
    """Linear interpolation between bins floor(x) and floor(x) + 1 reproduces a range profile that is affine in
    the bin index exactly, so with S[l, n] = (a + b*l) c_n the BPA sum has the closed form
    sum_d alpha_d exp(-j 2 k_mid R_d) (a + b R_d / dR) c_n (Sec. III-D with w_BP), at nominal and at supplied
    pulse positions (Eq. (37)).  Swapped interpolation weights, an off-by-one bin or a dropped term fail it."""
    L, n_az, M = 64, 360, 24
    rad = _radar77(L)
    dR = O.range_bin_spacing(rad, L)
    k_mid = O.wavenumber_centred(rad, L)
    rng = np.random.default_rng(11)
    a, b = complex(rng.standard_normal(), rng.standard_normal()), complex(rng.standard_normal(), 0.3)
    c = rng.standard_normal(n_az) + 1j * rng.standard_normal(n_az)
    S = (a + b * np.arange(L))[:, None] * c[None, :]
    dphi = rng.uniform(-1, 1, n_az) * math.radians(0.5) if errors else None
    dr = rng.uniform(-1, 1, n_az) * 0.4 * dR if errors else None
    d = np.arange(-(M // 2), M - M // 2)
    for r, th in ((10, 0), (25, 123), (50, 359)):
        R = rad.r0 + r * dR
        n = (th + d) % n_az
        phi_rel = O.phase_centre_angle(d, n_az) + (dphi[n] if errors else 0.0)
        r_n = rad.r0 + (dr[n] if errors else 0.0)
        R_d = O.slant_range(R, 0.0, r_n, phi_rel)
        assert np.all((R_d / dR >= 0) & (R_d / dR < L - 1))          # every sample inside the profile
        alpha = O.antenna_pattern(O.off_boresight_angle(R, 0.0, r_n, phi_rel))
        ref = np.sum(alpha * np.exp(-2j * k_mid * R_d) * (a + b * R_d / dR) * c[n])
        got = O.bpa_pixels(S, rad, n_az, M, [r], [th], interp="linear", dphi=dphi, dr=dr)[0]
        assert abs(got - ref) <= 1e-11 * np.sum(np.abs(alpha * (a + b * R_d / dR) * c[n]))


def test_pulse_position_error_bounds_the_slant_range_change():
    """The GPU BPA sizes its staged range window with this bound: moving a phase centre from (r0, phi) to
    (r0 + dr, phi + eps) changes its distance to any pixel (Eq. (2)) by at most |dr| + 2 r0 |sin(eps/2)|
    (triangle inequality), with equality for a pixel on the line through the two positions."""
    rng = np.random.default_rng(12)
    r0 = 0.25
    R = r0 + rng.uniform(0.0, 15.0, 20000)
    phi_t = rng.uniform(-math.pi, math.pi, R.shape)
    phi = rng.uniform(-math.pi, math.pi, R.shape)
    eps = rng.normal(0.0, math.radians(2.0), R.shape)
    dr = rng.normal(0.0, 0.01, R.shape)
    change = np.abs(O.slant_range(R, phi_t, r0 + dr, phi + eps) - O.slant_range(R, phi_t, r0, phi))
    bound = np.abs(dr) + 2.0 * r0 * np.abs(np.sin(eps / 2.0))
    assert np.all(change <= bound * (1 + 1e-12) + 1e-15)
    # tight: a radial move seen from a pixel beyond it on the same ray, and a rotation by eps seen from a pixel
    # on the extension of the chord between the two positions
    assert abs(O.slant_range(3.0, 0.0, r0 + 0.02, 0.0) - O.slant_range(3.0, 0.0, r0, 0.0)) == pytest.approx(0.02)
    e = 0.3
    p0, p1 = r0, r0 * complex(math.cos(e), math.sin(e))
    x = p1 + 2.0 * (p1 - p0) / abs(p1 - p0)
    d = O.slant_range(abs(x), math.atan2(x.imag, x.real), r0, 0.0) - O.slant_range(abs(x), math.atan2(x.imag, x.real), r0, e)
    assert d == pytest.approx(2.0 * r0 * math.sin(e / 2.0), rel=1e-12)


def test_bpa_uses_the_supplied_pulse_positions():
    """With rotation errors (Eq. (37)) in the data, BPA given the true positions recovers the
    error-free peak; BPA on nominal positions loses coherence."""
    L, n_az, M = 64, 360, 60
    rad = _radar77(L)
    dR = O.range_bin_spacing(rad, L)
    rng = np.random.default_rng(6)
    dphi = rng.standard_normal(n_az) * math.radians(1.0)
    dr = rng.standard_normal(n_az) * 3e-3
    R_t, phi_t = rad.r0 + 30 * dR, O.phase_centre_angle(100, n_az)
    n = np.arange(n_az)
    raw_j = O.if_cube(rad, n_az, L, [R_t], [phi_t], [1.0], O.phase_centre_angle(n, n_az) + dphi, rad.r0 + dr)
    raw_0 = O.if_cube(rad, n_az, L, [R_t], [phi_t], [1.0])
    win = O.hann_symmetric(L)
    Sj, S0 = O.range_compress(raw_j, win), O.range_compress(raw_0, win)
    ref = abs(O.bpa_pixels(S0, rad, n_az, M, [30], [100])[0])
    good = abs(O.bpa_pixels(Sj, rad, n_az, M, [30], [100], dphi=dphi, dr=dr)[0])
    bad = abs(O.bpa_pixels(Sj, rad, n_az, M, [30], [100])[0])
    assert good == pytest.approx(ref, rel=0.03)
    assert bad < 0.8 * ref


# ----------------------------------------------------------------- weights --

@pytest.mark.parametrize("M", [60, 61, 600])
def test_taylor_taper_matches_library(M):
    sw = pytest.importorskip("scipy.signal.windows")
    np.testing.assert_allclose(O.taylor_taper(M, 4, 30.0), sw.taylor(M, nbar=4, sll=30, norm=True), atol=1e-12)


def test_taylor_with_one_term_is_uniform():
    np.testing.assert_allclose(O.taylor_taper(37, nbar=1), np.ones(37), atol=1e-15)


def test_default_weights_unit_norm_and_boresight_phase():
    L, n_az, K, M = 64, 360, 16, 60
    rad = _radar77(L)
    dR = O.range_bin_spacing(rad, L)
    o = np.sort(np.random.default_rng(100).choice(M, K, replace=False)) - M // 2
    o[np.argmin(np.abs(o))] = 0
    o = np.sort(o)
    w = O.default_weights(rad, L, n_az, L, o, M)
    np.testing.assert_allclose(np.linalg.norm(w[1:], axis=1), 1.0, rtol=1e-12)
    k0 = int(np.nonzero(o == 0)[0][0])
    r = np.arange(1, L)
    ph = np.angle(w[1:, k0] * np.exp(2j * O.wavenumber_centred(rad, L) * r * dR))
    np.testing.assert_allclose(ph, 0.0, atol=1e-9)
    # row 0 (pixel on the rotation circle) keeps only the tap that faces it
    assert abs(w[0, k0]) == pytest.approx(1.0) and np.count_nonzero(w[0]) == 1


# ---------------------------------------------------------------- adjoints --

def _rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_adjoint_identities():
    rng = np.random.default_rng(7)
    n_rng, N, K = 5, 33, 6
    S, g = _rand_c(rng, n_rng, N), _rand_c(rng, n_rng, N)
    w = _rand_c(rng, n_rng, K)
    o = np.array([-9, -4, 0, 2, 5, 15])
    lhs = np.vdot(O.sparse_azimuth(S, w, o), g)
    np.testing.assert_allclose(lhs, np.vdot(S, O.sparse_azimuth_adjoint_S(g, w, o)), rtol=1e-12)
    # linear in w with coefficients S[r, theta + o_k]
    np.testing.assert_allclose(lhs, np.vdot(w, O.sparse_azimuth_adjoint_w(g, S, o)), rtol=1e-12)
    L = 16
    raw, G = _rand_c(rng, 7, L), _rand_c(rng, L, 7)
    win = O.hann_symmetric(L)
    for centred in (False, True):
        np.testing.assert_allclose(np.vdot(O.range_compress(raw, win, centred), G),
                                   np.vdot(raw, O.range_compress_adjoint(G, win, centred)), rtol=1e-12)


def test_gradients_match_central_differences():
    """Loss ||F(S*exp(j eps), w) - B||^2: oracle gradients in eps and w vs FP64 central differences."""
    rng = np.random.default_rng(8)
    n_rng, N, K, M = 8, 64, 16, 32
    S, B = _rand_c(rng, n_rng, N), _rand_c(rng, n_rng, N)
    w = _rand_c(rng, n_rng, K) / 4
    o = np.sort(rng.choice(M, K, replace=False)) - M // 2
    eps = rng.standard_normal(N) * 0.3

    def loss(eps_, w_):
        r = O.sparse_azimuth(O.apply_phase_errors(S, eps_), w_, o) - B
        return float(np.sum(np.abs(r) ** 2))

    St = O.apply_phase_errors(S, eps)
    g = 2.0 * (O.sparse_azimuth(St, w, o) - B)
    G = O.sparse_azimuth_adjoint_S(g, w, o)
    d_eps = O.phase_error_grad(St, G)
    d_w = O.sparse_azimuth_adjoint_w(g, St, o)
    h = 1e-6
    fd_eps = np.array([(loss(eps + h * e, w) - loss(eps - h * e, w)) / (2 * h) for e in np.eye(N)[:12]])
    np.testing.assert_allclose(d_eps[:12], fd_eps, rtol=1e-6, atol=1e-6 * np.abs(fd_eps).max())
    fd_w = np.zeros((2, K), dtype=np.float64)
    for k in range(K):
        for part, dz in enumerate((1.0, 1j)):
            e = np.zeros_like(w)
            e[3, k] = h * dz
            fd_w[part, k] = (loss(eps, w + e) - loss(eps, w - e)) / (2 * h)
    np.testing.assert_allclose(d_w[3], fd_w[0] + 1j * fd_w[1], rtol=1e-6, atol=1e-6 * np.abs(d_w[3]).max())


# ----------------------------------------------------------------- metrics --

def test_entropy_closed_forms():
    assert O.image_entropy(np.ones((4, 8))) == pytest.approx(math.log(32), rel=1e-14)
    z = np.zeros((3, 3), dtype=complex)
    z[1, 2] = 2 - 1j
    assert O.image_entropy(z) == 0.0
    z[0, 0] = 1 + 2j
    assert O.image_entropy(z) == pytest.approx(math.log(2), rel=1e-14)


def test_pisr_and_mainlobe_hand_cases():
    row = np.array([3.0, 1.0, 0.5, 0.2, 0.4, 1.0 + 0j])
    assert O.pisr(row, 0, [2, 3, 4]) == pytest.approx(9.0 / (0.25 + 0.04 + 0.16))
    assert O.half_mainlobe_width(row, 0) == 3          # both sides fall for 3 samples
    # right side falls for 3 samples, the left side (wrapping) for 2: the closer minimum wins
    assert O.half_mainlobe_width(np.array([3.0, 2.0, 1.0, 0.5, 0.7, 0.1, 1.5]), 0) == 2
    assert O.half_mainlobe_width(np.array([0.1, 0.5, 2.0, 1.5, 1.0, 0.7, 0.9]), 2) == 2


# ------------------------------------------------- range-migration-aware taps --

def test_migrating_filter_reduces_to_fixed_row():
    rng = np.random.default_rng(9)
    S = rng.standard_normal((6, 40)) + 1j * rng.standard_normal((6, 40))
    w = rng.standard_normal((6, 5)) + 1j * rng.standard_normal((6, 5))
    o = np.array([-7, -2, 0, 3, 9])
    assert np.array_equal(O.sparse_azimuth_migrating(S, w, o, np.zeros((6, 5), int)), O.sparse_azimuth(S, w, o))
    # a uniform shift of every tap by one row is the fixed-row filter on the shifted rows (last row reads zero)
    shifted = O.sparse_azimuth_migrating(S, w, o, np.ones((6, 5), int))
    np.testing.assert_array_equal(shifted[:5], O.sparse_azimuth(S[1:], w[:5], o))
    assert not shifted[5].any()


def test_migration_offsets_follow_eq40_and_focus_better():
    """dl[r,k] = l* - r with l* of Eq. (40) at the tap's slant range; reading those bins gathers more of a
    point target's energy than the fixed row (the paper's Eq. (43) uses l*_n), peak at the same pixel."""
    L, n_az, M = 256, 3600, 600
    rad = _radar77(L)
    dR = O.range_bin_spacing(rad, L)
    o = np.arange(-M // 2, M // 2, 9)
    dl = O.migration_offsets(rad, L, n_az, L, o)
    assert dl[16:].min() == 0 and dl[16:].max() == 1 and dl.max() <= 2   # at +-30 deg: <= 1 bin except near r0
    r_s, t_s = 4, 1000                                        # a pixel 0.5 m out: the outer taps migrate ~1 bin
    assert dl[r_s].max() == 1
    R_t = rad.r0 + r_s * dR
    raw = O.if_cube(rad, n_az, L, [R_t], [O.phase_centre_angle(t_s, n_az)], [1.0])
    S = O.range_compress(raw, O.hann_symmetric(L), bins=range(0, r_s + 6))
    Sw = np.zeros((r_s + 6, n_az), complex)
    Sw[:] = S
    rows = slice(r_s - 2, r_s + 3)
    w = O.default_weights(rad, L, n_az, L, o, M)[rows]
    fixed = O.sparse_azimuth(Sw[rows], w, o)
    mig = O.sparse_azimuth_migrating(Sw[r_s - 2:], w, o, dl[rows])
    assert np.unravel_index(np.argmax(np.abs(fixed)), fixed.shape) == (2, t_s)
    assert np.unravel_index(np.argmax(np.abs(mig)), mig.shape) == (2, t_s)
    assert np.abs(mig[2, t_s]) > 1.01 * np.abs(fixed[2, t_s])


# ------------------------------------------------- time-domain BPA and SAS --

def _rand_raw(rng, n_az, L):
    return rng.standard_normal((n_az, L)) + 1j * rng.standard_normal((n_az, L))


@pytest.mark.parametrize("centred", [False, True])
def test_time_domain_sas_with_one_facing_tap_is_the_range_dft(centred):
    """A single tap at pulse offset 0 sees the pixel of row r at slant range exactly r*dR, so W_SA's
    fast-time compensation is the DFT row of bin r (Eq. (38)/(40)): SAS with o = [0], w = 1 is the
    range compression, centred or not."""
    L, n_az = 64, 40
    rad = _radar77(L)
    rng = np.random.default_rng(21)
    raw = _rand_raw(rng, n_az, L)
    win = O.hann_symmetric(L)
    got = O.sas_time(raw, win, np.ones((L, 1)), np.array([0]), rad, L, centred=centred)
    ref = O.range_compress(raw, win, centred=centred)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_time_domain_bpa_with_one_pulse_equals_fft_bpa():
    """With M_ap = 1 the only tap faces the pixel, its slant range is r*dR, a whole bin: the
    time-domain BPA of Eq. (14) (k, fast time from m = 0) equals the range-compressed BPA (k_mid,
    centred DFT, nearest bin) -- the two phase references differ by exactly the centring factor."""
    L, n_az = 64, 30
    rad = _radar77(L)
    rng = np.random.default_rng(22)
    raw = _rand_raw(rng, n_az, L)
    win = O.hann_symmetric(L)
    got = O.bpa_time(raw, win, rad, L, 1)
    ref = O.bpa(O.range_compress(raw, win), rad, L, 1, interp="nearest")
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("use_win", [False, True])
def test_time_domain_bpa_compensates_a_point_at_the_pixel_exactly(use_win):
    """Sec. II-C: for a target at the imaged point every phase of W_BP . Y_IF cancels, so Eq. (14)
    returns A * sum_n p(theta_n)^2 * sum_m win[m] (amplitude of Eq. (15) times alpha_n = p(theta_n))."""
    L, n_az, M = 64, 360, 60
    rad = _radar77(L)
    dR = O.range_bin_spacing(rad, L)
    r_t, th_t, A = 25, 123, 0.7 - 0.4j
    R_t, phi_t = rad.r0 + r_t * dR, O.phase_centre_angle(th_t, n_az)
    raw = O.if_cube(rad, n_az, L, [R_t], [phi_t], [A])
    win = O.hann_symmetric(L) if use_win else None
    d = np.arange(-(M // 2), M - M // 2)
    phi_n = O.phase_centre_angle(th_t + d, n_az)
    p = O.antenna_pattern(O.off_boresight_angle(R_t, phi_t, rad.r0, phi_n))
    expect = A * np.sum(p * p) * (np.sum(win) if use_win else L)
    got = O.bpa_time_pixels(raw, win, rad, n_az, M, [r_t], [th_t])[0]
    assert abs(got - expect) <= 1e-9 * abs(expect)
    img = O.bpa_time(raw, win, rad, L, M)
    assert abs(img[r_t, th_t] - expect) <= 1e-9 * abs(expect)
    assert _peak_with_margin(img) == (r_t, th_t)


@pytest.mark.parametrize("centred", [False, True])
def test_time_domain_sas_with_matched_weights_is_fully_compensated(centred):
    """Algorithm 2 with w = conj(steering vector)/norm (Eq. (16), wavenumber k with W_SA verbatim,
    k_mid with the centred W_SA) returns A * sum(T p^2)/||T p|| * sum win at the target's own pixel."""
    L, n_az, K, M = 64, 360, 16, 60
    rad = _radar77(L)
    dR = O.range_bin_spacing(rad, L)
    r_t, th_t, A = 30, 7, 1.3 + 0.2j
    raw = O.if_cube(rad, n_az, L, [rad.r0 + r_t * dR], [O.phase_centre_angle(th_t, n_az)], [A])
    win = O.hann_symmetric(L)
    o = np.sort(np.random.default_rng(100).choice(M, K, replace=False)) - M // 2
    R = rad.r0 + r_t * dR
    rho = O.slant_range(R, 0.0, rad.r0, O.phase_centre_angle(o, n_az))
    p = O.antenna_pattern(O.off_boresight_angle(R, 0.0, rad.r0, O.phase_centre_angle(o, n_az)))
    T = O.taylor_taper(M)[o + M // 2]
    kk = O.wavenumber_centred(rad, L) if centred else O.wavenumber(rad)
    v = T * p * np.exp(-2j * kk * rho)
    w = np.zeros((L, K), dtype=np.complex128)
    w[r_t] = v / np.linalg.norm(v)
    expect = A * np.sum(T * p * p) / np.linalg.norm(T * p) * np.sum(win)
    got = O.sas_time_pixels(raw, win, w, o, rad, n_az, [r_t], [th_t], centred=centred)[0]
    assert abs(got - expect) <= 1e-9 * abs(expect)
    img = O.sas_time(raw, win, w, o, rad, L, centred=centred)
    assert abs(img[r_t, th_t] - expect) <= 1e-9 * abs(expect)


def test_time_domain_forms_match_brute_force_loops():
    """Scalar loops straight from Eq. (14) and Algorithm 2 (math module, no numpy broadcasting) on a
    tiny cube; the vectorised full-image and per-pixel forms must agree with them everywhere."""
    L, n_az, K, M, n_rng = 6, 11, 3, 4, 5
    rad = O.Radar(fc=77e9, slope=1e14, t_s=4e-6, t_start=8e-6, r0=0.25)
    rng = np.random.default_rng(23)
    raw = _rand_raw(rng, n_az, L)
    win = rng.uniform(0.2, 1.0, L)
    w = rng.standard_normal((n_rng, K)) + 1j * rng.standard_normal((n_rng, K))
    o = np.array([-5, 1, 3])
    dR = rad.c / (2 * rad.slope * rad.t_s * L)
    k = 2 * math.pi * (rad.slope * rad.t_start + rad.fc) / rad.c
    bpa = np.zeros((n_rng, n_az), dtype=complex)
    sas = np.zeros((n_rng, n_az), dtype=complex)
    for r in range(n_rng):
        R = rad.r0 + r * dR
        for t in range(n_az):
            for d in range(-(M // 2), M - M // 2):
                n = (t + d) % n_az
                dphi = 2 * math.pi * (n - t) / n_az
                Rn = math.sqrt(R * R + rad.r0 ** 2 - 2 * R * rad.r0 * math.cos(dphi))
                th = math.atan2(R * math.sin(abs(dphi)), R * math.cos(abs(dphi)) - rad.r0)
                a = math.cos(th) if abs(th) < math.pi / 2 else 0.0
                tau = 2 * Rn / rad.c
                for m in range(L):
                    W = a * complex(math.cos(-2 * math.pi * tau * rad.slope * m * rad.t_s - 2 * k * Rn),
                                    math.sin(-2 * math.pi * tau * rad.slope * m * rad.t_s - 2 * k * Rn))
                    bpa[r, t] += W * win[m] * raw[n, m]
            for kk in range(K):
                n = (t + o[kk]) % n_az
                dphi = 2 * math.pi * o[kk] / n_az
                rho = math.sqrt(R * R + rad.r0 ** 2 - 2 * R * rad.r0 * math.cos(dphi))
                tau = 2 * rho / rad.c
                acc = 0j
                for m in range(L):
                    ph = -2 * math.pi * tau * rad.slope * rad.t_s * (m - (L - 1) / 2)
                    acc += complex(math.cos(ph), math.sin(ph)) * win[m] * raw[n, m]
                sas[r, t] += w[r, kk] * acc
    tol = 1e-10 * np.abs(bpa).max()
    np.testing.assert_allclose(O.bpa_time(raw, win, rad, n_rng, M), bpa, rtol=0, atol=tol)
    rr, tt = np.meshgrid(np.arange(n_rng), np.arange(n_az), indexing="ij")
    np.testing.assert_allclose(O.bpa_time_pixels(raw, win, rad, n_az, M, rr, tt).reshape(n_rng, n_az), bpa,
                               rtol=0, atol=tol)
    tol = 1e-10 * np.abs(sas).max()
    np.testing.assert_allclose(O.sas_time(raw, win, w, o, rad, n_rng), sas, rtol=0, atol=tol)
    np.testing.assert_allclose(O.sas_time_pixels(raw, win, w, o, rad, n_az, rr, tt).reshape(n_rng, n_az), sas,
                               rtol=0, atol=tol)
    # per-row offsets: row r of a per-row table equal to o everywhere but one row
    orow = np.tile(o, (n_rng, 1))
    orow[2] = [-1, 0, 4]
    img = O.sas_time(raw, win, w, orow, rad, n_rng)
    np.testing.assert_allclose(np.delete(img, 2, axis=0), np.delete(sas, 2, axis=0), rtol=0, atol=tol)
    assert np.abs(img[2] - sas[2]).max() > 1e-3 * np.abs(sas).max()
