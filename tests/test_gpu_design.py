"""FPP-SCA weights (Algorithm 1) through the unchanged imaging path on the GPU.

The designed per-row taps (padded to a common K with zero weights) go through rosar_sparse_azimuth
and the frequency-domain plan; both must match the oracle's filter, and a point target at a designed
row must focus at its pixel.
"""

import numpy as np
import pytest

import oracle as O
import synth
from paper_2309_08038_gb300.design import fpp_sca as F

from test_gpu_parity import dev, host, rel_l2  # noqa: F401
from test_gpu_parity import rosar, torch  # noqa: F401  (fixtures)

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def designed():
    cfg = synth.INDOOR
    rad = cfg.radar
    L = 64
    orad = O.Radar(fc=rad.fc, slope=rad.slope, t_s=rad.t_sample(L), t_start=rad.t_start, r0=rad.r0, c=rad.c)
    geo = F.Geometry(r0=rad.r0, n_az=cfg.n_az, k=O.wavenumber_centred(orad, L), M_ap=80)
    dR = O.range_bin_spacing(orad, L)
    rows = [20, 30, 45]
    p = F.Params(phi_mw_deg=2.5, eta_db=-18.0, iters=20, mc_draws=200)
    ds = {r: F.design_row(geo, rad.r0 + r * dR, p) for r in rows}
    # every row of the L-row image gets the design of the nearest designed row
    per_row = [ds[min(rows, key=lambda q: abs(q - r))] for r in range(L)]
    w, o = F.to_taps(per_row)
    return cfg, orad, L, w, o


def test_designed_taps_match_the_oracle_filter(rosar, torch, designed):
    cfg, _, L, w, o = designed
    rng = np.random.default_rng(51)
    S = (rng.standard_normal((L, cfg.n_az)) + 1j * rng.standard_normal((L, cfg.n_az))).astype(np.complex64)
    ref = O.sparse_azimuth(S, w, o)
    got = host(rosar.sparse_azimuth(dev(torch, S), dev(torch, w), dev(torch, o)))
    assert rel_l2(got, ref) <= TOL
    H = rosar.azimuth_plan(dev(torch, w), dev(torch, o), cfg.n_az)
    got_f = host(rosar.sparse_azimuth_fft(dev(torch, S), H))
    assert rel_l2(got_f, ref) <= TOL


def test_point_target_focuses_with_designed_weights(rosar, torch, designed):
    cfg, orad, L, w, o = designed
    n_az = cfg.n_az
    dR = O.range_bin_spacing(orad, L)
    r_t, th_t = 30, 1234
    raw = O.if_cube(orad, n_az, L, [orad.r0 + r_t * dR], [O.phase_centre_angle(th_t, n_az)], [1.0])
    win = synth.hann_window(L)
    img = host(rosar.image(dev(torch, raw.astype(np.complex64)), dev(torch, win), dev(torch, w), dev(torch, o)))
    a = np.abs(img[r_t]) ** 2
    assert int(np.argmax(a)) == th_t
