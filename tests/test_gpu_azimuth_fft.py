"""The frequency-domain form of the sparse azimuth filter (rosar_azimuth_plan +
rosar_sparse_azimuth_fft / rosar_image_fft) against the FP64 oracle (GPU)."""

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL_IMAGE = 1e-4
TOL_FFT_FILTER = 5e-6      # float32 FFT of length <= 16384, relative to the row energy


@pytest.fixture(scope="module")
def rosar():
    from paper_2309_08038_gb300 import build
    build.build()
    import paper_2309_08038_gb300 as r
    return r


def _c(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("n_az", [2, 30, 48, 250, 360, 1800, 3600, 7200, 14400])
def test_fft_filter_matches_oracle(rosar, n_az):
    import torch
    rng = np.random.default_rng(n_az)
    n_rng = 5
    K = min(16, n_az)
    M = min(n_az, 600)
    o = (np.sort(rng.choice(M, K, replace=False)) - M // 2).astype(np.int32)
    S, w = _c(rng, n_rng, n_az), _c(rng, n_rng, K)
    H = rosar.azimuth_plan(torch.from_numpy(w).cuda(), torch.from_numpy(o).cuda(), n_az)
    got = rosar.sparse_azimuth_fft(torch.from_numpy(S).cuda(), H).cpu().numpy()
    ref = O.sparse_azimuth(S, w, o)
    for r in range(n_rng):
        assert _rel(got[r], ref[r]) < TOL_FFT_FILTER, (n_az, r)


def test_fft_filter_per_row_duplicate_and_wild_offsets(rosar):
    import torch
    rng = np.random.default_rng(7)
    n_rng, n_az, K = 6, 3600, 9
    o = np.stack([np.sort(rng.choice(600, K, replace=False)) - 300 for _ in range(n_rng)]).astype(np.int32)
    o[1, 3] = o[1, 2] + n_az              # the same pulse twice (mod n_az): weights add
    o[2, 0] = -2 ** 31
    o[3, 4] = 2 ** 31 - 1
    S, w = _c(rng, n_rng, n_az), _c(rng, n_rng, K)
    H = rosar.azimuth_plan(torch.from_numpy(w).cuda(), torch.from_numpy(o).cuda(), n_az)
    got = rosar.sparse_azimuth_fft(torch.from_numpy(S).cuda(), H).cpu().numpy()
    ref = O.sparse_azimuth(S, w, o.astype(np.int64))
    direct = rosar.sparse_azimuth(torch.from_numpy(S).cuda(), torch.from_numpy(w).cuda(),
                                  torch.from_numpy(o).cuda()).cpu().numpy()
    assert _rel(got, ref) < TOL_FFT_FILTER
    assert _rel(got, direct) < TOL_FFT_FILTER


def test_plan_is_the_transfer_function(rosar):
    """H holds FFT(g)/N in a permuted order: its DC term is sum(w)/N and Parseval holds."""
    import torch
    rng = np.random.default_rng(8)
    n_az, K = 3600, 40
    o = (np.sort(rng.choice(600, K, replace=False)) - 300).astype(np.int32)
    w = _c(rng, 3, K)
    H = rosar.azimuth_plan(torch.from_numpy(w).cuda(), torch.from_numpy(o).cuda(), n_az).cpu().numpy()
    for r in range(3):
        g = np.zeros(n_az, np.complex128)
        np.add.at(g, (-o.astype(np.int64)) % n_az, w[r])
        ref = np.fft.fft(g) / n_az
        assert abs(H[r, 0] - ref[0]) < 1e-6 * abs(ref).max()
        np.testing.assert_allclose(np.sum(np.abs(H[r]) ** 2), np.sum(np.abs(ref) ** 2), rtol=1e-5)


@pytest.mark.parametrize("name", ["tiny", "indoor"])
def test_image_fft_matches_oracle_chain(rosar, name):
    import torch
    cfg = synth.CONFIGS[name]
    sc = synth.make_scene(cfg)
    o = synth.draw_offsets(cfg)
    w = synth.default_weights(cfg, o)
    win = synth.hann_window(cfg.L)
    H = rosar.azimuth_plan(torch.from_numpy(w).cuda(), torch.from_numpy(o).cuda(), cfg.n_az)
    got = rosar.image_fft(torch.from_numpy(sc.raw).cuda(), torch.from_numpy(win).cuda(), H).cpu().numpy()
    ref = O.sparse_azimuth(O.range_compress(sc.raw, win), w, o)
    assert _rel(got, ref) < TOL_IMAGE
    a = np.abs(ref) ** 2
    p = np.unravel_index(np.argmax(a), a.shape)
    b = a.copy()
    b[max(p[0] - 1, 0):p[0] + 2][:, [(p[1] + j) % a.shape[1] for j in (-1, 0, 1)]] = 0
    assert b.max() < (1 - 1e-3) * a[p]                       # the peak is unambiguous ...
    assert np.unravel_index(np.argmax(np.abs(got)), got.shape) == p   # ... and found on the GPU


def test_highres_fft_sampled_rows(rosar):
    import torch
    cfg = synth.HIGHRES
    rng = np.random.default_rng(78)
    raw = _c(rng, cfg.n_az, cfg.L)
    o = synth.draw_offsets(cfg)
    w = synth.default_weights(cfg, o)
    win = synth.hann_window(cfg.L)
    H = rosar.azimuth_plan(torch.from_numpy(w).cuda(), torch.from_numpy(o).cuda(), cfg.n_az)
    got = rosar.image_fft(torch.from_numpy(raw).cuda(), torch.from_numpy(win).cuda(), H)
    rows = [1, 400, 1023]
    ref = O.sparse_azimuth(O.range_compress(raw, win, bins=rows), w[rows], o[rows])
    g = got[rows].cpu().numpy()
    for i in range(len(rows)):
        assert _rel(g[i], ref[i]) < TOL_IMAGE, rows[i]


def test_unsupported_length_is_refused(rosar):
    import torch
    assert not rosar.azimuth_fft_supported(7 * 64)
    assert rosar.azimuth_fft_supported(3600)
    w = torch.zeros((2, 3), dtype=torch.complex64, device="cuda")
    o = torch.zeros(3, dtype=torch.int32, device="cuda")
    with pytest.raises(rosar.RosarError, match="UNSUPPORTED"):
        rosar.azimuth_plan(w, o, 7 * 64)


@pytest.mark.parametrize("pinned", [True, False])
def test_image_fft_host_equals_device_call(rosar, pinned):
    """rosar_image_fft_host = H2D copy + rosar_image_fft + D2H copy: the image in host memory is bit for bit
    the device call's, with page-locked and with pageable host buffers, on a side stream; consecutive calls
    on three streams with their own buffers give each scan's own image."""
    import torch
    cfg = synth.TINY
    rng = np.random.default_rng(61)
    o = synth.draw_offsets(cfg)
    w = torch.from_numpy(synth.default_weights(cfg, o)).cuda()
    H = rosar.azimuth_plan(w, torch.from_numpy(o).cuda(), cfg.n_az)
    win = torch.from_numpy(synth.hann_window(cfg.L)).cuda()
    raws = [_c(rng, cfg.n_az, cfg.L) for _ in range(3)]
    streams = [torch.cuda.Stream() for _ in range(3)]
    outs_host = []
    for i, r in enumerate(raws):
        hr = torch.from_numpy(r)
        ho = torch.empty((cfg.L, cfg.n_az), dtype=torch.complex64)
        if pinned:
            hr, ho = hr.pin_memory(), ho.pin_memory()
        rd = torch.empty((cfg.n_az, cfg.L), dtype=torch.complex64, device="cuda")
        ws = torch.empty((cfg.L, cfg.n_az), dtype=torch.complex64, device="cuda")
        od = torch.empty((cfg.L, cfg.n_az), dtype=torch.complex64, device="cuda")
        rosar.image_fft_host(hr, win, H, rd, ws, od, ho, stream=streams[i])
        outs_host.append(ho)
    torch.cuda.synchronize()
    for r, ho in zip(raws, outs_host):
        ref = rosar.image_fft(torch.from_numpy(r).cuda(), win, H).cpu()
        assert torch.equal(ho, ref)


@pytest.mark.parametrize("name,n_az,L,n_scans", [
    ("tiny", 360, 64, 1), ("tiny", 360, 64, 2), ("tiny", 360, 64, 5),
    ("indoor", 3600, 256, 3), ("1800x128", 1800, 128, 4), ("3600x512", 3600, 512, 2),
    ("fallback", 3000, 32, 3)])
def test_image_fft_scans_equals_per_scan_calls(rosar, name, n_az, L, n_scans):
    """rosar_image_fft_scans gives every scan the image of its own rosar_image_fft call, bit for bit: the
    pipelined stages (azimuth rows of scan s-1 with the range tiles of scan s in one launch, alternating
    workspaces, programmatic overlap) and the one-scan-after-another fallback alike."""
    import torch
    rng = np.random.default_rng(n_az + L + n_scans)
    K = 16
    o = (np.sort(rng.choice(min(n_az, 600), K, replace=False)) - min(n_az, 600) // 2).astype(np.int32)
    w = torch.from_numpy(_c(rng, L, K)).cuda()
    H = rosar.azimuth_plan(w, torch.from_numpy(o).cuda(), n_az)
    win = torch.from_numpy(synth.hann_window(L)).cuda()
    raw = torch.from_numpy(_c(rng, n_scans, n_az, L)).cuda()
    assert rosar.image_fft_scans_pipelined(L, n_az) == (name != "fallback")
    got = rosar.image_fft_scans(raw, win, H)
    for s in range(n_scans):
        assert torch.equal(got[s], rosar.image_fft(raw[s], win, H)), s


def test_image_fft_scans_matches_oracle_and_replays_in_a_graph(rosar):
    """Three tiny scenes (the scene rotated in azimuth) through one pipelined call against the FP64 oracle
    chain, then the same call captured in a CUDA graph and replayed on a side stream gives the same images."""
    import torch
    cfg = synth.TINY
    sc = synth.make_scene(cfg)
    o = synth.draw_offsets(cfg)
    w = synth.default_weights(cfg, o)
    win = synth.hann_window(cfg.L)
    raws = np.stack([np.roll(sc.raw, 37 * s, axis=0) for s in range(3)])
    H = rosar.azimuth_plan(torch.from_numpy(w).cuda(), torch.from_numpy(o).cuda(), cfg.n_az)
    raw_d, win_d = torch.from_numpy(raws).cuda(), torch.from_numpy(win).cuda()
    got = rosar.image_fft_scans(raw_d, win_d, H)
    for s in range(3):
        ref = O.sparse_azimuth(O.range_compress(raws[s], win), w, o)
        assert _rel(got[s].cpu().numpy(), ref) < TOL_IMAGE, s
    ws = torch.empty((2, cfg.L, cfg.n_az), dtype=torch.complex64, device="cuda")
    out = torch.zeros_like(got)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            rosar.image_fft_scans(raw_d, win_d, H, workspace=ws, out=out, stream=side)
        for _ in range(2):
            g.replay()
    side.synchronize()
    assert torch.equal(out, got)


def test_image_fft_scans_full_size_in_the_benchmark_configuration(rosar):
    """The benchmark's launch configuration: 16 indoor scans (3600 x 256, K = 64 of M = 600) in one
    rosar_image_fft_scans call; sampled rows of the first, a middle and the last scan against the FP64 oracle
    (range DFT of the sampled bins, then the sparse filter), each within 1e-4."""
    import torch
    cfg = synth.INDOOR
    rng = np.random.default_rng(16)
    n_scans = 16
    raw = _c(rng, n_scans, cfg.n_az, cfg.L)
    o = synth.draw_offsets(cfg)
    w = synth.default_weights(cfg, o)
    win = synth.hann_window(cfg.L)
    H = rosar.azimuth_plan(torch.from_numpy(w).cuda(), torch.from_numpy(o).cuda(), cfg.n_az)
    assert rosar.image_fft_scans_pipelined(cfg.L, cfg.n_az)
    got = rosar.image_fft_scans(torch.from_numpy(raw).cuda(), torch.from_numpy(win).cuda(), H)
    rows = [0, 1, 97, 255]
    for s in (0, 7, 15):
        ref = O.sparse_azimuth(O.range_compress(raw[s], win, bins=rows), w[rows], o)
        g = got[s, rows].cpu().numpy()
        for i, r in enumerate(rows):
            if not np.any(ref[i]):              # the default weights of the rotation-circle row are zero
                assert not np.any(g[i]), (s, r)
            else:
                assert _rel(g[i], ref[i]) < TOL_IMAGE, (s, r)
