"""Batched form: one persistent graph-captured launch over uneven scans (GPU).

Each scan's image must equal rosar_image of that scan bit for bit (same tiles,
same arithmetic, same tap order) and the FP64 oracle within the image bar; every
tuning must give the same bits; a dependency wait that cannot be met must end
with ROSAR_ERR_TIMEOUT and leave the context usable.
"""

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


def _crand(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


SHAPES = [  # (n_az, L, K, per_row_offsets, window)
    (360, 64, 16, False, True),
    (1800, 128, 32, False, True),
    (37, 16, 1, False, False),
    (1031, 256, 300, False, True),
    (3600, 512, 64, True, True),
    (900, 1024, 128, False, True),
    (250, 2048, 8, False, False),
    (7200, 32, 64, False, True),
]


def _make_scans(torch, seed=0):
    rng = np.random.default_rng(seed)
    scans, host = [], []
    for n_az, L, K, per_row, use_win in SHAPES:
        M = max(K, min(n_az, n_az // 6 if n_az >= 6 * K else n_az))
        raw = _crand(rng, n_az, L)
        if per_row:
            o = np.stack([np.sort(rng.choice(M, K, replace=False)) - M // 2 for _ in range(L)]).astype(np.int32)
        else:
            o = (np.sort(rng.choice(M, K, replace=False)) - M // 2).astype(np.int32)
        w = _crand(rng, L, K)
        win = synth.hann_window(L) if use_win else None
        scans.append({"raw": torch.from_numpy(raw).cuda(), "w": torch.from_numpy(w).cuda(),
                      "o": torch.from_numpy(o).cuda(),
                      "win": torch.from_numpy(win).cuda() if win is not None else None})
        host.append((raw, w, o, win))
    return scans, host


def _per_scan_reference(rosar, scans):
    return [rosar.image(s["raw"], s["win"], s["w"], s["o"]).cpu().numpy() for s in scans]


def test_batch_equals_per_scan_image_and_oracle(rosar):
    import torch
    scans, host = _make_scans(torch)
    ref = _per_scan_reference(rosar, scans)
    b = rosar.Batch(scans)
    info = b.info()
    assert info["ctas"] >= 1 and info["range_tiles"] > 0 and info["azimuth_tiles"] > 0
    b.launch()
    b.status()
    for i, (out, r) in enumerate(zip(b.outs, ref)):
        assert np.array_equal(out.cpu().numpy(), r), i
    for i in (0, 3, 4):
        raw, w, o, win = host[i]
        orc = O.sparse_azimuth(O.range_compress(raw, win), w, o)
        got = b.outs[i].cpu().numpy()
        assert np.linalg.norm(got - orc) / np.linalg.norm(orc) < 1e-4, i
    b.close()


@pytest.mark.parametrize("az_tile,interleave,ctas", [(256, 0, 0), (512, 1, 0), (2048, 0, 1), (1024, 1, 2),
                                                      (1024, 2, 0), (512, 3, 1), (1024, 8, 0)])
def test_every_tuning_gives_the_same_bits(rosar, az_tile, interleave, ctas):
    import torch
    scans, _ = _make_scans(torch, seed=1)
    ref = _per_scan_reference(rosar, scans)
    b = rosar.Batch(scans, rosar.Tuning(az_tile=az_tile, interleave=interleave, ctas_per_sm=ctas))
    for _ in range(2):                         # relaunch: the graph resets its counters
        b.launch()
        b.status()
        for i, (out, r) in enumerate(zip(b.outs, ref)):
            assert np.array_equal(out.cpu().numpy(), r), (i, az_tile, interleave)
        for out in b.outs:
            out.zero_()
    b.close()


def test_unmet_dependency_times_out_and_context_survives(rosar):
    """A wait that nothing can satisfy (test hook: one range tile more than exists) gives up after
    its poll limit; the host reads ROSAR_ERR_TIMEOUT and the next batch runs normally."""
    import torch
    scans, _ = _make_scans(torch, seed=2)
    bad = rosar.Batch(scans, rosar.Tuning(spin_limit=20000, debug_unmet_scan=2))
    bad.launch()
    with pytest.raises(rosar.RosarError, match="TIMEOUT"):
        bad.status()
    bad.close()
    ref = _per_scan_reference(rosar, scans)
    good = rosar.Batch(scans)
    good.launch()
    good.status()
    for out, r in zip(good.outs, ref):
        assert np.array_equal(out.cpu().numpy(), r)
    good.close()


def test_full_batched_workload_matches_per_scan(rosar):
    """The 256-scan workload (n_az in {1800, 3600, 7200}, L in {128..1024}, K in {32, 64, 128},
    M = n_az/6) in the launch configuration the benchmark times: bit-exact vs per-scan images."""
    import torch
    cfgs = synth.batched_configs()
    rng = np.random.default_rng(3)
    cubes = {}
    scans = []
    for c in cfgs:
        key = (c.n_az, c.L)
        if key not in cubes:
            cubes[key] = torch.from_numpy(_crand(rng, c.n_az, c.L)).cuda()
        o = synth.draw_offsets(c)
        scans.append({"raw": cubes[key].clone(), "w": torch.from_numpy(synth.default_weights(c, o)).cuda(),
                      "o": torch.from_numpy(o).cuda(), "win": torch.from_numpy(synth.hann_window(c.L)).cuda()})
    b = rosar.Batch(scans)
    b.launch()
    b.status()
    for i in range(0, len(scans), 17):
        s = scans[i]
        ref = rosar.image(s["raw"], s["win"], s["w"], s["o"])
        assert torch.equal(b.outs[i], ref), i
    b.close()


def test_batch_with_fft_plans_equals_image_fft(rosar):
    """Scans given their frequency-domain plan run whole-row FFT azimuth tiles: bit-exact vs
    rosar_image_fft scan by scan (the others keep gather tiles, bit-exact vs rosar_image)."""
    import torch
    scans, host = _make_scans(torch, seed=4)
    ref = []
    for i, s in enumerate(scans):
        n_az = s["raw"].shape[0]
        if rosar.azimuth_fft_supported(n_az) and i % 2 == 0:
            s["H"] = rosar.azimuth_plan(s["w"], s["o"], n_az)
            ref.append(rosar.image_fft(s["raw"], s["win"], s["H"]).cpu().numpy())
        else:
            ref.append(rosar.image(s["raw"], s["win"], s["w"], s["o"]).cpu().numpy())
    assert sum("H" in s for s in scans) >= 3
    D = rosar.batch.DISCARD_S
    for tuning in (rosar.Tuning(), rosar.Tuning(interleave=1, az_tile=512), rosar.Tuning(interleave=2, mix=8, flags=D),
                   rosar.Tuning(interleave=3, mix=32, flags=D), rosar.Tuning(interleave=2, mix=3),
                   rosar.Tuning(interleave=0, flags=D)):
        b = rosar.Batch(scans, tuning)
        b.launch()
        b.status()
        for i, (out, r) in enumerate(zip(b.outs, ref)):
            assert np.array_equal(out.cpu().numpy(), r), i
        b.close()
    raw, w, o, win = host[0]
    orc = O.sparse_azimuth(O.range_compress(raw, win), w, o)
    assert np.linalg.norm(ref[0] - orc) / np.linalg.norm(orc) < 1e-4


@pytest.mark.parametrize("tuning", [dict(), dict(interleave=2, mix=8, flags=2), dict(interleave=3, mix=32, flags=2)])
def test_full_batched_workload_with_plans(rosar, tuning):
    """The 256-scan workload with whole-row FFT tiles in the tile orders and L2 options the autotuner times:
    bit-exact vs rosar_image_fft, twice in a row (S dropped from L2 in the first launch is rewritten)."""
    import torch
    cfgs = synth.batched_configs()
    rng = np.random.default_rng(6)
    cubes = {}
    scans = []
    for c in cfgs:
        key = (c.n_az, c.L)
        if key not in cubes:
            cubes[key] = torch.from_numpy(_crand(rng, c.n_az, c.L)).cuda()
        o = torch.from_numpy(synth.draw_offsets(c)).cuda()
        w = torch.from_numpy(synth.default_weights(c, synth.draw_offsets(c))).cuda()
        scans.append({"raw": cubes[key].clone(), "w": w, "o": o, "H": rosar.azimuth_plan(w, o, c.n_az),
                      "win": torch.from_numpy(synth.hann_window(c.L)).cuda()})
    b = rosar.Batch(scans, rosar.Tuning(**tuning))
    refs = {i: rosar.image_fft(scans[i]["raw"], scans[i]["win"], scans[i]["H"]) for i in range(0, len(scans), 23)}
    for _ in range(2):
        for out in b.outs:
            out.zero_()
        b.launch()
        b.status()
        for i, r in refs.items():
            assert torch.equal(b.outs[i], r), i
    b.close()
