"""The autotuner picks a valid choice, caches it, and the tuned launches give the same images (GPU)."""

import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rosar(tmp_path_factory):
    from paper_2309_08038_gb300 import build
    build.build()
    os.environ["ROSAR_AUTOTUNE_CACHE"] = str(tmp_path_factory.mktemp("tune") / "autotune.json")
    import paper_2309_08038_gb300 as r
    return r


def test_choose_azimuth_and_cache(rosar):
    res = rosar.autotune.choose_azimuth(256, 3600, 64, reps=5)
    assert res["path"] in ("fft", "gather") and set(res["us"]) == {"fft", "gather"}
    assert res["us"][res["path"]] == min(res["us"].values())
    assert rosar.autotune.choose_azimuth(256, 3600, 64) == res            # served from the cache
    with open(os.environ["ROSAR_AUTOTUNE_CACHE"]) as f:
        assert any(k.startswith("azimuth/") for k in json.load(f))
    assert rosar.autotune.choose_azimuth(8, 1031, 16, reps=3)["path"] == "gather"   # no FFT plan for 1031


def test_tuned_batch_gives_the_same_images(rosar):
    import torch
    rng = np.random.default_rng(0)
    scans = []
    for n_az, L, K in [(1800, 128, 32), (3600, 256, 64), (7200, 128, 128), (1031, 64, 16)]:
        raw = (rng.standard_normal((n_az, L)) + 1j * rng.standard_normal((n_az, L))).astype(np.complex64)
        o = (np.sort(rng.choice(n_az // 6, K, replace=False)) - n_az // 12).astype(np.int32)
        w = (rng.standard_normal((L, K)) + 1j * rng.standard_normal((L, K))).astype(np.complex64)
        sc = {"raw": torch.from_numpy(raw).cuda(), "w": torch.from_numpy(w).cuda(), "o": torch.from_numpy(o).cuda(),
              "win": torch.from_numpy(synth.hann_window(L)).cuda()}
        if rosar.azimuth_fft_supported(n_az):
            sc["H"] = rosar.azimuth_plan(sc["w"], sc["o"], n_az)
        scans.append(sc)
    res = rosar.autotune.tune_batch(scans, reps=2)
    assert len(res["ms"]) == len(rosar.autotune.batch_candidates(fft_tiles=False))   # one scan has no plan
    b = rosar.Batch(scans, res["tuning"])
    b.launch()
    b.status()
    for sc, out in zip(scans, b.outs):
        ref = (rosar.image_fft(sc["raw"], sc["win"], sc["H"]) if "H" in sc
               else rosar.image(sc["raw"], sc["win"], sc["w"], sc["o"]))
        assert torch.equal(out, ref)
    b.close()
    assert rosar.autotune.tune_batch(scans)["cached"]
