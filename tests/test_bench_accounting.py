"""Host logic of bench.py that the reported numbers rest on: the bytes counted per pixel, the FP32/SFU
fractions of the BPA kernels, the flat-buffer layout of the batched workload and the stated workload size.
CPU only (no GPU, no library calls)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def test_diff_bytes_per_pixel_match_the_kernels_inputs_and_outputs():
    """Forward: the stacked range compression (raw in, S out: 16), the plan H once per step (8 / 16 scans),
    the filter (S in, image out: 16, + H, + the stored spectrum: 8 when a gradient follows).  Backward: loss
    (image, reference: 16), loss gradient (image, reference in, gradient out: 24), adjoint filter (16 + H + its
    spectrum), weight gradient from the two spectra (16), phase gradient (S and the filter gradient: 16)."""
    fwd, bwd = bench.diff_bytes_per_px(16, True, True, False)
    assert sum(b for _, b in fwd) == pytest.approx(16 + 0.5 + 16.5)
    fwd_g, bwd = bench.diff_bytes_per_px(16, True, True, True)
    assert sum(b for _, b in fwd_g) + sum(b for _, b in bwd) == pytest.approx(137.5)
    # without the fused phase the phase-corrected stack is written and read back (16 more)
    fwd_u, _ = bench.diff_bytes_per_px(16, False, True, True)
    assert sum(b for _, b in fwd_u) - sum(b for _, b in fwd_g) == pytest.approx(16.0)


def test_bpa_fractions():
    """FP32 and SFU fractions from algorithmic work per pixel-pulse, time and the derived peaks."""
    pp = 553e6
    e = bench.bpa_entry(1.0e-3, pp, bench.BPA_FLOPS_ERR, 4, 80.0, 5.0)
    assert e["pixel_pulses_per_s"] == pytest.approx(pp / 1e-3)
    assert e["fp32_tflops"] == pytest.approx(34 * pp / 1e-3 / 1e12)
    assert e["fp32_frac"] == pytest.approx(e["fp32_tflops"] / 80.0)
    assert e["sfu_frac"] == pytest.approx(4 * pp / 1e-3 / 1e12 / 5.0)
    nominal = bench.bpa_entry(0.5e-3, pp, bench.BPA_FLOPS_NOM, 0, 80.0, 5.0)
    assert "sfu_frac" not in nominal and nominal["fp32_tflops"] == pytest.approx(12 * pp / 0.5e-3 / 1e12)


def test_batched_buffers_are_256_byte_aligned_and_disjoint():
    cfgs = synth.batched_configs()
    sizes = [c.L * c.n_az for c in cfgs]
    offs, total = bench._aligned_offsets(sizes)
    assert all(o % 32 == 0 for o in offs)                    # 32 complex64 = 256 bytes
    assert all(offs[i] + sizes[i] <= offs[i + 1] for i in range(len(offs) - 1))
    assert offs[-1] + sizes[-1] <= total < offs[-1] + sizes[-1] + 32


def test_stated_workload_matches_the_configs():
    """The headline's pixel count and shapes as the benchmark line states them."""
    cfgs = synth.batched_configs()
    assert len(cfgs) == 256
    assert sum(c.L * c.n_az for c in cfgs) == 480_844_800
    assert f"{480_844_800:,}" in bench.WORKLOAD
    assert {c.n_az for c in cfgs} <= {1800, 3600, 7200} and {c.L for c in cfgs} <= {128, 256, 512, 1024}


def test_traffic_records_parse():
    """Every committed DRAM-traffic record is (kernel, workload, 16-hex source hash, integer bytes)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    n = 0
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kernel, workload, h, nbytes = line.split()
            int(h, 16)
            assert len(h) == 16 and int(nbytes) > 0
            n += 1
    assert n >= 5
