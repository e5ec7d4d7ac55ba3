"""The C ABI: librosar.so loads, exports every function include/*.h declares, and rejects
bad arguments on the host before any launch (CPU only; no compute call is made)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2309_08038_gb300 import build, _lib
    build.build()
    return _lib.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(rosar_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("rosar_range_compress", "rosar_sparse_azimuth", "rosar_bpa", "rosar_image",
                 "rosar_status_string", "rosar_last_error"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    assert lib.rosar_status_string(0) == b"ROSAR_OK"
    assert lib.rosar_status_string(2) == b"ROSAR_ERR_UNSUPPORTED"
    assert lib.rosar_status_string(99) == b"ROSAR_ERR_UNKNOWN"
    assert lib.rosar_version() >= 100


FAKE = ctypes.c_void_p(0x10000)      # never dereferenced: validation fails first
FAKE2 = ctypes.c_void_p(0x20000000)


def test_range_compress_rejects_bad_arguments(lib):
    assert lib.rosar_range_compress(None, None, 10, 64, 1, FAKE2, None) == 1
    assert lib.rosar_range_compress(FAKE, None, 0, 64, 1, FAKE2, None) == 1
    assert lib.rosar_range_compress(FAKE, None, 10, 48, 1, FAKE2, None) == 2
    assert b"power of two" in lib.rosar_last_error()
    assert lib.rosar_range_compress(FAKE, None, 10, 8192, 1, FAKE2, None) == 2
    assert lib.rosar_range_compress(FAKE, None, 10, 64, 1, FAKE, None) == 1          # in place
    assert lib.rosar_range_compress(ctypes.c_void_p(0x10004), None, 10, 64, 1, FAKE2, None) == 1   # misaligned


def test_sparse_azimuth_rejects_bad_arguments(lib):
    f = lib.rosar_sparse_azimuth
    assert f(FAKE, FAKE, None, 0, 4, 100, 8, FAKE2, None) == 1
    assert f(FAKE, FAKE, FAKE, 0, 4, 100, 0, FAKE2, None) == 1
    assert f(FAKE, FAKE, FAKE, 5, 4, 100, 8, FAKE2, None) == 1          # row stride < K
    assert b"o_row_stride" in lib.rosar_last_error()
    assert f(FAKE, FAKE, FAKE, 0, 4, 100, 8, FAKE, None) == 1           # out aliases S


def test_bpa_rejects_bad_arguments(lib):
    from paper_2309_08038_gb300 import _lib as L
    rad = L.RadarStruct(77e9, 1e14, 1e-7, 8e-6, 0.25, 0.0)
    f = lib.rosar_bpa
    assert f(FAKE, ctypes.byref(rad), None, None, 64, 65, 360, 60, 1, FAKE2, None) == 1      # n_rng > L
    assert f(FAKE, ctypes.byref(rad), None, None, 64, 64, 360, 361, 1, FAKE2, None) == 1     # M_ap > n_az
    assert f(FAKE, ctypes.byref(rad), None, None, 64, 64, 360, 60, 2, FAKE2, None) == 1      # interp
    bad = L.RadarStruct(77e9, 0.0, 1e-7, 8e-6, 0.25, 0.0)
    assert f(FAKE, ctypes.byref(bad), None, None, 64, 64, 360, 60, 1, FAKE2, None) == 1
    assert f(FAKE, None, None, None, 64, 64, 360, 60, 1, FAKE2, None) == 1


def test_time_domain_rejects_bad_arguments(lib):
    from paper_2309_08038_gb300 import _lib as L
    rad = L.RadarStruct(77e9, 1e14, 1e-7, 8e-6, 0.25, 0.0)
    b = lib.rosar_bpa_time
    assert b(FAKE, None, ctypes.byref(rad), 360, 24, 64, 60, FAKE2, None) == 2           # L % 16 != 0
    assert b(FAKE, None, ctypes.byref(rad), 360, 8, 64, 60, FAKE2, None) == 1            # L < 16
    assert b(FAKE, None, ctypes.byref(rad), 360, 64, 64, 361, FAKE2, None) == 1          # M_ap > n_az
    assert b(ctypes.c_void_p(0x10008), None, ctypes.byref(rad), 360, 64, 64, 60, FAKE2, None) == 1   # raw not 16-B
    assert b(FAKE, None, None, 360, 64, 64, 60, FAKE2, None) == 1
    assert b(FAKE, None, ctypes.byref(rad), 360, 64, 64, 60, FAKE, None) == 1            # out aliases raw
    f = lib.rosar_sas_time
    assert f(FAKE, None, FAKE, FAKE, 0, ctypes.byref(rad), 360, 64, 64, 16, 2, FAKE2, None) == 1    # centred
    assert f(FAKE, None, FAKE, FAKE, 5, ctypes.byref(rad), 360, 64, 64, 16, 1, FAKE2, None) == 1    # stride < K
    assert f(FAKE, None, None, FAKE, 0, ctypes.byref(rad), 360, 64, 64, 16, 1, FAKE2, None) == 1
    assert f(FAKE, None, FAKE, FAKE, 0, ctypes.byref(rad), 360, 40, 64, 16, 1, FAKE2, None) == 2    # L % 16
    assert f(FAKE, None, FAKE, FAKE, 0, ctypes.byref(rad), 360, 64, 64, 0, 1, FAKE2, None) == 1     # K = 0


def test_image_fft_host_rejects_bad_arguments(lib):
    f = lib.rosar_image_fft_host
    hr, ho = ctypes.c_void_p(0x70000000), ctypes.c_void_p(0x78000000)
    ws, od = ctypes.c_void_p(0x40000000), ctypes.c_void_p(0x48000000)
    assert f(None, None, FAKE2, 360, 64, FAKE, ws, od, ho, None) == 1          # no host input
    assert f(hr, None, FAKE2, 360, 64, FAKE, ws, od, None, None) == 1          # no host output
    assert f(hr, None, None, 360, 64, FAKE, ws, od, ho, None) == 1             # no plan
    assert f(hr, None, FAKE2, 360, 48, FAKE, ws, od, ho, None) == 2            # L not a power of two
    assert f(hr, None, FAKE2, 7 * 360, 64, FAKE, ws, od, ho, None) == 2        # n_az has a factor 7
    assert f(hr, None, FAKE2, 360, 64, FAKE, ws, ws, ho, None) == 1            # out_dev aliases workspace
    assert f(hr, None, FAKE2, 360, 64, FAKE, ws, od, hr, None) == 1            # host buffers alias


def test_image_fft_scans_rejects_bad_arguments(lib):
    f = lib.rosar_image_fft_scans
    raw, ws, out = ctypes.c_void_p(0x10000000), ctypes.c_void_p(0x40000000), ctypes.c_void_p(0x48000000)
    assert f(raw, None, FAKE2, 0, 360, 64, ws, out, None) == 1                # no scans
    assert f(raw, None, None, 2, 360, 64, ws, out, None) == 1                 # no plan
    assert f(raw, None, FAKE2, 2, 360, 48, ws, out, None) == 2                # L not a power of two
    assert f(raw, None, FAKE2, 2, 7 * 360, 64, ws, out, None) == 2            # n_az has a factor 7
    cube = 360 * 64 * 8
    assert f(raw, None, FAKE2, 2, 360, 64, ctypes.c_void_p(0x10000000 + cube), out, None) == 1   # ws inside raw[1]
    assert f(raw, None, FAKE2, 2, 360, 64, ws, ctypes.c_void_p(0x40000000 + cube), None) == 1    # out inside ws[1]


def test_pipelined_plans_are_the_planner_radices(lib):
    """The multi-scan pipeline covers the compile-time (L, n_az) pairs whose azimuth radices match the
    run-time planner; other shapes fall back to one scan after another (host-side query, no launch)."""
    f = lib.rosar_image_fft_scans_pipelined
    for L, n_az in [(64, 360), (128, 1800), (256, 1800), (128, 3600), (256, 3600), (512, 3600)]:
        assert f(L, n_az) == 1, (L, n_az)
    for L, n_az in [(256, 7200), (64, 3600), (1024, 14400), (48, 360), (256, 0)]:
        assert f(L, n_az) == 0, (L, n_az)


def test_stacked_range_calls_reject_bad_arguments(lib):
    raw, S = ctypes.c_void_p(0x10000000), ctypes.c_void_p(0x40000000)
    for f in (lib.rosar_range_compress_scans, lib.rosar_range_compress_adjoint_scans):
        assert f(raw, None, 0, 360, 64, 1, S, None) == 1                          # no scans
        assert f(raw, None, 65536, 360, 64, 1, S, None) == 1                      # too many scans
        assert f(raw, None, 2, 360, 48, 1, S, None) == 2                          # L not a power of two
        assert f(raw, None, 2, 360, 64, 1, ctypes.c_void_p(0x10000000 + 360 * 64 * 8), None) == 1   # overlap


def test_image_loss_rejects_bad_arguments(lib):
    a, b, ws, out = (ctypes.c_void_p(x) for x in (0x10000000, 0x20000000, 0x30000000, 0x40000000))
    assert lib.rosar_image_l2_loss_workspace_bytes() >= 8
    f, fg = lib.rosar_image_l2_loss, lib.rosar_image_l2_loss_grad
    assert f(None, b, 10, ws, out, None) == 1                                  # no image
    assert f(a, b, 0, ws, out, None) == 1                                      # empty
    assert f(a, b, 10, None, out, None) == 1                                   # no workspace
    assert f(ctypes.c_void_p(0x10000004), b, 10, ws, out, None) == 1           # misaligned
    assert fg(a, b, 10, None, out, None) == 1                                  # no upstream gradient
    assert fg(a, b, -1, out, out, None) == 1                                   # empty
    assert fg(a, b, 10, out, ctypes.c_void_p(0x10000008), None) == 1           # grad partly overlaps out


def test_image_rejects_bad_arguments(lib):
    f = lib.rosar_image
    assert f(FAKE, None, FAKE, FAKE, 0, 100, 60, 8, FAKE2, ctypes.c_void_p(0x40000000), None) == 2
    assert f(FAKE, None, FAKE, FAKE, 0, 100, 64, 8, None, ctypes.c_void_p(0x40000000), None) == 1


def test_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    import paper_2309_08038_gb300 as rosar
    raw = torch.zeros((8, 64), dtype=torch.complex64)
    with pytest.raises(ValueError, match="CUDA"):
        rosar.range_compress(raw)


def test_batch_create_rejects_bad_arguments(lib):
    from paper_2309_08038_gb300 import _lib as L
    ws = ctypes.c_void_p(0x40000000)
    h = ctypes.c_void_p()
    n = lib.rosar_batch_workspace_bytes(2)
    assert n > 0 and lib.rosar_batch_workspace_bytes(0) == 0
    scans = (L.ScanStruct * 2)()
    for s in scans:
        s.raw, s.w, s.o, s.S, s.out = 0x10000, 0x20000, 0x30000, 0x40000, 0x50000
        s.n_az, s.L, s.K = 100, 64, 4
    assert lib.rosar_batch_create(scans, 2, None, ws, n - 1, ctypes.byref(h)) == 1          # workspace too small
    assert lib.rosar_batch_create(scans, 2, None, ctypes.c_void_p(0x40000010), n, ctypes.byref(h)) == 1  # alignment
    scans[1].L = 4096
    assert lib.rosar_batch_create(scans, 2, None, ws, n, ctypes.byref(h)) == 2              # L out of range
    scans[1].L = 64
    scans[0].o = None
    assert lib.rosar_batch_create(scans, 2, None, ws, n, ctypes.byref(h)) == 1              # null offsets
    scans[0].o = 0x30000
    t = L.BatchTuningStruct(300, 0, 0, 0, -1)
    assert lib.rosar_batch_create(scans, 2, ctypes.byref(t), ws, n, ctypes.byref(h)) == 1   # az_tile
    for il in (-1, 9):
        t = L.BatchTuningStruct(1024, 0, il, 0, -1)
        assert lib.rosar_batch_create(scans, 2, ctypes.byref(t), ws, n, ctypes.byref(h)) == 1   # interleave
    t = L.BatchTuningStruct(1024, 0, 2, 0, -1, 33, 0)
    assert lib.rosar_batch_create(scans, 2, ctypes.byref(t), ws, n, ctypes.byref(h)) == 1       # mix > 32
    t = L.BatchTuningStruct(1024, 0, 2, 0, -1, 8, 1)
    assert lib.rosar_batch_create(scans, 2, ctypes.byref(t), ws, n, ctypes.byref(h)) == 1       # unknown flag
    assert h.value is None


def test_migrating_fft_rejects_bad_arguments(lib):
    FAKE3, FAKE4 = ctypes.c_void_p(0x30000000), ctypes.c_void_p(0x40000000)
    p = lib.rosar_azimuth_plan_migrating
    assert p(FAKE, FAKE2, 0, None, 0, 2, 4, 3600, 8, FAKE3, None) == 1            # null dl
    assert p(FAKE, FAKE2, 0, FAKE4, 0, 17, 4, 3600, 8, FAKE3, None) == 1          # n_d > 16
    assert p(FAKE, FAKE2, 0, FAKE4, 0, 0, 4, 3600, 8, FAKE3, None) == 1           # n_d < 1
    assert p(FAKE, FAKE2, 0, FAKE4, 0, 2, 4, 1031, 8, FAKE3, None) == 2           # 1031 has no FFT plan
    f = lib.rosar_sparse_azimuth_migrating_fft
    assert f(FAKE, 8, FAKE2, 0, 2, 8, 3600, None, FAKE4, None) == 1               # null spectrum
    assert f(FAKE, 8, FAKE2, 0, 2, 8, 3600, FAKE, FAKE4, None) == 1               # spectrum aliases S
    assert f(FAKE, 8, FAKE2, 0, 2, 8, 1031, FAKE3, FAKE4, None) == 2              # no FFT plan
    assert b"1031" in lib.rosar_last_error()
    g = lib.rosar_image_migrating_fft
    assert g(FAKE, None, FAKE2, 0, 2, 3600, 48, FAKE3, FAKE4, None) == 2          # L not a power of two


def test_fused_phase_calls_reject_bad_arguments(lib):
    FAKE3 = ctypes.c_void_p(0x30000000)
    assert lib.rosar_phasors(None, 10, FAKE2, None) == 1
    assert lib.rosar_phasors(FAKE, 0, FAKE2, None) == 1
    assert lib.rosar_phasors(FAKE, 10, FAKE, None) == 1                                   # P overlaps eps
    f = lib.rosar_sparse_azimuth_fft_scans_ex
    assert f(FAKE, None, None, 2, 4, 3600, 0, FAKE3, None, None) == 1                    # null H
    assert f(FAKE, None, FAKE2, 2, 4, 3600, 2, FAKE3, None, None) == 1                   # adjoint not 0/1
    assert f(FAKE, None, FAKE2, 2, 4, 3600, 0, FAKE3, FAKE3, None) == 1                  # spectrum aliases out
    assert f(FAKE, FAKE2, FAKE3, 2, 4, 1031, 0, ctypes.c_void_p(0x40000000), None, None) == 2   # no FFT plan
    assert lib.rosar_azimuth_weight_grad_spectra(FAKE, None, FAKE3, 0, 2, 4, 3600, 8, FAKE2, FAKE3, None) == 1
    assert lib.rosar_azimuth_weight_grad_spectra(FAKE, FAKE2, FAKE3, 0, 2, 4, 3600, 8, FAKE, FAKE3, None) == 1  # ws = G
    assert lib.rosar_azimuth_weight_grad_fft_phase(FAKE, FAKE2, None, FAKE3, 0, 2, 4, 3600, 8, FAKE3, None) == 1
    assert lib.rosar_phase_grad_phasor(FAKE, FAKE2, FAKE3, 2, 4, 3600, None, None, None) == 1   # nothing to compute


def test_time_domain_plans_reject_bad_arguments(lib):
    from paper_2309_08038_gb300 import _lib as L
    rad = L.RadarStruct(77e9, 1e14, 1e-7, 8e-6, 0.25, 0.0)
    FAKE3 = ctypes.c_void_p(0x30000000)
    n = lib.rosar_time_domain_plan_bytes(64, 64, 16)
    assert n == 16384 * 1 * 16 * 4 + 8 * 16
    assert lib.rosar_time_domain_plan_bytes(65, 32, 3) == 16384 * 2 * 3 * 2 + 32
    assert lib.rosar_sas_time_plan(None, FAKE, FAKE2, ctypes.byref(rad), 360, 64, 64, 16, 1, FAKE3, n - 1, None) == 1
    assert lib.rosar_sas_time_plan(None, FAKE, FAKE2, ctypes.byref(rad), 360, 48 + 2, 64, 16, 1, FAKE3, n, None) == 2
    assert lib.rosar_sas_time_plan(None, FAKE, FAKE2, ctypes.byref(rad), 360, 64, 64, 16, 1, ctypes.c_void_p(0x30000008),
                                   n, None) == 1                                        # plan not 16-byte aligned
    assert lib.rosar_bpa_time_plan(None, ctypes.byref(rad), 360, 64, 64, 361, FAKE3,
                                   lib.rosar_time_domain_plan_bytes(64, 64, 361), None) == 1   # M_ap > n_az
    assert lib.rosar_sas_time_planned(FAKE, None, 360, 64, 64, 16, FAKE2, None) == 1            # null plan
    assert lib.rosar_sas_time_planned(ctypes.c_void_p(0x10000008), FAKE3, 360, 64, 64, 16, FAKE2, None) == 1  # raw
    assert lib.rosar_sas_time_planned(FAKE, FAKE3, 360, 40, 64, 16, FAKE2, None) == 2            # L % 16
    assert lib.rosar_bpa_time_planned(FAKE, FAKE3, 360, 64, 64, 60, FAKE, None) == 1            # out aliases raw
