"""Differentiable form: adjoint kernels and autograd against the FP64 oracle and finite differences (GPU).

Bar: gradients within 1e-3 relative error of the FP64 reference (they land near 1e-6).
"""

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3


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


def _cuda(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_phase_apply_and_adjoints_match_oracle(rosar):
    import torch
    rng = np.random.default_rng(1)
    n_scans, n_rng, n_az, K, M = 3, 9, 1031, 40, 300
    S = _c(rng, n_scans, n_rng, n_az)
    eps = (rng.standard_normal((n_scans, n_az)) * 0.3).astype(np.float32)
    w = _c(rng, n_rng, K)
    o = (np.sort(rng.choice(M, K, replace=False)) - M // 2).astype(np.int32)
    g = _c(rng, n_scans, n_rng, n_az)
    S_t = rosar.phase_apply(_cuda(torch, S), _cuda(torch, eps))
    out = rosar.sparse_azimuth_scans(S_t, _cuda(torch, w), _cuda(torch, o)).cpu().numpy()
    gS, gw = rosar.sparse_azimuth_adjoint(_cuda(torch, g), S_t, _cuda(torch, w), _cuda(torch, o))
    ge, gSraw = rosar.phase_grad(S_t, gS, _cuda(torch, eps), want_eps=True, want_S=True)
    S_t = S_t.cpu().numpy()
    ref_gw = np.zeros((n_rng, K), np.complex128)
    for s in range(n_scans):
        ref_t = O.apply_phase_errors(S[s], eps[s])
        assert _rel(S_t[s], ref_t) < 1e-6
        assert _rel(out[s], O.sparse_azimuth(ref_t, w, o)) < 1e-5
        ref_gS = O.sparse_azimuth_adjoint_S(g[s], w, o)
        assert _rel(gS[s].cpu().numpy(), ref_gS) < 1e-5
        assert _rel(ge[s].cpu().numpy(), O.phase_error_grad(ref_t, ref_gS)) < 1e-5
        assert _rel(gSraw[s].cpu().numpy(), ref_gS * np.exp(-1j * eps[s].astype(np.float64))[None, :]) < 1e-5
        ref_gw += O.sparse_azimuth_adjoint_w(g[s], ref_t, o)
    assert _rel(gw.cpu().numpy(), ref_gw) < 1e-5


def test_weight_grad_wide_span_and_per_row_offsets(rosar):
    """Offsets spanning more than the staged window (direct-gather path) and per-row offsets."""
    import torch
    rng = np.random.default_rng(2)
    n_rng, n_az, K = 4, 9000, 12
    o = np.stack([np.sort(rng.choice(np.arange(-4400, 4400), K, replace=False)) for _ in range(n_rng)]).astype(np.int32)
    S, g, w = _c(rng, 1, n_rng, n_az), _c(rng, 1, n_rng, n_az), _c(rng, n_rng, K)
    gS, gw = rosar.sparse_azimuth_adjoint(_cuda(torch, g), _cuda(torch, S), _cuda(torch, w), _cuda(torch, o))
    assert _rel(gw.cpu().numpy(), O.sparse_azimuth_adjoint_w(g[0], S[0], o)) < 1e-5
    assert _rel(gS[0].cpu().numpy(), O.sparse_azimuth_adjoint_S(g[0], w, o)) < 1e-5


@pytest.mark.parametrize("L,n_az", [(8, 37), (64, 360), (256, 100), (1024, 33), (4096, 5)])
def test_range_compress_adjoint_matches_oracle(rosar, L, n_az):
    import torch
    rng = np.random.default_rng(L)
    g = _c(rng, L, n_az)
    win = synth.hann_window(L)
    for centred in (True, False):
        got = rosar.range_compress_adjoint(_cuda(torch, g), _cuda(torch, win), centred=centred).cpu().numpy()
        assert _rel(got, O.range_compress_adjoint(g, win, centred)) < 2e-6, (L, n_az, centred)


@pytest.mark.parametrize("L,n_az,n_scans", [(64, 360, 3), (256, 3600, 2), (16, 37, 5)])
def test_stacked_range_calls_equal_per_scan_calls(rosar, L, n_az, n_scans):
    """rosar_range_compress_scans / rosar_range_compress_adjoint_scans (one launch, grid.y = scan) give each scan
    the bits of its own single-scan call, with and without centring."""
    import torch
    rng = np.random.default_rng(L + n_scans)
    raw, g = _cuda(torch, _c(rng, n_scans, n_az, L)), _cuda(torch, _c(rng, n_scans, L, n_az))
    win = _cuda(torch, synth.hann_window(L))
    for centred in (True, False):
        S = rosar.range_compress(raw, win, centred=centred)
        gr = rosar.range_compress_adjoint(g, win, centred=centred)
        for s in range(n_scans):
            assert torch.equal(S[s], rosar.range_compress(raw[s], win, centred=centred)), (s, centred)
            assert torch.equal(gr[s], rosar.range_compress_adjoint(g[s], win, centred=centred)), (s, centred)


def test_range_compress_autograd_stack(rosar):
    import torch
    rng = np.random.default_rng(41)
    n_scans, n_az, L = 3, 50, 64
    raw = _c(rng, n_scans, n_az, L)
    B = _c(rng, n_scans, L, n_az)
    win = synth.hann_window(L)
    t = _cuda(torch, raw).requires_grad_(True)
    S = rosar.autograd.range_compress(t, _cuda(torch, win))
    torch.sum(torch.abs(S - _cuda(torch, B)) ** 2).backward()
    for s in range(n_scans):
        ref = O.range_compress_adjoint(2.0 * (O.range_compress(raw[s], win) - B[s]), win)
        assert _rel(t.grad[s].cpu().numpy(), ref) < 1e-5, s


@pytest.mark.parametrize("shape", [(1,), (7,), (3, 257), (16, 256, 3600)])
def test_image_l2_loss_and_gradient(rosar, shape):
    """rosar_image_l2_loss against the FP64 sum of |out - ref|^2 (ragged sizes down to one element and the
    differentiable workload's 16-scan stack), bit-identical on repeated calls; the autograd gradient against
    2 g (out - ref), and ref's gradient its negative."""
    import torch
    rng = np.random.default_rng(len(shape) + shape[-1])
    out, ref = _c(rng, *shape), _c(rng, *shape)
    to, tr = _cuda(torch, out), _cuda(torch, ref)
    loss = rosar.image_l2_loss(to, tr)
    exact = float(np.sum(np.abs(out.astype(np.complex128) - ref.astype(np.complex128)) ** 2))
    assert abs(loss.item() - exact) <= 1e-6 * exact
    assert torch.equal(loss, rosar.image_l2_loss(to, tr))
    a = to.clone().requires_grad_(True)
    b = tr.clone().requires_grad_(True)
    l2 = rosar.autograd.image_l2_loss(a, b)
    (3.0 * l2).backward()
    d = (out.astype(np.complex128) - ref.astype(np.complex128)) * 6.0
    assert _rel(a.grad.cpu().numpy(), d) < 1e-6
    assert torch.equal(b.grad, -a.grad)


def _crop_problem(seed=3):
    """The 64-pulse crop: 64 pulses, 32 range rows, K = 16 taps of M = 32, two scans."""
    rng = np.random.default_rng(seed)
    n_scans, n_rng, n_az, K, M = 2, 32, 64, 16, 32
    S = _c(rng, n_scans, n_rng, n_az)
    B = _c(rng, n_scans, n_rng, n_az)
    w = (_c(rng, n_rng, K) / 4).astype(np.complex64)
    o = (np.sort(rng.choice(M, K, replace=False)) - M // 2).astype(np.int32)
    eps = (rng.standard_normal((n_scans, n_az)) * 0.3).astype(np.float32)
    return S, B, w, o, eps


def _oracle_loss(S, B, w, o, eps):
    return float(sum(np.sum(np.abs(O.sparse_azimuth(O.apply_phase_errors(S[s], eps[s]), w, o) - B[s]) ** 2)
                     for s in range(S.shape[0])))


@pytest.mark.parametrize("method", ["gather", "fft"])
def test_autograd_matches_fp64_finite_differences_on_crop(rosar, method):
    import torch
    S, B, w, o, eps = _crop_problem()
    tS = _cuda(torch, S).requires_grad_(True)
    te = _cuda(torch, eps).requires_grad_(True)
    tw = _cuda(torch, w).requires_grad_(True)
    out = rosar.autograd.sparse_azimuth_phase(tS, te, tw, _cuda(torch, o), method=method)
    loss = torch.sum(torch.abs(out - _cuda(torch, B)) ** 2)
    loss.backward()
    # FP64 oracle gradients
    ref_w = np.zeros_like(w, dtype=np.complex128)
    ref_e = np.zeros_like(eps, dtype=np.float64)
    ref_S = np.zeros_like(S, dtype=np.complex128)
    for s in range(S.shape[0]):
        St = O.apply_phase_errors(S[s], eps[s])
        gr = 2.0 * (O.sparse_azimuth(St, w, o) - B[s])
        G = O.sparse_azimuth_adjoint_S(gr, w, o)
        ref_w += O.sparse_azimuth_adjoint_w(gr, St, o)
        ref_e[s] = O.phase_error_grad(St, G)
        ref_S[s] = G * np.exp(-1j * eps[s].astype(np.float64))[None, :]
    assert _rel(tw.grad.cpu().numpy(), ref_w) < TOL_GRAD
    assert _rel(te.grad.cpu().numpy(), ref_e) < TOL_GRAD
    assert _rel(tS.grad.cpu().numpy(), ref_S) < TOL_GRAD
    # FP64 central differences of the loss (h = 1e-6) on sampled coordinates
    S64, B64, w64, e64 = S.astype(np.complex128), B.astype(np.complex128), w.astype(np.complex128), eps.astype(np.float64)
    h = 1e-6
    for (s, n) in [(0, 0), (0, 17), (1, 40), (1, 63)]:
        ep, em = e64.copy(), e64.copy()
        ep[s, n] += h
        em[s, n] -= h
        fd = (_oracle_loss(S64, B64, w64, o, ep) - _oracle_loss(S64, B64, w64, o, em)) / (2 * h)
        assert abs(te.grad[s, n].item() - fd) <= TOL_GRAD * max(abs(fd), np.abs(ref_e).max() * 1e-2)
    for (r, k) in [(0, 0), (5, 7), (31, 15)]:
        fd = 0j
        for part, dz in enumerate((1.0, 1j)):
            wp, wm = w64.copy(), w64.copy()
            wp[r, k] += h * dz
            wm[r, k] -= h * dz
            fd += (1 if part == 0 else 1j) * (_oracle_loss(S64, B64, wp, o, e64) - _oracle_loss(S64, B64, wm, o, e64)) / (2 * h)
        assert abs(complex(tw.grad[r, k].item()) - fd) <= TOL_GRAD * max(abs(fd), np.abs(ref_w).max() * 1e-2)


def test_range_compress_autograd(rosar):
    import torch
    rng = np.random.default_rng(4)
    n_az, L = 50, 64
    raw = _c(rng, n_az, L)
    B = _c(rng, L, n_az)
    win = synth.hann_window(L)
    t = _cuda(torch, raw).requires_grad_(True)
    S = rosar.autograd.range_compress(t, _cuda(torch, win))
    torch.sum(torch.abs(S - _cuda(torch, B)) ** 2).backward()
    ref = O.range_compress_adjoint(2.0 * (O.range_compress(raw, win) - B), win)
    assert _rel(t.grad.cpu().numpy(), ref) < 1e-5


@pytest.mark.parametrize("method", ["gather", "fft"])
def test_full_diff_workload_against_oracle(rosar, method):
    """16 indoor-geometry scans, shared w [256, 64], eps [16, 3600]: grad w and grad eps of
    ||image - reference||^2 in the launch configurations the benchmark times, vs the FP64 oracle."""
    import torch
    cfg = synth.INDOOR
    rng = np.random.default_rng(5)
    n_scans = 16
    S = _c(rng, n_scans, cfg.L, cfg.n_az)
    Bref = _c(rng, n_scans, cfg.L, cfg.n_az)
    o = synth.draw_offsets(cfg)
    w = synth.default_weights(cfg, o)
    eps = (rng.standard_normal((n_scans, cfg.n_az)) * 0.3).astype(np.float32)
    tw = _cuda(torch, w).requires_grad_(True)
    te = _cuda(torch, eps).requires_grad_(True)
    out = rosar.autograd.sparse_azimuth_phase(_cuda(torch, S), te, tw, _cuda(torch, o), method=method)
    torch.sum(torch.abs(out - _cuda(torch, Bref)) ** 2).backward()
    gw = tw.grad.cpu().numpy()
    ge = te.grad.cpu().numpy()
    ref_w = np.zeros((cfg.L, cfg.K), np.complex128)
    for s in range(n_scans):
        St = O.apply_phase_errors(S[s], eps[s])
        gr = 2.0 * (O.sparse_azimuth(St, w, o) - Bref[s])
        ref_w += O.sparse_azimuth_adjoint_w(gr, St, o)
        if s in (0, 15):
            assert _rel(ge[s], O.phase_error_grad(St, O.sparse_azimuth_adjoint_S(gr, w, o))) < TOL_GRAD
    assert _rel(gw, ref_w) < TOL_GRAD


@pytest.mark.parametrize("n_az,per_row,n_scans", [(48, False, 3), (1000, True, 3), (3600, False, 3), (7200, True, 3),
                                                  (3600, False, 1), (3600, True, 9), (1800, True, 6), (360, False, 16)])
def test_frequency_domain_adjoints_match_oracle(rosar, n_az, per_row, n_scans):
    """Stacked FFT filter (plan shared by the scans), its adjoint (conj of the plan) and the cross-spectrum
    weight gradient against the oracle's filter and adjoints; shared and per-row offsets, wrapping offsets.
    360/1800/3600-pulse rows take the cluster-split weight gradient (1, 2 or 4 CTAs per row by scan count)."""
    import torch
    rng = np.random.default_rng(n_az + n_scans)
    n_rng, K = 5, 12
    M = min(n_az, 600)
    if per_row:
        o = np.stack([np.sort(rng.choice(M, K, replace=False)) - M // 2 for _ in range(n_rng)]).astype(np.int32)
        o[1, 0] -= 3 * n_az
    else:
        o = (np.sort(rng.choice(M, K, replace=False)) - M // 2).astype(np.int32)
    S, g = _c(rng, n_scans, n_rng, n_az), _c(rng, n_scans, n_rng, n_az)
    w = _c(rng, n_rng, K)
    tw, to = _cuda(torch, w), _cuda(torch, o)
    H = rosar.azimuth_plan(tw, to, n_az)
    out = rosar.sparse_azimuth_fft_scans(_cuda(torch, S), H).cpu().numpy()
    adj = rosar.sparse_azimuth_fft_scans(_cuda(torch, g), H, adjoint=True).cpu().numpy()
    gw = rosar.azimuth_weight_grad_fft(_cuda(torch, g), _cuda(torch, S), to, K).cpu().numpy()
    ref_w = np.zeros((n_rng, K), np.complex128)
    for s in range(n_scans):
        assert _rel(out[s], O.sparse_azimuth(S[s], w, o)) < 1e-5
        assert _rel(adj[s], O.sparse_azimuth_adjoint_S(g[s], w, o)) < 1e-5
        ref_w += O.sparse_azimuth_adjoint_w(g[s], S[s], o)
    assert _rel(gw, ref_w) < 1e-5


@pytest.mark.parametrize("n_az,per_row,n_scans", [(3600, False, 16), (1800, True, 3), (1000, False, 2), (360, True, 5)])
def test_phase_fused_kernels_equal_the_materialized_path(rosar, n_az, per_row, n_scans):
    """The frequency-domain step without S_t in memory (phase factors applied as S is loaded) gives the same bits
    as rosar_phase_apply followed by the filter, the weight gradient and the phase gradient on S_t; and matches the
    oracle (compile-time plans 3600/1800/360 and the run-time plan of 1000 pulses)."""
    import torch
    rng = np.random.default_rng(n_az + 7)
    n_rng, K = 5, 12
    M = min(n_az, 600)
    if per_row:
        o = np.stack([np.sort(rng.choice(M, K, replace=False)) - M // 2 for _ in range(n_rng)]).astype(np.int32)
    else:
        o = (np.sort(rng.choice(M, K, replace=False)) - M // 2).astype(np.int32)
    S, g, w = _c(rng, n_scans, n_rng, n_az), _c(rng, n_scans, n_rng, n_az), _c(rng, n_rng, K)
    eps = (rng.standard_normal((n_scans, n_az)) * 0.3).astype(np.float32)
    tS, tg, tw, to, te = (_cuda(torch, x) for x in (S, g, w, o, eps))
    H = rosar.azimuth_plan(tw, to, n_az)
    P = rosar.phasors(te)
    S_t = rosar.phase_apply(tS, te)
    X, G = torch.empty_like(tS), torch.empty_like(tS)
    out = rosar.sparse_azimuth_fft_scans_ex(tS, H, P=P, spectrum=X)
    assert torch.equal(out, rosar.sparse_azimuth_fft_scans(S_t, H))
    adj = rosar.sparse_azimuth_fft_scans_ex(tg, H, adjoint=True, spectrum=G)
    assert torch.equal(adj, rosar.sparse_azimuth_fft_scans(tg, H, adjoint=True))
    assert torch.equal(rosar.azimuth_weight_grad_fft_phase(tg, tS, P, to, K), rosar.azimuth_weight_grad_fft(tg, S_t, to, K))
    ge1, gs1 = rosar.phase_grad_phasor(tS, P, tg, want_eps=True, want_S=True)
    ge0, gs0 = rosar.phase_grad(S_t, tg, te, want_eps=True, want_S=True)
    assert torch.equal(ge1, ge0) and torch.equal(gs1, gs0)
    out = out.cpu().numpy()
    ref_w = np.zeros((n_rng, K), np.complex128)
    for s in range(n_scans):
        St = O.apply_phase_errors(S[s], eps[s])
        assert _rel(out[s], O.sparse_azimuth(St, w, o)) < 1e-5
        ref_w += O.sparse_azimuth_adjoint_w(g[s], St, o)
    # the weight gradient from the two calls' stored spectra
    assert _rel(rosar.azimuth_weight_grad_spectra(G, X, to, K).cpu().numpy(), ref_w) < 1e-5


def test_differentiable_step_replays_from_a_cuda_graph(rosar):
    """Forward, image loss and backward of the frequency-domain form captured in one CUDA graph: every replay
    gives the eager step's loss and gradients bit for bit (the benchmark times the step this way too)."""
    import torch
    rng = np.random.default_rng(21)
    n_scans, n_rng, n_az, K = 3, 16, 3600, 24
    S = _cuda(torch, _c(rng, n_scans, n_rng, n_az))
    B = _cuda(torch, _c(rng, n_scans, n_rng, n_az))
    o = _cuda(torch, (np.sort(rng.choice(600, K, replace=False)) - 300).astype(np.int32))
    w = _cuda(torch, _c(rng, n_rng, K)).requires_grad_(True)
    eps = _cuda(torch, (rng.standard_normal((n_scans, n_az)) * 0.3).astype(np.float32)).requires_grad_(True)

    def step():
        loss = rosar.autograd.image_l2_loss(rosar.autograd.sparse_azimuth_phase(S, eps, w, o, method="fft"), B)
        loss.backward()
        return loss

    ref_loss = step().detach().clone()
    ref_w, ref_e = w.grad.clone(), eps.grad.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        w.grad = eps.grad = None
        step()
    torch.cuda.current_stream().wait_stream(side)
    w.grad = eps.grad = None
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        loss = step()
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(loss, ref_loss)
        assert torch.equal(w.grad, ref_w) and torch.equal(eps.grad, ref_e)
