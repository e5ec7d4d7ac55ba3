"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a scratch copy of the oracle: a flipped sign, a dropped factor, an off-by-one
index, a conjugate in the wrong place, a wrong reference sample. It then runs the pin suite
(test_oracle_pins.py) against that copy, which must fail. The repository's oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle", "rosar_oracle.py")

AZ_TAIL = "    return out\n\n\ndef sparse_azimuth_migrating"

# name: (text in the oracle, the mistake planted in its place)
MISTAKES = {
    # range compression, Eq. (38) and the centring reading
    "centring_sign": ("Y = Y * np.exp(1j * math.pi", "Y = Y * np.exp(-1j * math.pi"),
    "window_dropped": ("Y = (raw * win[None, :]) @ F.T", "Y = raw @ F.T"),
    "dft_sign": ("F = np.exp(-2j * math.pi * (np.outer(l", "F = np.exp(2j * math.pi * (np.outer(l"),
    # sparse azimuth filter, Eq. (43)
    "offset_sign": ("out[r] += w[r, k] * S[r, (theta + o[r, k]) % n_az]\n" + AZ_TAIL,
                    "out[r] += w[r, k] * S[r, (theta - o[r, k]) % n_az]\n" + AZ_TAIL),
    "weight_conjugated": ("out[r] += w[r, k] * S[r, (theta + o[r, k]) % n_az]\n" + AZ_TAIL,
                          "out[r] += np.conj(w[r, k]) * S[r, (theta + o[r, k]) % n_az]\n" + AZ_TAIL),
    "migration_row_sign": ("row = r + dl[r, k]", "row = r - dl[r, k]"),
    # FFT+BPA, Sec. III-D with w_BP and Eq. (37)
    "bpa_phase_sign": ("return np.sum(alpha * np.exp(-2j * k_mid * R_n) * s, axis=1)",
                       "return np.sum(alpha * np.exp(2j * k_mid * R_n) * s, axis=1)"),
    "nearest_is_floor": ("np.floor(x + 0.5).astype(np.int64), n)", "np.floor(x).astype(np.int64), n)"),
    "interp_weights_swapped": ("s = (1.0 - f) * s0 + f * s1", "s = f * s0 + (1.0 - f) * s1"),
    "interp_off_by_one": ("s1 = _read_bins(S, l0 + 1, n)", "s1 = _read_bins(S, l0 + 2, n)"),
    "rotation_error_sign": ("phi_n = phi_n + np.asarray(dphi", "phi_n = phi_n - np.asarray(dphi"),
    "radius_error_sign": ("r_n = r_n + np.asarray(dr", "r_n = r_n - np.asarray(dr"),
    # time-domain forms, Eq. (14) and Algorithm 2
    "fast_time_sign": ("return win * np.exp(-2j * math.pi * (tau", "return win * np.exp(2j * math.pi * (tau"),
    "bpa_time_reference_sample": ("_fast_time_compensation(radar, R_n, win, L, 0.0)",
                                  "_fast_time_compensation(radar, R_n, win, L, 1.0)"),
    "sas_centre_sample": ("    m_ref = (L - 1) / 2.0 if centred else 0.0\n    rows",
                          "    m_ref = L / 2.0 if centred else 0.0\n    rows"),
    # default weights (Eq. (16), Taylor taper)
    "taper_centre": ("x = (np.arange(M, dtype=np.float64) - (M - 1) / 2.0) / M",
                     "x = (np.arange(M, dtype=np.float64) - M / 2.0) / M"),
    "steering_sign": ("a = p * np.exp(2j * k_mid * rho)", "a = p * np.exp(-2j * k_mid * rho)"),
    # adjoints of the differentiable form
    "adjoint_S_offset": ("g[r, (n - o[r, k]) % n_az]", "g[r, (n + o[r, k]) % n_az]"),
    "adjoint_w_conjugate": ("out[r, k] = np.sum(g[r] * np.conj(S[r, (th + o[r, k]) % n_az]))",
                            "out[r, k] = np.sum(np.conj(g[r]) * S[r, (th + o[r, k]) % n_az])"),
    "phase_grad_sign": ("return np.sum(np.imag(np.conj(np.asarray(S_tilde))",
                        "return -np.sum(np.imag(np.conj(np.asarray(S_tilde))"),
    "range_adjoint_centring": ("g = g * np.exp(-1j * math.pi * l * (L - 1) / L)[:, None]",
                               "g = g * np.exp(1j * math.pi * l * (L - 1) / L)[:, None]"),
    # image metrics, Eqs. (44), (45)
    "entropy_base": ("return float(-np.sum(d * np.log(d)))", "return float(-np.sum(d * np.log2(d)))"),
    "pisr_power": ("return float(np.abs(I_row[main_idx]) ** 2 / np.sum(np.abs(I_row[np.asarray(side_idx)]) ** 2))",
                   "return float(np.abs(I_row[main_idx]) / np.sum(np.abs(I_row[np.asarray(side_idx)])))"),
}


@pytest.fixture(scope="module")
def scratch(tmp_path_factory):
    """A scratch tree with the oracle package and the pin suite (its golden files and conftest)."""
    root = tmp_path_factory.mktemp("oracle_mutations")
    shutil.copytree(os.path.join(ROOT, "oracle"), root / "oracle",
                    ignore=shutil.ignore_patterns("__pycache__", "*.so", "lib"))
    (root / "tests").mkdir()
    for name in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", name), root / "tests" / name)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), root / "tests" / "golden")
    return root


def _pins(root):
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           "tests/test_oracle_pins.py"], cwd=root, capture_output=True, text=True, timeout=600)


def test_pins_pass_on_the_unmodified_copy(scratch):
    r = _pins(scratch)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_planted_mistake_fails_a_pin(scratch, name):
    text, wrong = MISTAKES[name]
    with open(ORACLE) as f:
        src = f.read()
    assert src.count(text) == 1, f"{name}: the text to replace must occur once in the oracle"
    target = scratch / "oracle" / "rosar_oracle.py"
    try:
        target.write_text(src.replace(text, wrong))
        r = _pins(scratch)
    finally:
        target.write_text(src)
    assert r.returncode != 0, f"{name}: no pin failed\n{r.stdout[-1500:]}"
