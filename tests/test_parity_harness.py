"""The per-echo comparison that judges every GPU result against the oracle
(oracle/parity.py), checked on the CPU with results whose differences are
planted by hand: an exact copy passes, and each departure from the bar
(waveform L2, a bin, the range, the EPW, the intensity, a missing echo) fails,
while a run edge on a bin inside the guard band around the threshold is
counted as ambiguous instead of failed.

The oracle's own echo extraction (oracle.extract_echoes) supplies the
reference echoes of hand-made waveforms: two Gaussian returns on an ambient
floor."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import parity as PR
from paper_2512_05932_gb300 import scenes as S

T = 1e-5
BAND = 1e-5
MAX_ECHOES = 3


@pytest.fixture(scope="module")
def pulse():
    return S.pulse(1024, 0.1e-9)


@pytest.fixture(scope="module")
def coef(pulse):
    return O.fit_epw(pulse, T)


def waveform(n=1024, bumps=((300.0, 8.0, 4e-5), (620.0, 11.0, 2.5e-5)), floor=1e-6):
    k = np.arange(n, dtype=np.float64)
    xi = np.full(n, floor)
    for c, s, a in bumps:
        xi += a * np.exp(-0.5 * ((k - c) / s) ** 2)
    return xi


def reference(xi, pulse, coef):
    return O.extract_echoes(xi, pulse, T, coef)


def compare(xi_o, ech_o, wave_g, ech_g, n_g=None):
    return PR.compare_beam(xi_o, ech_o, wave_g, ech_g, len(ech_g) if n_g is None else n_g, T, MAX_ECHOES, BAND)


def test_exact_copy_passes(pulse, coef):
    xi = waveform()
    e = reference(xi, pulse, coef)
    assert len(e) == 2
    st, fails = compare(xi, e, xi.astype(np.float32), e.copy())
    assert not fails and st["echoes"] == 2 and st["ambiguous"] == 0 and st["mismatched"] == 0
    assert st["max_l2"] < 1e-7


def test_waveform_l2_beyond_the_bar_fails(pulse, coef):
    xi = waveform()
    e = reference(xi, pulse, coef)
    _, fails = compare(xi, e, xi * 1.002, e.copy())
    assert any("L2" in f for f in fails)
    _, fails = compare(xi, e, xi * 1.0005, e.copy())
    assert not fails


@pytest.mark.parametrize("field, delta, word", [("bin_start", 1, "bins"), ("bin_end", -1, "bins"),
                                                ("bin_peak", 1, "peak bin")])
def test_a_shifted_bin_fails(pulse, coef, field, delta, word):
    xi = waveform()
    e = reference(xi, pulse, coef)
    g = e.copy()
    g[1][field] += delta
    st, fails = compare(xi, e, xi, g)
    assert st["mismatched"] == 1 and any(word in f for f in fails)


def test_range_and_epw_within_a_millimetre(pulse, coef):
    xi = waveform()
    e = reference(xi, pulse, coef)
    g = e.copy()
    g[0]["range_m"] += 0.9e-3
    g[1]["epw_m"] -= 0.9e-3
    assert not compare(xi, e, xi, g)[1]
    g[0]["range_m"] += 0.2e-3
    assert any("range" in f for f in compare(xi, e, xi, g)[1])
    g = e.copy()
    g[1]["epw_m"] += 1.1e-3
    assert any("EPW" in f for f in compare(xi, e, xi, g)[1])


def test_intensity_and_peak_within_1e3(pulse, coef):
    xi = waveform()
    e = reference(xi, pulse, coef)
    g = e.copy()
    g[0]["intensity"] *= 1.0009
    assert not compare(xi, e, xi, g)[1]
    g[0]["intensity"] *= 1.0011 / 1.0009
    assert any("intensity" in f for f in compare(xi, e, xi, g)[1])
    g = e.copy()
    g[1]["peak"] *= 0.998
    assert any("peak" in f for f in compare(xi, e, xi, g)[1])


def test_missing_or_extra_echo_fails(pulse, coef):
    xi = waveform()
    e = reference(xi, pulse, coef)
    _, fails = compare(xi, e, xi, e.copy(), n_g=1)
    assert any("clean echoes" in f for f in fails)
    extra = np.concatenate([e, e[-1:]])
    extra[-1]["bin_start"] += 200
    extra[-1]["bin_end"] += 200
    _, fails = compare(xi, e, xi, extra)
    assert any("clean echoes" in f for f in fails)


def test_run_edge_inside_the_guard_band_is_ambiguous_not_failed(pulse, coef):
    xi = waveform()
    e = reference(xi, pulse, coef)
    # put the first bin of the second run within BAND * T of T: an FP32 result
    # may then start the run one bin later
    k0 = int(e[1]["bin_start"])
    xi_b = xi.copy()
    xi_b[k0] = T * (1.0 + 0.5 * BAND)
    e_b = reference(xi_b, pulse, coef)
    assert int(e_b[1]["bin_start"]) == k0
    g = e_b.copy()
    g[1]["bin_start"] = k0 + 1
    st, fails = compare(xi_b, e_b, xi_b, g)
    assert not fails and st["ambiguous"] == 1
    # the same shift with the bin outside the band is a mismatch
    xi_c = xi.copy()
    xi_c[k0] = T * (1.0 + 3.0 * BAND)
    e_c = reference(xi_c, pulse, coef)
    g = e_c.copy()
    g[1]["bin_start"] = k0 + 1
    st, fails = compare(xi_c, e_c, xi_c, g)
    assert fails and st["ambiguous"] == 0


def test_frame_totals_and_failure_beams(pulse, coef):
    xi = np.stack([waveform(), waveform(bumps=((500.0, 9.0, 3e-5),))])
    ref = {"xi": xi, "echoes": [], "counts": []}
    ech = np.zeros((2, 8), O.ECHO_DTYPE)
    cnt = np.zeros(2, np.int32)
    for b in range(2):
        e = reference(xi[b], pulse, coef)
        ref["echoes"].append(e)
        ref["counts"].append(len(e))
        ech[b, :len(e)] = e
        cnt[b] = len(e)
    ech[1, 0]["bin_end"] += 1
    tot, fails = PR.compare_frame(ref, np.array([0, 1]), xi, ech, cnt, T, MAX_ECHOES, BAND)
    assert tot["beams"] == 2 and tot["echoes"] == 3 and tot["failures"] == 1
    assert fails[0][0] == 1
