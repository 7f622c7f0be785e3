"""Per-echo comparison of a simulated frame with the FP64 oracle.

TEST INFRASTRUCTURE ONLY: used by the tests and by the benchmark's oracle leg
to judge a GPU result against the oracle's. It computes nothing of the beam
model itself; it compares two results of it.

The bar (per beam): waveform relative L2 error <= tol_l2; echo counts and bins
(start, end, peak) bit-exact; range and EPW within 1 mm; intensity and peak
within 1e-3 relative.

Guard band. The echo scan compares each bin with the threshold T strictly
(Sec. II-C); a bin whose oracle value lies within band * T of T may fall on
either side in FP32 arithmetic, which can start, end, split or merge a run.
An echo (of either side) whose run or its two neighbouring bins touch such a
bin is ambiguous: it is left out of the bit-exact comparison and counted.
Clean echoes must appear on both sides in the same order with the same bins;
ambiguous ones may shift which clean echoes fit in the first max_echoes.
"""
from __future__ import annotations

import numpy as np

# oracle echo flags (lidar_oracle.c)
CLIPPED_START, CLIPPED_END, NEAR_THRESHOLD, PEAK_AMBIGUOUS = 1, 2, 4, 8


def _touches(amb, bs, be):
    lo = max(int(bs) - 1, 0)
    return bool(amb[lo:int(be) + 2].any())


class Stats(dict):
    def merge(self, o):
        for k, v in o.items():
            if k.startswith("max_"):
                self[k] = max(self.get(k, 0.0), v)
            else:
                self[k] = self.get(k, 0) + v
        return self


def compare_beam(xi_o, echoes_o, wave_g, echoes_g, count_g, T, max_echoes, band, tol_l2=1e-3):
    """Compares one beam. xi_o: oracle waveform (FP64); echoes_o: every run the
    oracle found, nearest first (structured, oracle ECHO_DTYPE); wave_g: the
    GPU waveform or None (echo-only output); echoes_g / count_g: the GPU's
    echo records and count. Returns (Stats, list of failure strings)."""
    fails = []
    st = Stats(beams=1, echoes=0, ambiguous=0, mismatched=0, max_l2=0.0, max_dr=0.0, max_depw=0.0,
               max_dev_T=0.0)
    if wave_g is not None:
        nrm = np.linalg.norm(xi_o)
        d = np.asarray(wave_g, np.float64) - xi_o
        err = np.linalg.norm(d) / nrm if nrm > 0 else float(np.abs(wave_g).max())
        st["max_l2"] = err
        if err > tol_l2:
            fails.append(f"waveform rel. L2 error {err:.3g}")
        near = np.abs(xi_o - T) <= 0.5 * T
        if near.any():
            st["max_dev_T"] = float(np.abs(d[near]).max() / T)
    amb = np.abs(xi_o - T) <= band * T
    o_amb = [_touches(amb, e["bin_start"], e["bin_end"]) for e in echoes_o]
    n_g = int(count_g)
    g = [echoes_g[i] for i in range(n_g)]
    g_amb = [_touches(amb, e["bin_start"], e["bin_end"]) for e in g]
    clean_o = [e for e, a in zip(echoes_o, o_amb) if not a]
    clean_g = [e for e, a in zip(g, g_amb) if not a]
    n_amb_g = sum(g_amb)
    # echoes the oracle reports in the first max_echoes, ambiguous ones counted
    st["echoes"] = min(len(echoes_o), max_echoes)
    st["ambiguous"] = sum(o_amb[:max_echoes])
    # a GPU echo in the band that overlaps no ambiguous oracle echo (a run
    # started by a bin that the oracle puts at or below T) counts as one more
    o_spans = [(int(e["bin_start"]) - 1, int(e["bin_end"]) + 1) for e, a in zip(echoes_o, o_amb) if a]
    st["ambiguous"] += sum(1 for e, a in zip(g, g_amb)
                           if a and not any(lo <= int(e["bin_end"]) and int(e["bin_start"]) <= hi
                                            for lo, hi in o_spans))
    want = min(len(clean_o), max_echoes - n_amb_g)
    if len(clean_g) != want:
        fails.append(f"{len(clean_g)} clean echoes vs {want} expected ({n_g} GPU echoes, "
                     f"{len(echoes_o)} oracle runs, {n_amb_g} GPU echoes in the band)")
    for i in range(min(len(clean_g), len(clean_o))):
        o, e = clean_o[i], clean_g[i]
        bad = []
        if (int(e["bin_start"]), int(e["bin_end"])) != (int(o["bin_start"]), int(o["bin_end"])):
            bad.append(f"bins {e['bin_start']}..{e['bin_end']} vs {o['bin_start']}..{o['bin_end']}")
        else:
            depw = abs(float(e["epw_m"]) - float(o["epw_m"]))
            st["max_depw"] = max(st["max_depw"], depw)
            if depw > 1e-3:
                bad.append(f"EPW off by {depw:.3g} m")
            if abs(float(e["intensity"]) - float(o["intensity"])) > 1e-3 * abs(float(o["intensity"])):
                bad.append(f"intensity {e['intensity']} vs {o['intensity']}")
            if (int(e["flags"]) & 3) != (int(o["flags"]) & 3):
                bad.append(f"clip flags {e['flags']} vs {o['flags']}")
            if not (int(o["flags"]) & PEAK_AMBIGUOUS):
                dr = abs(float(e["range_m"]) - float(o["range_m"]))
                st["max_dr"] = max(st["max_dr"], dr)
                if int(e["bin_peak"]) != int(o["bin_peak"]):
                    bad.append(f"peak bin {e['bin_peak']} vs {o['bin_peak']}")
                if dr > 1e-3:
                    bad.append(f"range off by {dr:.3g} m")
                if abs(float(e["peak"]) - float(o["peak"])) > 1e-3 * abs(float(o["peak"])):
                    bad.append(f"peak {e['peak']} vs {o['peak']}")
        if bad:
            st["mismatched"] += 1
            fails.append(f"echo {i}: " + "; ".join(bad))
    return st, fails


def compare_frame(ref, beams, wave, echoes, counts, T, max_echoes, band, tol_l2=1e-3):
    """Compares the sampled beams of a frame. ref: oracle.simulate's result for
    `beams` (in that order); wave / echoes / counts: the GPU's full outputs
    (numpy; wave may be None), indexed by beam. Returns (Stats, failures) with
    failures as (beam, message) pairs."""
    tot = Stats()
    fails = []
    for s, b in enumerate(beams):
        n_o = int(ref["counts"][s])
        st, f = compare_beam(ref["xi"][s], ref["echoes"][s][:n_o], None if wave is None else wave[b],
                             echoes[b], counts[b], T, max_echoes, band, tol_l2)
        tot.merge(st)
        fails += [(int(b), m) for m in f]
    tot["failures"] = len(fails)
    return tot, fails
