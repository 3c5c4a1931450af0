"""Mutation test of the oracle pins.

Each case plants one plausible mistake in a copy of ``oracle/hp_oracle.c`` (a
wrong rounding, a dropped term, an off-by-one, a flipped comparison), builds
it on the CPU and runs the pin suite against it: every mutant must make at
least one pin fail.  The mistakes are planted only in the oracle, never in
the CUDA library.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hp_oracle.c")

MUTANTS = {
    "delay_floor": ("(int32_t)rint(sec / tsamp)", "(int32_t)floor(sec / tsamp)"),
    "delay_ref_infinity": ("(1.0 / (f * f) - inv_top2)", "(1.0 / (f * f))"),
    "delay_half_channel": ("double f = f_top + (double)c * chan_bw;",
                           "double f = f_top + ((double)c + 0.5) * chan_bw;"),
    "dedisp_drop_channel": ("for (int c = 0; c < nchans; ++c) {\n                    int64_t row",
                            "for (int c = 0; c < nchans - 1; ++c) {\n                    int64_t row"),
    "dedisp_shift": ("int64_t row = t + dl[c];", "int64_t row = t + dl[c] + (c & 1);"),
    "remedian_upper": ("return s[(r - 1) / 2];", "return s[r / 2];"),
    "baseline_trunc": ("b[t] = m[j] + floor_div((m[j + 1] - m[j]) * (t - cj), P);",
                       "b[t] = m[j] + ((m[j + 1] - m[j]) * (t - cj)) / P;"),
    "baseline_centre": ("int64_t half = (P - 1) / 2;", "int64_t half = 0;"),
    "baseline_mean_count": ("b[t] = floor_div(pre[hi + 1] - pre[lo], hi - lo + 1);",
                            "b[t] = floor_div(pre[hi + 1] - pre[lo], hi - lo + 2);"),
    "mad_upper": ("int64_t v = a[(n - 1) / 2];", "int64_t v = a[n / 2];"),
    "sigma_factor": ("HPO_MAD_TO_SIGMA = 1.482602218505602;", "HPO_MAD_TO_SIGMA = 1.0;"),
    "thr_strict": ("if ((double)S >= lim) {", "if ((double)S > lim) {"),
    "peak_last_tie": ("if (S2 > best_S) { best_S = S2; best_t = t; }",
                      "if (S2 >= best_S) { best_S = S2; best_t = t; }"),
    "snr_no_sqrt": (": (double)best_S / (sigma * sw);", ": (double)best_S / sigma;"),
    "window_short": ("int64_t S = P[t + W] - P[t];", "int64_t S = P[t + W - 1] - P[t];"),
    "merge_gap_strict": ("if (gap <= t_gap) uf_union(parent, i, j);",
                         "if (gap < t_gap) uf_union(parent, i, j);"),
    "merge_dm_tol": ("c[j].dm_idx <= c[i].dm_idx + dm_tol;", "c[j].dm_idx < c[i].dm_idx + dm_tol;"),
    "merge_rep_last_tie": ("if (c[i].snr > o->snr) {", "if (c[i].snr >= o->snr) {"),
    "merge_t_hi": ("if (e > o->t_hi) o->t_hi = e;", "if (c[i].sample > o->t_hi) o->t_hi = c[i].sample;"),
    "raw_snr_no_sqrt": ("c[i].snr = (double)c[i].S / (sigma[c[i].dm_idx] * sw);",
                        "c[i].snr = (double)c[i].S / sigma[c[i].dm_idx];"),
    "raw_snr_wrong_trial": ("c[i].snr = (double)c[i].S / (sigma[c[i].dm_idx] * sw);",
                            "c[i].snr = (double)c[i].S / (sigma[0] * sw);"),
    # streamed search (window rule, carry, time offset)
    "stream_window_inclusive": ("if (first >= nwin) break;", "if (first > nwin) break;"),
    "stream_no_carry": ("if (first == 0 && carry_in && carry_in[k]) continue;",
                        "if (0 && first == 0 && carry_in && carry_in[k]) continue;"),
    "stream_carry_at_nwin": ("carry_out[k] = (double)(P[nwin - 1 + W] - P[nwin - 1]) >= lim;",
                             "carry_out[k] = (double)(P[nwin + W] - P[nwin]) >= lim;"),
    "stream_no_offset": ("r.sample = best_t + t_offset;", "r.sample = best_t;"),
    "stream_peak_first_start": ("if (first == 0 && carry_in", "best_t = first;\n            if (first == 0 && carry_in"),
    # RFI mitigation
    "rfi_median_index": ("if (c > k) return v;", "if (c >= k) return v;"),
    "rfi_chan_flag_inclusive": ("chan_flag[c] = dm > (int64_t)nb_k", "chan_flag[c] = dm >= (int64_t)nb_k"),
    "rfi_zero_dm_unmasked": ("acc += chan_flag[c] ? m[c] : x[t * nchans + c];",
                             "acc += x[t * nchans + c];"),
    "rfi_mad_from_raw": ("ha[v > m[c] ? v - m[c] : m[c] - v] += h[v];", "ha[v] += h[v];"),
    # sub-band dedispersion variant
    "subband_nominal_upper": ("int n = g * G + (len - 1) / 2;", "int n = g * G + len / 2;"),
    "subband_top_index": ("int top = (c / S) * S;", "int top = c / S;"),
    "subband_rel_at_trial": ("at_d[top] + at_n[c] - at_n[top]", "at_d[top] + at_d[c] - at_d[top]"),
    "subband_no_stage2_shift": ("at_d[top] + at_n[c] - at_n[top]", "at_n[c]"),
    # per-width normalisation variant
    "wsig_upper_median": ("mad = a[(m - 1) / 2];", "mad = a[m / 2];"),
    "wsig_sqrt_kept": ("double lim = sigma_w ? thr_d * sigma_w[k] : thr_d * sigma * sw;",
                       "double lim = sigma_w ? thr_d * sigma_w[k] * sw : thr_d * sigma * sw;"),
    "wsig_starts_short": ("int64_t m = n - W + 1;", "int64_t m = n - W;"),
    # decimated boxcars
    "decim_no_grid": ("int64_t q = decim_step(W, decimate);", "int64_t q = 1;"),
    "decim_double_step": ("W % R == 0) ? W / R : 1;", "W % R == 0) ? 2 * W / R : 1;"),
    "decim_run_every_start": ("t += q;\n                while (t <= last) {",
                              "t += 1;\n                while (t <= last) {"),
    "wsig_snr_sqrt": ("r.snr = sigma_w ? (double)best_S / sigma_w[k] :",
                      "r.snr = sigma_w ? (double)best_S / (sigma_w[k] * sqrt((double)widths[k])) :"),
}

# the pin files that each group of mutants is checked against
PINS = {"rfi_": ["test_oracle_rfi.py"], "stream_": ["test_oracle_stream.py"],
        "subband_": ["test_oracle_subband.py"], "wsig_": ["test_oracle_widthsigma.py"],
        "decim_": ["test_oracle_decimate.py"]}
DEFAULT_PINS = ["test_oracle_pins.py", "test_oracle_stream.py"]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, source, tmp_path):
    find, repl = MUTANTS[name]
    # a site shared by the plain and the streamed detection is mutated in both
    assert source.count(find) >= 1, f"mutation site for {name} missing"
    csrc = tmp_path / "mutant.c"
    csrc.write_text(source.replace(find, repl))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", str(csrc), "-o", str(so), "-lm"], check=True)
    env = dict(os.environ, HPO_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    files = next((v for k, v in PINS.items() if name.startswith(k)), DEFAULT_PINS)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "-k", "not stress"] + [os.path.join(ROOT, "tests", f) for f in files],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught mutant {name}:\n{r.stdout[-2000:]}"
