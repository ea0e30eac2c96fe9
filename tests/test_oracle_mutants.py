"""Planted mistakes: each mutant of the oracle must fail at least one pin.

The mutants are textual edits of a COPY of oracle/cdmt_oracle.c (or of the
module's own composition code in oracle/__init__.py), compiled into a temporary
directory on the CPU; the oracle itself is never modified.  Every
edit is a plausible slip (a flipped sign, a dropped term, a wrong index or
centre); the pins in test_oracle_pins.py must reject each one.  (Swapping the
reference of the subband-wide chirp for the channel centre while keeping the
absolute frequencies is not listed: it changes the phase only at second order,
since the reference's linear terms cancel against the shifted 1/F term.)
"""
import importlib.util
import os
import shutil

import pytest

import test_oracle_pins as pins

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

# (name, original text, replacement, occurrence index or None for all)
MUTANTS = [
    ("chirp_sign", "- I * sin(2.0 * ORC_PI * phi)", "+ I * sin(2.0 * ORC_PI * phi)", None),
    ("subband_not_channel_centre", "double nu_c = orc_channel_centre(nu_s, bw, nchan, c);",
     "double nu_c = nu_s;", None),
    ("channel_centre_half_off", "((double)c + 0.5) * bw", "((double)c) * bw", None),
    ("no_forward_swap", "xs[i] = tmp[(i + n / 2) % n] * sc;", "xs[i] = tmp[i] * sc;", None),
    ("forward_sign", "orc_fft(tmp, n, -1);", "orc_fft(tmp, n, +1);", None),
    ("fft_twiddle_sign", "double ang = (double)sign * 2.0 * ORC_PI * (double)k / (double)len;",
     "double ang = -(double)sign * 2.0 * ORC_PI * (double)k / (double)len;", None),
    ("inverse_norm", "double sc = 1.0 / sqrt((double)m);", "double sc = 1.0 / (double)m;", None),
    ("bin_grid_half_off", "((double)j - 0.5 * (double)m) * bw", "((double)j - 0.5 * (double)m + 0.5) * bw", None),
    ("linear_not_quadratic", "dm * nu * nu /", "dm * nu /", None),
    ("no_unpad_offset", "pw[nd / 2 + u * nint + qq]", "pw[u * nint + qq]", None),
    ("one_pol_detected", "for (int p = 0; p < 2; p++) {\n                channel_series",
     "for (int p = 0; p < 1; p++) {\n                channel_series", None),
    ("short_integration", "for (int qq = 0; qq < nint; qq++)", "for (int qq = 0; qq < nint - 1; qq++)", None),
    ("eq2_reversed", "(1.0 / (nu_min * nu_min) - 1.0 / (nu_max * nu_max))",
     "(1.0 / (nu_max * nu_max) - 1.0 / (nu_min * nu_min))", None),
    ("overlap_uses_top_channel", "double lo = nu_s0 - 0.5 * bw;", "double lo = nu_s0 + 0.5 * bw - bw / (double)nchan;",
     None),
    ("segment_stride_wrong", "(size_t)(k * sv)) * 4;", "(size_t)(k * nbin)) * 4;", None),
    ("subband_chirp_no_offset", "chirp ? nu_c - nu_s : 0.0", "0.0", None),
    ("subband_overlap_channel_width", "(chirp ? bw : bw / (double)nchan)", "(bw / (double)nchan)", None),
    ("incoh_delay_sign", "(1.0 / (nu[r] * nu[r]) - 1.0 / (top * top))", "(1.0 / (top * top) - 1.0 / (nu[r] * nu[r]))",
     None),
    ("incoh_no_coherent_dm", "double dm = dm_c[i] + ddm_lo", "double dm = ddm_lo", None),
    ("incoh_tsamp_no_nint", "(double)nint * (double)nchan / (bw * 1e6)", "(double)nchan / (bw * 1e6)", None),
    ("incoh_subband_freq_in_channel_mode", "chirp ? nu_s : orc_channel_centre(nu_s, bw, nchan, c)", "nu_s", None),
    ("redig_sample_sigma", "s2 / (double)nt - mu * mu", "(s2 - mu * s1) / (double)(nt - 1)", None),
    ("redig_offset_127", "fmaf(row[t] - muf, g, 128.0f)", "fmaf(row[t] - muf, g, 127.0f)", None),
    ("redig_truncate", "float x = rintf(", "float x = truncf(", None),
    ("redig_increasing_order", "(size_t)(rows - 1 - r)] = (uint8_t)x;", "(size_t)r] = (uint8_t)x;", None),
    ("redig_no_clip_high", "if (x > 255.0f) x = 255.0f;", "if (x > 255.0f) x = x - 256.0f;", None),
    ("sk_shape_factor_dropped", "(n * k + 1.0) / (n - 1.0)", "(n + 1.0) / (n - 1.0)", None),
    ("sk_sigma_without_k_plus_1", "sqrt(2.0 * (double)(k + 1) / ((double)k * (double)n))",
     "sqrt(2.0 / ((double)k * (double)n))", None),
    ("sk_mean_not_squared", "(n * s2 / (s1 * s1) - 1.0)", "(s2 / s1 - 1.0)", None),
    ("sk_one_sided", "fabs(v - 1.0) > thr", "v - 1.0 > thr", None),
]

PIN_CALLS = [
    lambda o: pins.test_fft_matches_naive_dft(o, 16, -1),
    lambda o: pins.test_fft_matches_naive_dft(o, 16, +1),
    lambda o: pins.test_eq2_worked_values(o),
    lambda o: pins.test_lofar_channelisation_and_volume(o),
    lambda o: pins.test_tone_at_channel_centre_is_dm_invariant(o, 3),
    lambda o: pins.test_impulse_lands_in_one_sample_per_channel(o),
    lambda o: pins.test_parseval_per_segment(o),
    lambda o: pins.test_physical_impulse_recovered_at_true_dm(o),
    lambda o: pins.test_brute_force_dense_matrices(o),
    lambda o: pins.test_noise_mean_and_variance(o),
    lambda o: pins.test_overlap_rule_values(o),
    lambda o: pins.test_overlap_covers_every_channel_and_is_minimal(o),
    lambda o: pins.test_subband_chirp_aligns_channels(o),
    lambda o: pins.test_subband_chirp_is_the_channel_chirp_for_one_channel(o),
    lambda o: pins.test_subband_overlap_covers_subband_sweep_and_is_minimal(o),
    lambda o: pins.test_subband_chirp_is_unitary(o),
    lambda o: pins.test_incoherent_zero_dm_is_the_channel_sum(o),
    lambda o: pins.test_incoherent_dispersed_impulse_lines_up_at_its_dm(o, 0),
    lambda o: pins.test_incoherent_dispersed_impulse_lines_up_at_its_dm(o, 1),
    lambda o: pins.test_incoherent_delay_table(o),
    lambda o: pins.test_incoherent_is_linear_and_shift_covariant(o),
    lambda o: pins.test_redigitise_two_level_channel(o),
    lambda o: pins.test_redigitise_constant_channel_is_the_mean_code(o),
    lambda o: pins.test_redigitise_clips_an_outlier(o),
    lambda o: pins.test_redigitise_gaussian_row_statistics(o),
    lambda o: pins.test_redigitise_order_and_independence(o),
    lambda o: pins.test_redigitise_scale_invariance(o),
    lambda o: pins.test_sk_gamma_noise_mean_and_spread(o, 1),
    lambda o: pins.test_sk_gamma_noise_mean_and_spread(o, 16),
    lambda o: pins.test_sk_equals_brute_force_moments(o),
    lambda o: pins.test_sk_flags_impulsive_and_steady_rows(o),
    lambda o: pins.test_redigitise_sk_zaps_flagged_rows_only(o),
]


# mistakes in the composition that the Python module does itself (DM groups)
MUTANTS_PY = [
    ("grouped_no_offset", "off = (nd_max - nd_g) * nchan // 2", "off = 0", None),
    ("grouped_offset_sign", "(nd_max - nd_g) * nchan // 2", "(nd_g - nd_max) * nchan // 2", None),
    ("grouped_offset_not_halved", "(nd_max - nd_g) * nchan // 2", "(nd_max - nd_g) * nchan", None),
    ("grouped_no_coverage_step", "while not segments_cover(n, nd_g):", "while False:", None),
    ("grouped_overlap_of_first_dm", "dms = dm[first:first + count]", "dms = dm[first:first + 1]", None),
    ("grouped_all_nd_max", "if nd_g < 0 or nd_g > nd_max:", "if True:", None),
    # per-group FFT lengths
    ("grouped_lengths_plan_grid", "grid(nsamp - off, n, nchan, nd_g, nint)", "grid(nsamp - off, nbin, nchan, nd_g, nint)",
     None),
    ("grouped_lengths_most_work", "if w < work * (1 - 1e-12):", "if w > work * (1 + 1e-12):", None),
    ("grouped_lengths_overlap_at_plan_n", "nd_g = overlap(nsub, f_centre, bw, dms, nchan, nint, n, chirp)",
     "nd_g = overlap(nsub, f_centre, bw, dms, nchan, nint, nbin, chirp)", None),
]

GROUPED_PIN_CALLS = [
    lambda o: pins.test_grouped_overlaps_cover_their_group_and_are_minimal(o, 0, 2),
    lambda o: pins.test_grouped_overlaps_cover_their_group_and_are_minimal(o, 1, 4),
    lambda o: pins.test_grouped_overlaps_cover_their_group_and_are_minimal(o, 1, 3),
    lambda o: pins.test_grouped_filterbank_keeps_the_ungrouped_time_axis(o),
    lambda o: pins.test_grouped_impulse_at_the_closed_form_time(o, 5.0),
    lambda o: pins.test_grouped_impulse_at_the_closed_form_time(o, 10.0),
    lambda o: pins.test_grouped_lengths_cover_and_save_work(o, 0),
    lambda o: pins.test_grouped_lengths_cover_and_save_work(o, 1),
    lambda o: pins.test_grouped_lengths_keep_the_time_axis(o),
    lambda o: pins.test_grouped_lengths_impulse_at_the_closed_form_time(o, 5.0),
    lambda o: pins.test_grouped_lengths_impulse_at_the_closed_form_time(o, 10.0),
]


def _load_mutant(tmp_path, name, old, new, target="cdmt_oracle.c"):
    srcs = {f: open(os.path.join(ORACLE_DIR, f)).read() for f in ("cdmt_oracle.c", "__init__.py")}
    assert old in srcs[target], f"mutation anchor for {name} not found"
    srcs[target] = srcs[target].replace(old, new)
    d = tmp_path / f"oracle_{name}"
    d.mkdir()
    for f, text in srcs.items():
        (d / f).write_text(text)
    spec = importlib.util.spec_from_file_location(f"oracle_{name}", d / "__init__.py",
                                                  submodule_search_locations=[str(d)])
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    return mod


@pytest.mark.parametrize("name,old,new,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new, occ):
    mod = _load_mutant(tmp_path, name, old, new)
    caught = []
    for i, call in enumerate(PIN_CALLS):
        try:
            call(mod)
        except (AssertionError, ValueError, IndexError):
            caught.append(i)
    assert caught, f"mutant {name} passed every pin"


@pytest.mark.parametrize("name,old,new,occ", MUTANTS_PY, ids=[m[0] for m in MUTANTS_PY])
def test_python_mutant_is_caught(tmp_path, name, old, new, occ):
    mod = _load_mutant(tmp_path, name, old, new, target="__init__.py")
    caught = []
    for i, call in enumerate(GROUPED_PIN_CALLS):
        try:
            call(mod)
        except (AssertionError, ValueError, IndexError):
            caught.append(i)
    assert caught, f"mutant {name} passed every pin"
