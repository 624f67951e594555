"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of the oracle's C source -- a dropped
term, a wrong sign, index or operand, an off-by-one bound, a wrong rounding
-- builds the copy in a temporary directory, and runs the pins of
``test_oracle_pins.py`` that should catch it against that copy, in a child
interpreter whose ``import oracle`` resolves to the copy.  The case passes
when at least one of those pins fails.  A control case runs the same pins
against an unmodified copy and requires them to pass, so a failure of the
harness itself cannot pass for a caught mistake.  The repository's oracle is
never modified.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "psw_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (name, text in the oracle's source (must occur exactly once), replacement,
#  pins expected to catch it as a pytest -k expression).  Only mistakes that
#  change some output are listed: e.g. taking one tail instead of both for
#  the escape slot changes no table, its mass (below 2e-7 with the support
#  at 7 sigma) staying under one count of 2^16 either way.
MUTANTS = [
    ("rmsnorm_sum_not_mean", "sqrt(ss / (double)d + OR_EPS)", "sqrt(ss + OR_EPS)", "rmsnorm"),
    ("silu_wrong_sign", "return x / (1.0 + exp(-x));", "return x / (1.0 + exp(x));", "silu"),
    ("swiglu_gate_on_up", "g[f] = or_silu(g[f]) * u[f];", "g[f] = g[f] * or_silu(u[f]);", "swiglu"),
    ("attention_unscaled", "double scale = 1.0 / sqrt((double)dh);", "double scale = 1.0;", "attention"),
    ("attention_bias_sign", "s[j] = acc * scale + bias[(long)j * nh + h];",
     "s[j] = acc * scale - bias[(long)j * nh + h];", "attention"),
    ("wavefront_label_transposed", "return 2 * i + j; ", "return i + 2 * j; ", "fig2b or interior or step_counts"),
    ("cyclic_label_wrong", "if (mask == 1) return ((i % 4) + (j % 4)) % 4;",
     "if (mask == 1) return ((i % 4) + 2 * (j % 4)) % 4;", "fig2a"),
    ("self_attention_excludes_equal_label", "int ok = (kind == 0) ? (lq < lp) : (lq <= lp);",
     "int ok = (kind == 0) ? (lq < lp) : (lq < lp);", "fig2b or interior"),
    ("accumulator_includes_equal_label", "int ok = (kind == 0) ? (lq < lp) : (lq <= lp);",
     "int ok = (kind == 0) ? (lq <= lp) : (lq <= lp);", "fig2b or interior"),
    ("raster_tiebreak_dropped", "if (mask == 0) ok = ok && ((long)qi * W + qj < (long)pi * W + pj);",
     "if (mask == 0) ok = ok;", "fig2b or interior or same_step"),
    ("relative_bias_index_transposed", "off[n] = (di + w) * c->k + (dj + w);",
     "off[n] = (dj + w) * c->k + (di + w);", "dense_mask_formulation"),
    ("relative_bias_by_absolute_column", "off[n] = (di + w) * c->k + (dj + w);",
     "off[n] = (di + w) * c->k + (qj % c->k);", "translation"),
    ("attention_residual_dropped",
     "or_matvec(o, WP(bw->Wo), d, d, t);\n    for (int e = 0; e < d; e++) xp[e] += t[e];\n    if (c->temporal)",
     "or_matvec(o, WP(bw->Wo), d, d, t);\n    for (int e = 0; e < d; e++) xp[e] = t[e];\n    if (c->temporal)",
     "dense_mask_formulation"),
    ("accumulator_query_wrong_gain", "or_rmsnorm(ep, WP(aw->g_q), d, n);", "or_rmsnorm(ep, WP(aw->g_ffn), d, n);",
     "dense_mask_formulation"),
    ("mu_offset_sign", "s->mu[(long)p * C + ch] = WP(s->lay.gamma_mu)[ch] * o[ch] + WP(s->lay.beta_mu)[ch];",
     "s->mu[(long)p * C + ch] = WP(s->lay.gamma_mu)[ch] * o[ch] - WP(s->lay.beta_mu)[ch];",
     "dense_mask_formulation"),
    ("temporal_age_reversed", "int slot = f % c->Tf, age = s->frame - f;", "int slot = f % c->Tf, age = f - f0;",
     "dense_mask_formulation"),
    ("channel_shift_missing", "int cc = (g - 1) * Cg + ch;", "int cc = g * Cg + ch;",
     "channel_groups_causal or dense_mask_formulation"),
    ("mu_scale_channel_index", "WP(s->lay.gamma_mu)[ch] * o[ch]", "WP(s->lay.gamma_mu)[0] * o[ch]",
     "dense_mask_formulation"),
    ("lrp_window_masked",
     "int nw = or_window_keys(c, -1, p, idx, off);\n            for (int ff = f0; ff <= f; ff++) {\n"
     "                int sl = ff % Tw",
     "int nw = or_window_keys(c, 1, p, idx, off);\n            for (int ff = f0; ff <= f; ff++) {\n"
     "                int sl = ff % Tw", "lrp"),
    ("lrp_bias_ignores_age", "WP(bw->bias)[((long)h * Tw + age) * kk + off[j]]",
     "WP(bw->bias)[((long)h * Tw + 0) * kk + off[j]]", "lrp"),
    ("context_sees_current_frame_only",
     "for (int ff = f0; ff <= f; ff++) {\n                int sl = ff % c->Tf, age = f - ff;",
     "for (int ff = f; ff <= f; ff++) {\n                int sl = ff % c->Tf, age = f - ff;",
     "dense_mask_formulation"),
    ("ct_mask_reads_next_group", "(i / dg <= o / dg) ? M", "(i / dg <= o / dg + 1) ? M",
     "channel_groups_causal or dense_mask_formulation"),
    ("ct_mask_drops_own_group", "(i / dg <= o / dg) ? M", "(i / dg < o / dg) ? M", "dense_mask_formulation"),
    ("ct_group_norm_over_all_groups",
     "for (int j = 0; j < G; j++) or_rmsnorm(x + (long)j * w, g + (long)j * w, w, y + (long)j * w);",
     "or_rmsnorm(x, g, n, y);", "channel_groups_causal or dense_mask_formulation"),
    ("context_padding_zero", "if (f == 0) memcpy(g + (long)p * d, WP(s->lay.pad), sizeof(double) * d);",
     "if (f == 0) memset(g + (long)p * d, 0, sizeof(double) * d);", "dense_mask_formulation"),
    ("context_final_norm_gain", "or_rmsnorm(g + (long)p * d, WP(s->lay.g_ctx), d, cn);",
     "or_rmsnorm(g + (long)p * d, WP(s->lay.ctx[0].g_attn), d, cn);", "dense_mask_formulation"),
    ("cross_keys_from_value_weights", "or_matvec(cn, WP(bw->Wxk), d, d, s->XK + base);",
     "or_matvec(cn, WP(bw->Wxv), d, d, s->XK + base);", "dense_mask_formulation"),
    ("hyper_tap_index_transposed", "int sub = (i % c->r) * c->r + (j % c->r);",
     "int sub = (j % c->r) * c->r + (i % c->r);", "dense_mask_formulation"),
    ("latent_embedding_bias_dropped", "for (int e = 0; e < c->d; e++) out[e] += WP(b_off)[e];", "",
     "dense_mask_formulation"),
    ("accumulator_residual_dropped", "xp[e] = ep[e] + t[e];", "xp[e] = t[e];", "dense_mask_formulation"),
    ("sigma_lower_clamp_dropped",
     "if (v < lo) v = lo;\n        if (v > hi) v = hi;\n        s->sigma[(long)p * C + ch]",
     "if (v > hi) v = hi;\n        s->sigma[(long)p * C + ch]", "sigma_clamped"),
    ("sigma_upper_clamp_grouped_heads_dropped",
     "if (v > hi) v = hi;\n            s->sigma[(long)p * C + cc]", "s->sigma[(long)p * C + cc]", "sigma_clamped"),
    ("lrp_reads_module1_stream", "or_rmsnorm(s->x2 + (long)p * d, WP(s->lay.lrp_g_rep), d, nr);",
     "or_rmsnorm(s->x1 + (long)p * d, WP(s->lay.lrp_g_rep), d, nr);", "lrp"),
    ("pixel_shuffle_transposed", "(2 * a + b) * C + c]", "(2 * b + a) * C + c]", "hyperprior_matches_dense"),
    ("conv_tap_wrong_column", "int ii = st * i + di - 1, jj = st * j + dj - 1;",
     "int ii = st * i + di - 1, jj = st * j + di - 1;", "hyperprior_matches_dense"),
    ("downsampling_skip_dropped", "for (long e = 0; e < n; e++) t[e] += k[e];\n    free(a); free(k);",
     "free(a); free(k);", "hyperprior_matches_dense"),
    ("synthesis_crop_stride", "x + (long)i * w * c->d, sizeof(double) * c->W * c->d)",
     "x + (long)i * c->W * c->d, sizeof(double) * c->W * c->d)", "hyperprior_matches_dense"),
    ("zhat_floor_not_round", "double r = nearbyint(x[e]);", "double r = floor(x[e]);", "hyperprior_matches_dense"),
    ("likelihood_bin_width",
     "double p = 0.5 * (erfc((u - 0.5) / den) - erfc((u + 0.5) / den));\n    return p < 1e-9",
     "double p = 0.5 * (erfc((u - 1.0) / den) - erfc((u + 0.5) / den));\n    return p < 1e-9",
     "likelihood or rate"),
    ("cdf_escape_floor_dropped", "erfc(((double)T + 0.5) / den);\n    freq[2 * T + 1] = 1u + (uint32_t)floor(",
     "erfc(((double)T + 0.5) / den);\n    freq[2 * T + 1] = (uint32_t)floor(", "cdf"),
    ("prior_escape_lower_tail_dropped", "double pesc = prior_cdf(w, L, ch, -T - 0.5) + (1.0 - ",
     "double pesc = (1.0 - ", "factorized_prior"),
    ("prior_slot_offset", "double pmf = prior_cdf(w, L, ch, v + 0.5) - prior_cdf(w, L, ch, v - 0.5);",
     "double pmf = prior_cdf(w, L, ch, v + 1.0) - prior_cdf(w, L, ch, v);", "factorized_prior"),
    ("cdf_slot_mass_shifted", "double u = (double)(s < 0 ? -s : s);", "double u = (double)(s < 0 ? -s : s) + 0.25;",
     "cdf_table_closed_form"),
    ("cdf_support_narrower", "int T = (int)ceil(7.0 * (double)tab[l]);", "int T = (int)ceil(6.0 * (double)tab[l]);",
     "cdf"),
    ("rans_escape_digit_order", "for (int q = 1; q >= 0; q--) {     /* d1 first: decoded last */",
     "for (int q = 0; q < 2; q++) {", "rans"),
    ("rans_escape_sign", "sv = (vv & 1) ? -mag : mag;", "sv = (vv & 1) ? mag : -mag;", "rans"),
    ("rans_decoder_lane", "int lane = (int)(k % 32), l = idx[(long)a * D->C + c], T = D->tb.T[l];",
     "int lane = (int)((k + 1) % 32), l = idx[(long)a * D->C + c], T = D->tb.T[l];", "rans"),
    ("rans_final_state_unchecked", "for (int l = 0; l < 32; l++) if (D->x[c][l] != OR_LOW) bad = 1;", "",
     "rans"),
    ("rans_latent_range_unchecked", "if (yv < -32768 || yv > 32767) { D->err = 1; yv = 0; }", "",
     "outside_int16"),
    ("window_radius_short", "for (int di = -w; di <= w; di++) {", "for (int di = -w; di < w; di++) {",
     "dense_mask_formulation or lrp"),
    ("mean_truncated_not_rounded", "m[a] = (int32_t)rintf(mc);", "m[a] = (int32_t)mc;", "quantize"),
    ("likelihood_floor_lower", "return p < 1e-9 ? 1e-9 : p;", "return p < 1e-12 ? 1e-12 : p;", "likelihood or rate"),
    ("e4m3_tensor_scale_exponent", "s = ldexp(1.0, e - 7);", "s = ldexp(1.0, e - 8);", "e4m3"),
    ("e4m3_saturation", "if (v > 448.0) v = 448.0;", "if (v > 480.0) v = 480.0;", "e4m3"),
    # self-consistent coder changes (round trips still pass): only a reader
    # of the format written apart from the oracle catches them
    ("container_escape_digits_swapped",
     ("for (int q = 1; q >= 0; q--) {     /* d1 first: decoded last */", "uint32_t vv = dig[0] | (dig[1] << 16);"),
     ("for (int q = 0; q < 2; q++) {", "uint32_t vv = dig[1] | (dig[0] << 16);"), "independent_reader"),
    ("container_lanes_reversed",
     ("int lane = (int)(k % 32), l = idx[a], T = tb.T[l];",
      "int lane = (int)(k % 32), l = idx[(long)a * D->C + c], T = D->tb.T[l];"),
     ("int lane = 31 - (int)(k % 32), l = idx[a], T = tb.T[l];",
      "int lane = 31 - (int)(k % 32), l = idx[(long)a * D->C + c], T = D->tb.T[l];"), "independent_reader"),
    ("container_header_H_W_swapped",
     ("put16(out + 8, (uint16_t)H); put16(out + 10, (uint16_t)W);",
      "get16(buf + 8) != H || get16(buf + 10) != W"),
     ("put16(out + 8, (uint16_t)W); put16(out + 10, (uint16_t)H);",
      "get16(buf + 8) != W || get16(buf + 10) != H"), "independent_reader"),
    ("e4m3_ties_away", "double v = nearbyint(a / q) * q;", "double v = round(a / q) * q;", "e4m3"),
    ("e4m3_subnormal_step", "if (e < -6) e = -6;", "if (e < -7) e = -7;", "e4m3"),
    ("scale_index_strict", "if (tab[t] >= sigma[a]) { l = t; break; }", "if (tab[t] > sigma[a]) { l = t; break; }",
     "quantize"),
]


def _run_pins(tmp_path, name, source, kexpr):
    """Build the oracle from `source` under tmp_path and run the pins
    selected by kexpr against it; returns (exit code, the library was built,
    the last line of pytest's summary)."""
    d = tmp_path / name
    (d / "oracle").mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), d / "oracle" / "__init__.py")
    (d / "oracle" / "psw_oracle.c").write_text(source)
    # the copy first, then the repository (synth); no conftest, which would
    # put the repository's own oracle first; run from the copy's directory
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(d), ROOT]), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "--noconftest", "-x", "-q", "-p", "no:cacheprovider",
                        "-W", "ignore::pytest.PytestUnknownMarkWarning", PINS, "-k", kexpr],
                       cwd=str(d), env=env, capture_output=True, text=True, timeout=600)
    built = (d / "oracle" / "libpsw_oracle.so").exists()
    last = (r.stdout.strip().splitlines() or [r.stderr[-400:]])[-1]
    return r.returncode, built, last


def _case(tmp_path, mutant):
    name, old, new, kexpr = mutant
    src = open(SRC).read()
    # a tuple: one mistake made at several places that agree with each other
    # (the encoder and the decoder changed together)
    pairs = list(zip(old, new)) if isinstance(old, tuple) else [(old, new)]
    for o, n in pairs:
        if src.count(o) != 1:
            return name, "the mutated text does not occur exactly once in the oracle"
        src = src.replace(o, n)
    rc, built, last = _run_pins(tmp_path, name, src, kexpr)
    if not built:
        return name, "the mutated oracle did not build: " + last
    # 1: some pin failed; a signal: the oracle crashed under the pins (e.g. a
    # zero frequency reaching the coder); anything else (no test selected, a
    # collection error, every pin passing) means the mistake went unnoticed
    if rc == 1 or rc < 0:
        return name, None
    return name, f"no pin failed (exit {rc}: {last})"


def test_harness_control_passes_on_the_unmodified_oracle(tmp_path):
    src = open(SRC).read()
    kexpr = " or ".join(sorted({m[3] for m in MUTANTS}))
    rc, built, last = _run_pins(tmp_path, "control", src, kexpr)
    assert built, last
    assert rc == 0, last


def test_every_planted_mistake_fails_a_pin(tmp_path):
    """All cases at once (a few child processes at a time, each with a few
    threads); the failure message lists every mistake no pin caught."""
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(lambda m: _case(tmp_path, m), MUTANTS))
    missed = [f"{name}: {why}" for name, why in res if why]
    assert not missed, "\n".join(missed)
