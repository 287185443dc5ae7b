"""Planted-mistake check of the oracle pins.

Each case copies ks_oracle.c, plants one plausible mistake (a dropped term, a
wrong sign, a transposed operand, a reversed walk), builds the copy with gcc
and runs the pin tests against it in a child process.  The pins must fail for
every mutant, which shows they constrain each part of the oracle.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ks_oracle.c")

MUTANTS = {
    "exclusive_demand": ("    run += buy[p];\n    dcum[p] = run;", "    dcum[p] = run;\n    run += buy[p];"),
    "highest_tick_tie": ("if (best < 0) { best = p; continue; }", "best = p; continue;"),
    "sells_from_top": ("for (int32_t p = 0; p < L && left > 0; ++p) {",
                       "for (int32_t p = L - 1; p >= 0 && left > 0; --p) {"),
    "buyer_cash_sign": ("ag->cash[a] -= (int64_t)cr.pstar * f;", "ag->cash[a] += (int64_t)cr.pstar * f;"),
    "philox_operand": ("KO_PHILOX_MUL_B * (uint64_t)x2", "KO_PHILOX_MUL_B * (uint64_t)x1"),
    "philox_key_schedule": ("k1 += KO_PHILOX_WEYL_B;", "k1 += KO_PHILOX_WEYL_A;"),
    "history_not_shifted": ("ms->hist[0] = ms->last;\n    ms->last_v = (int32_t)cr.vstar;",
                            "ms->hist[0] = ms->hist[1];\n    ms->last_v = (int32_t)cr.vstar;"),
    "cda_history_not_shifted": ("ms->hist[0] = ms->last;\n    ms->last_v = (int32_t)vol;",
                                "ms->hist[0] = ms->hist[1];\n    ms->last_v = (int32_t)vol;"),
    "marginal_buy_strict": ("if (dcum[p] >= vmax) res->p_buy = p;", "if (dcum[p] > vmax) res->p_buy = p;"),
    "mixer_shift": ("z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;", "z = (z ^ (z >> 28)) * 0x94d049bb133111ebull;"),
    "agent_priority_reversed": ("for (int32_t a = 0; a < A; ++a) {\n    if (qty[a] <= 0) continue;\n    order[",
                                "for (int32_t a = A - 1; a >= 0; --a) {\n    if (qty[a] <= 0) continue;\n    order["),
    "mlp_relu_mask_dropped": ("dh2[k] = a2[k] > 0.0 ? acc : 0.0;", "dh2[k] = acc;"),
    "mlp_w2_transposed": ("acc += v->W2[i * KO_H + k] * h1[k];", "acc += v->W2[k * KO_H + i] * h1[k];"),
    "mlp_w1_transposed_back": ("acc += v.W2[i * KO_H + k] * dh2[i];", "acc += v.W2[k * KO_H + i] * dh2[i];"),
    "mlp_bias_dropped": ("double acc = v->b3[i];", "double acc = 0.0;"),
    "mlp_mse_factor": ("dz[KO_OUT - 1] = 2.0 * e;", "dz[KO_OUT - 1] = e;"),
    "mlp_sample_le": ("if (u < c) return i;", "if (u <= c) return i;"),
    "mlp_qty_rounding": ("double q = floor(exp(z[KO_OUT - 1]) + 0.5);", "double q = floor(exp(z[KO_OUT - 1]));"),
    # the policy's raw features and its optimiser
    "features_sides_swapped": ("raw[9 + k] = (pa >= 0 && pa < L) ? (int32_t)sell[pa] : 0;",
                               "raw[9 + k] = (pa >= 0 && pa < L) ? (int32_t)buy[pa] : 0;"),
    "features_k_off_by_one": ("int32_t pa = ms->last + k, pb = ms->last - k;",
                              "int32_t pa = ms->last + k - 1, pb = ms->last - k + 1;"),
    "features_grid_edge": ("raw[13 + k] = (pb >= 0 && pb < L)", "raw[13 + k] = (pb > 0 && pb < L)"),
    "features_after_cancellation": (
        "        if (ag->qty[a] <= 0) continue;\n        if (ag->side[a] == 0) buy[",
        "        uint32_t cw[4];\n        ko_draw(P->seed, s, (uint32_t)a, m, 0u, cw);\n"
        "        if (ag->qty[a] <= 0 || (P->carry_book && cw[0] < P->cancel_thresh)) continue;\n"
        "        if (ag->side[a] == 0) buy["),
    "adam_no_bias_correction": ("w[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);",
                                "w[i] -= lr * m[i] / (sqrt(v[i]) + eps);"),
    "adam_eps_inside_sqrt": ("w[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);",
                             "w[i] -= lr * (m[i] / c1) / sqrt(v[i] / c2 + eps);"),
    "adam_b1_in_second_moment": ("v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];",
                                 "v[i] = b1 * v[i] + (1.0 - b1) * g[i] * g[i];"),
    # the rule decisions
    "rule_coin_reversed": ("int32_t coin = (w[1] >> 31) ? 1 : 0;", "int32_t coin = (w[1] >> 31) ? 0 : 1;"),
    "rule_zi_range_short": ("int64_t off = ko_range(w[2], 2 * (int64_t)P->zi_offset + 1) - P->zi_offset;",
                            "int64_t off = ko_range(w[2], 2 * (int64_t)P->zi_offset) - P->zi_offset;"),
    "rule_momentum_lag": ("int32_t ret = ms->hist[0] - ms->hist[P->mom_lookback];",
                          "int32_t ret = ms->hist[0] - ms->hist[P->mom_lookback - 1];"),
    "rule_reversion_away": ("s = last < ms->fund ? 0 : (last > ms->fund ? 1 : coin);",
                            "s = last < ms->fund ? 1 : (last > ms->fund ? 0 : coin);"),
    "rule_through_price_sign": ("*tick = ko_clamp((int64_t)last + (s == 0 ? off : -off), 0, L - 1);",
                                "*tick = ko_clamp((int64_t)last + (s == 0 ? -off : off), 0, L - 1);"),
    "rule_qty_uses_zi_qmax": ("*qty = 1 + (int32_t)ko_range(w[3], P->rb_qmax);",
                              "*qty = 1 + (int32_t)ko_range(w[3], P->zi_qmax);"),
    "init_class_threshold": ("if (pct < P->mix_pct[0]) ag->atype[a] = KO_ZI;", "if (pct <= P->mix_pct[0]) ag->atype[a] = KO_ZI;"),
    "init_fundamental_stream": ("ko_draw(P->seed, 0u, 0u, m, 2u, w);", "ko_draw(P->seed, 0u, 0u, m, 1u, w);"),
    # the continuous double auction
    "cda_lifo": ("if (better || (t == tb && stamp[b] < stamp[best])) best = b;",
                 "if (better || (t == tb && stamp[b] > stamp[best])) best = b;"),
    "cda_fill_at_arrival_price": ("const int32_t px = ag->tick[r];", "const int32_t px = tk;"),
    "cda_worst_price_first": ("const int better = side == 0 ? (t < tb) : (t > tb);",
                              "const int better = side == 0 ? (t > tb) : (t < tb);"),
    "cda_strict_cross": ("if (side == 0 ? t > tick : t < tick) continue;",
                         "if (side == 0 ? t >= tick : t <= tick) continue;"),
    "cda_last_from_first_fill": ("        last_fill = px;\n", "        if (last_fill < 0) last_fill = px;\n"),
    "cda_resting_seller_cash_sign": ("ag->inv[r] -= f; ag->cash[r] += (int64_t)px * f;",
                                     "ag->inv[r] -= f; ag->cash[r] -= (int64_t)px * f;"),
    # the paper-agent mode
    "paper_maker_parity": ("sd = (int32_t)(((int64_t)a + (int64_t)s) % 2);",
                           "sd = (int32_t)(((int64_t)a + (int64_t)s + 1) % 2);"),
    "paper_round_half_up": ("return (q % 2 != 0) ? q + 1 : q;", "return q + 1;"),
    "paper_marketable_sides": ("p = sd ? 0 : L - 1;", "p = sd ? L - 1 : 0;"),
    "paper_momentum_reversed": ("sd = ret > 0 ? 0 : 1;", "sd = ret > 0 ? 1 : 0;"),
    "paper_mid_fallback": ("int32_t mid2 = (bb >= 0 && ba < L) ? bb + ba : 2 * ms->last;",
                           "int32_t mid2 = (bb >= 0 && ba < L) ? bb + ba : ms->mid2;"),
    "paper_marginal_residual": ("else if (p == cr.p_buy) nb = buy[p] - (cr.vstar - above_b);",
                                "else if (p == cr.p_buy) nb = buy[p] - cr.vstar;"),
    "paper_counter_layout": ("(uint64_t)step * 8ull", "(uint64_t)step * 4ull"),
    "paper_class_threshold": ("if (pct < P->maker_pct) return KO_PAPER_MAKER;",
                              "if (pct <= P->maker_pct) return KO_PAPER_MAKER;"),
    "paper_noise_width": ("int64_t num = ((int64_t)mid2 - 2 * D) * (1ll << 32) + 4 * D * (int64_t)w_price;",
                          "int64_t num = ((int64_t)mid2 - 2 * D) * (1ll << 32) + 2 * D * (int64_t)w_price;"),
    # the sliding window
    "window_odd_shift": ("int32_t k = 2 * (int32_t)ko_floor_div(dev, 4);", "int32_t k = (int32_t)ko_floor_div(dev, 2);"),
    "window_last_not_moved": ("        ms->last -= k;\n", "        ms->last -= 0;\n"),
    "window_trigger_band": ("if (dev > L / 2 || dev < -(L / 2)) {", "if (dev > L / 4 || dev < -(L / 4)) {"),
    "window_trace_relative": ("trace[2 * j] = P->window ? (int32_t)(ms->base + ms->last) : pabs;",
                              "trace[2 * j] = P->window ? ms->last : pabs;"),
    "window_sum_relative": ("ms->sum_p += ms->base + cr.pstar;", "ms->sum_p += cr.pstar;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mut.c")
        so = os.path.join(d, "libmut.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", so, c, "-lm"], check=True)
        env = dict(os.environ, KS_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                            os.path.join(ROOT, "tests", "test_oracle_mlp_pins.py"),
                            os.path.join(ROOT, "tests", "test_oracle_paper_pins.py"),
                            os.path.join(ROOT, "tests", "test_oracle_cda_pins.py"),
                            os.path.join(ROOT, "tests", "test_oracle_rule_pins.py")],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
