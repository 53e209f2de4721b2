"""Plants plausible mistakes in copies of the CPU oracle and checks that the pins catch each.

Each mutant is a textual edit of ``oracle/cvoracle.c`` (a dropped term, a wrong sign or
bound, a transposed operand, ...), compiled into a temporary library. The real oracle is
never modified. A mutant that passes every pin would mean the pins are blind to that
mistake, so the test fails.
"""
import os
import shutil
import subprocess

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "cvoracle.c")

MUTANTS = {
    "haversine_no_half": ("double s_phi = sin(dphi / 2.0);", "double s_phi = sin(dphi);"),
    "haversine_no_cos": ("cos(phi1) * cos(phi2) * s_lam * s_lam", "s_lam * s_lam"),
    "haversine_no_asin": ("return 2.0 * radius_m * asin(r);", "return 2.0 * radius_m * r;"),
    "haversine_transposed": ("double dlam = (lon2 - lon1) * rad;", "double dlam = (lat2 - lat1) * rad;"),
    "bin_truncates": ("if ((a % bin_ms != 0) && (a < 0)) q -= 1;", ""),
    "grid_top_edge": ("!(f < (double)n)", "!(f <= (double)n)"),
    "key_row_col_swapped": ("(uint64_t)p->n_rows + (uint64_t)r) * (uint64_t)p->n_cols +\n                       (uint64_t)c)",
                            "(uint64_t)p->n_rows + (uint64_t)c) * (uint64_t)p->n_cols +\n                       (uint64_t)r)"),
    "sort_ties_reversed": ("  return i < j ? -1 : (i > j ? 1 : 0);\n}\n\n/* Order sorted positions",
                           "  return i > j ? -1 : (i < j ? 1 : 0);\n}\n\n/* Order sorted positions"),
    "start_by_position_only": ("int start = (k == 0) || (jid[order[k - 1]] != jid[i]);", "int start = (k == 0);"),
    "dup_threshold": ("if (dt == 0) f |= ORC_F_DUP;", "if (dt <= 1) f |= ORC_F_DUP;"),
    "accel_no_kmh": ("ac = (((double)spd[i] - (double)spd[q]) / 3.6) / dt_s;", "ac = ((double)spd[i] - (double)spd[q]) / dt_s;"),
    "vhat_no_kmh": ("vh = d / dt_s * 3.6;", "vh = d / dt_s;"),
    "dwell_or": ("if (spd[q] < p->v_stop_kmh && spd[i] < p->v_stop_kmh)", "if (spd[q] < p->v_stop_kmh || spd[i] < p->v_stop_kmh)"),
    "no_negzero_canon": ("spd[i] = (speed[i] == 0.0f) ? 0.0f : speed[i];", "spd[i] = speed[i];"),
    "distance_not_summed": ("jr->distance_m[j] += pts->d[k];", "jr->distance_m[j] = pts->d[k];"),
    "decimal_16_digits": ("if (n_int + n_frac > 15) return 0;", "if (n_int + n_frac > 16) return 0;"),
    "lat_range_180": ("!(fabs(la) <= 90.0)", "!(fabs(la) <= 180.0)"),
    "cell_sum_first_only": ("cl->sum[c] += (double)s;", "if (cl->count[c] == 1) cl->sum[c] += (double)s;"),
    "cell_min_as_max": ("if (s < cl->min[c]) cl->min[c] = s;", "if (s > cl->min[c]) cl->min[c] = s;"),
    "direction_no_offset": ("fmod(h + (mode == ORC_DXN_CARDINAL ? 45.0 : 0.0), 360.0)", "fmod(h, 360.0)"),
    "direction_negative_unwrapped": ("  if (r < 0.0) r += 360.0;\n  if (r >= 360.0) r = 0.0;", "  if (r >= 360.0) r = 0.0;"),
    "volume_counts_points": ("if (e == a || jid[ent[e - 1]] != jid[i]) vol += 1;", "vol += 1;"),
    "lattice_sum_by_point_order": ("  if (g_jid[i] != g_jid[j]) return g_jid[i] < g_jid[j] ? -1 : 1;\n  return i < j ? -1 : (i > j ? 1 : 0);\n}\n\nint orc_lattice",
                                   "  return i < j ? -1 : (i > j ? 1 : 0);\n}\n\nint orc_lattice"),
    "normalise_global": ("const float mn0 = ch_min[2 * d], mx0 = ch_max[2 * d],", "const float mn0 = ch_min[0], mx0 = ch_max[0],"),
    "cell_volume_counts_points": ("if (cl->count[c] == 0 || jid[order[byk[t - 1]]] != jid[order[k]]) cl->volume[c] += 1;", "cl->volume[c] += 1;"),
    "stop_run_not_reset": ("run_stop = (f & ORC_F_STOP) ? run_stop + dwell : 0;", "run_stop = run_stop + dwell;"),
    "speed_accel_in_kmh": ("const double v = d / dt_s;", "const double v = d / dt_s * 3.6;"),
    "journey_end_lon_is_start": ("jr->end_lon[j] = lon[i];", "jr->end_lon[j] = jr->start_lon[j];"),
    "journey_start_lon_from_lat": ("jr->start_lon[nj] = lon[i];", "jr->start_lon[nj] = lat[i];"),
    "journey_end_lat_from_lon": ("jr->end_lat[j] = lat[i];", "jr->end_lat[j] = lon[i];"),
    "lattice_key_dir_bin_swapped":("lkey[i] = (((uint32_t)b * 4u + (uint32_t)d)", "lkey[i] = (((uint32_t)d * 4u + (uint32_t)b)"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path, small_day):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / "cvoracle.c"
    mut.write_text(src.replace(old, new))
    shutil.copy(os.path.join(os.path.dirname(SRC), "cvoracle.h"), tmp_path / "cvoracle.h")
    so = str(tmp_path / "libmutant.so")
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", so, str(mut), "-lm"])
    o = oracle.Oracle(so)
    caught = []
    for pin in P.CPU_PINS:
        try:
            pin(o)
        except AssertionError:
            caught.append(pin.__name__)
    if not caught:
        for pin in P.DATA_PINS:
            try:
                pin(o, small_day)
            except AssertionError:
                caught.append(pin.__name__)
    assert caught, f"no pin catches the mutant {name}"
