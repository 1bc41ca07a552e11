"""The oracle's pins catch plausible mistakes: each case plants one mistake in
a copy of the oracle's source (a swapped comparison, a dropped term, a wrong
factor or sign), builds it on the CPU, and runs the pin that must notice it
against that copy; the pin has to fail.  The product is not involved."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.cpp")

CASES = [
    # (what, original text, planted mistake, pin that must fail)
    ("helix step: half-angle factor of the arc length",
     "const Real u = kappa * chord * Real(0.5);", "const Real u = kappa * chord * Real(0.25);",
     "tests/test_oracle_pins.py::test_propagation_matches_closed_form_helix_fp64"),
    ("neighbour finding: worst instead of best pair",
     "if (bu < 0 || d2 < best ||", "if (bu < 0 || d2 > best ||",
     "tests/test_oracle_pins.py::test_neighbours_equal_brute_force_on_tiny_frames"),
    ("selector: shared-cluster budget off by one",
     "Real(shared + 1) <= P.shared_frac * Real(kept + 1)",
     "Real(shared) <= P.shared_frac * Real(kept + 1)",
     "tests/test_oracle_pins.py::test_selector_matches_greedy_restatement_and_budget"),
    ("cleaner: upward links kept without the mutual test",
     "if (up[c] >= 0 && dn[up[c]] == c) cu[c] = up[c];", "if (up[c] >= 0) cu[c] = up[c];",
     "tests/test_oracle_pins.py::test_cleaner_and_start_hit_invariants"),
    ("Phase III: candidates cut with the interpolation cut instead of the stricter one",
     "if (c2 < P.ext_chi2) cands.push_back({c2, id});",
     "if (c2 < P.int_chi2) cands.push_back({c2, id});",
     "tests/test_oracle_fit_pins.py::test_inward_extrapolation_recovers_inner_segments"),
    ("cluster removal: looper legs required to have the same charge sign",
     "if ((qa > Real(0)) == (qb > Real(0))) continue;",
     "if ((qa > Real(0)) != (qb > Real(0))) continue;",
     "tests/test_oracle_removal_pins.py::test_secondary_legs_follow_generator_truth"),
    ("seeding iterations: start clusters of accepted tracklets left free",
     "        F.used[TL[i].start] = 1;\n", "",
     "tests/test_oracle_seeding_pins.py::test_second_iteration_equals_tracking_the_leftover_clusters"),
    ("cluster removal: interpolation of the tube centre shifted by a row",
     "const Real f = Real(r - rl) / Real(rh - rl);", "const Real f = Real(r - rl + 1) / Real(rh - rl);",
     "tests/test_oracle_removal_pins.py::test_tubes_equal_all_pairs_scan"),
    ("Kalman update: cross term of the covariance update dropped",
     "t.c[ci(i, j)] = t.c[ci(i, j)] - (k0[i] * h0[j] + k1[i] * h1[j]);",
     "t.c[ci(i, j)] = t.c[ci(i, j)] - (k0[i] * h0[j]);",
     "tests/test_oracle_pins.py::test_update_equals_information_form"),
    ("scattering: (1 + tan^2 lambda) not squared for tan lambda",
     "c[9] = c[9] + th2 * a * a;", "c[9] = c[9] + th2 * a;",
     "tests/test_oracle_pins.py::test_scattering_noise_matches_the_generated_random_walk"),
    ("B-spline: wrong coefficient in the second weight",
     "w[1] = (Real(3) * f3 - Real(6) * f2 + Real(4)) / Real(6);",
     "w[1] = (Real(3) * f3 - Real(6) * f2 + Real(3)) / Real(6);",
     "tests/test_oracle_fit_pins.py::test_spline_partition_of_unity_and_linear_reproduction"),
    ("interpolation: the stored inward estimate left out of the weighted mean",
     "const Real v0 = (wa00 * a[0] + wa01 * a[1]) + (wb00 * b[0] + wb01 * b[1]);",
     "const Real v0 = (wa00 * a[0] + wa01 * a[1]);",
     "tests/test_oracle_fit_pins.py::test_noise_free_helices_recovered_to_1e9_fp64"),
    ("merging: rotation into the neighbouring sector with the wrong sense",
     "if (ds == 1 && !rotate(t, 1, P, P.fit_max_snp)) return false;",
     "if (ds == 1 && !rotate(t, -1, P, P.fit_max_snp)) return false;",
     "tests/test_oracle_fit_pins.py::test_merging_restores_sector_crossing_tracks"),
    ("first ambiguity: chi2/ndf term of the score with the wrong sign",
     "const Real sc = Real(T.n) - P.score_w * (T.chi2 / Real(T.ndf));",
     "const Real sc = Real(T.n) + P.score_w * (T.chi2 / Real(T.ndf));",
     "tests/test_oracle_ambiguity_pins.py::"
     "test_tracklet_key_follows_its_definition_and_prefers_small_chi2"),
    ("track following: worst instead of best cluster of the window",
     "if (best < 0 || R.chi2 < bres.chi2 || (R.chi2 == bres.chi2 && id < best)) {",
     "if (best < 0 || R.chi2 > bres.chi2 || (R.chi2 == bres.chi2 && id < best)) {",
     "tests/test_oracle_ambiguity_pins.py::test_following_picks_the_best_cluster_of_the_window"),
    ("second ambiguity: largest instead of smallest bid",
     "if (it == bid.end() || key < it->second) bid[c] = key;",
     "if (it == bid.end() || key > it->second) bid[c] = key;",
     "tests/test_oracle_ambiguity_pins.py::test_second_ambiguity_hand_made_cases"),
    ("second ambiguity: rounds run from the last choice to the first",
     "  for (int k = 0; k < P.cand_k; ++k) {\n    bid.clear();",
     "  for (int k = P.cand_k - 1; k >= 0; --k) {\n    bid.clear();",
     "tests/test_oracle_ambiguity_pins.py::test_second_ambiguity_hand_made_cases"),
    ("edge following: rotation into the neighbouring sector on the wrong edge",
     "const int dir = t.p[0] > Real(0) ? 1 : -1;", "const int dir = t.p[0] > Real(0) ? -1 : 1;",
     "tests/test_oracle_edge_pins.py::test_short_segments_in_the_adjacent_sector_are_recovered"),
    ("central electrode: sign of the far side's z shift",
     "  dz = t.p[1] - B.ie.p[1];", "  dz = B.ie.p[1] - t.p[1];",
     "tests/test_oracle_electrode_pins.py::test_far_side_shift_measures_the_collision_time"),
]


def _run_case(tmp, i, what, orig, planted, pin):
    """Plant the mistake, build the variant, run its pin: '' if the pin fails."""
    text = open(SRC).read()
    if text.count(orig) != 1:
        return f"mutation site of '{what}' not found once"
    d = os.path.join(tmp, f"case{i}")
    os.makedirs(d)
    src = os.path.join(d, "oracle.cpp")
    with open(src, "w") as fh:
        fh.write(text.replace(orig, planted))
    lib = os.path.join(d, "liboracle_variant.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", src, "-o", lib])
    env = dict(os.environ, TPC_ORACLE_VARIANT_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        pin], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return "" if r.returncode == 1 else f"pin did not catch '{what}':\n{r.stdout[-1500:]}"


def test_pins_catch_planted_mistakes(tmp_path):
    """All cases at once (each is a compile and a pytest run of its own)."""
    from concurrent.futures import ThreadPoolExecutor

    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    with ThreadPoolExecutor(max_workers=max(1, min(len(CASES), os.cpu_count() or 1))) as ex:
        errors = list(ex.map(lambda ic: _run_case(str(tmp_path), ic[0], *ic[1]), enumerate(CASES)))
    errors = [e for e in errors if e]
    assert not errors, "\n\n".join(errors)
