"""The oracle pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle source (never in the
oracle itself), compiles it, and checks that at least one pin of
test_oracle_pins (hand-derived values, exact plane recovery, sphere
convergence order) rejects it.
"""
import os

import numpy as np
import pytest

import oracle
from tests import test_oracle_pins as pins
from tests import test_oracle_points as point_pins
from tests import test_oracle_sep5 as sep5_pins
from tests import test_oracle_weighted as weighted_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "tfn_oracle.c")

MUTANTS = {
    "candidate_sign": ("cand = ((qx - px) * nx + (qy - py) * ny) / dz;",
                       "cand = ((qx - px) * nx - (qy - py) * ny) / dz;"),
    "dropped_neighbour_offset": ("double qx = Z[a][b] * (u + du - J->u0) / J->fx",
                                 "double qx = Z[a][b] * (u - J->u0) / J->fx"),
    "wrong_focal_in_backprojection": ("double px = Z[1][1] * (u - J->u0) / J->fx, py = Z[1][1] * (v - J->v0) / J->fy;",
                                      "double px = Z[1][1] * (u - J->u0) / J->fx, py = Z[1][1] * (v - J->v0) / J->fx;"),
    "swapped_principal_point": ("double qx = Z[a][b] * (u + du - J->u0) / J->fx, qy = Z[a][b] * (v + dv - J->v0) / J->fy;",
                                "double qx = Z[a][b] * (u + du - J->v0) / J->fx, qy = Z[a][b] * (v + dv - J->u0) / J->fy;"),
    "convolution_not_correlation": ("hu += delta[b] * (img[k][2 + b] - img[k][2 - b]);",
                                    "hu += delta[b] * (img[k][2 - b] - img[k][2 + b]);"),
    "transposed_vertical_filter": ("hv += delta[b] * (img[2 + b][k] - img[2 - b][k]);",
                                   "hv += delta[b] * (img[k][2 + b] - img[k][2 - b]);"),
    "upper_median": ("phi = (m & 1) ? c[m / 2] : 0.5 * (c[m / 2 - 1] + c[m / 2]);",
                     "phi = c[m / 2];"),
    "mean_divides_by_eight": ("phi = acc / m;", "phi = acc / 8;"),
    "no_dz_exclusion": ("if (dz == 0.0) continue; /* reading R4 */", ""),
    "orientation_away_from_camera": ("n0[idx] = -nx / len; /* reading R7 */\n    n1[idx] = -ny / len;\n    n2[idx] = -nz / len;",
                                     "n0[idx] = nx / len;\n    n1[idx] = ny / len;\n    n2[idx] = nz / len;"),
    "nz_sign": ("double nz = -phi;", "double nz = phi;"),
    "scharr_weights": ("case OR_SCHARR: w[0] = 3; w[1] = 10; w[2] = 3;",
                       "case OR_SCHARR: w[0] = 3; w[1] = 10; w[2] = 4;"),
    "sobel_weights": ("case OR_SOBEL: w[0] = 1; w[1] = 2; w[2] = 1;",
                      "case OR_SOBEL: w[0] = 1; w[1] = 1; w[2] = 1;"),
    # (Dropping f from Z = f t_c / d is no mistake: it rescales every depth
    # alike and the estimated direction is invariant to a global depth scale.)
    "disparity_gradient_on_inverse": ("(disparity ? s[a][b] : 1.0 / s[a][b])",
                                      "(disparity ? 1.0 / s[a][b] : 1.0 / s[a][b])"),
    "depth_instead_of_inverse": ("img[a][b] = ok[a][b] ? (disparity ? s[a][b] : 1.0 / s[a][b]) : 0.0;",
                                 "img[a][b] = ok[a][b] ? s[a][b] : 0.0;"),
    "prewitt_weights": ("default: w[0] = 1; w[1] = 1; w[2] = 1; break;",
                        "default: w[0] = 1; w[1] = 2; w[2] = 1; break;"),
    "nx_without_focal": ("else { nx = J->fx * gu; ny = J->fy * gv; }", "else { nx = gu; ny = J->fy * gv; }"),
    # the back-projected point cloud
    "points_wrong_focal": ("Y = Z * (v - v0) / fy;", "Y = Z * (v - v0) / fx;"),
    "points_swapped_principal_point": ("X = Z * (u - u0) / fx;", "X = Z * (u - v0) / fx;"),
    "points_disparity_without_baseline": ("Z = disparity ? fx * tc / s : s;", "Z = disparity ? fx / s : s;"),
    # the weighted filter family
    "weighted_reversed": ("w[0] = custom[0]; w[1] = custom[1]; w[2] = custom[2];",
                          "w[0] = custom[2]; w[1] = custom[1]; w[2] = custom[0];"),
    "weighted_ignores_weights": ("w[0] = custom[0]; w[1] = custom[1]; w[2] = custom[2];",
                                 "w[0] = 1; w[1] = 2; w[2] = 1;"),
    # the 5x5 separable family
    "fd5_profile_swapped": ("case OR_FD5: d1 = 8; d2 = -1;", "case OR_FD5: d1 = -1; d2 = 8;"),
    "sobel5_smoothing_order": ("case OR_SOBEL5: d1 = 2; d2 = 1; s0 = 6; s1 = 4; s2 = 1;",
                               "case OR_SOBEL5: d1 = 2; d2 = 1; s0 = 4; s1 = 6; s2 = 1;"),
    "sep5_smoothing_reversed": ("rho[0] = s2; rho[1] = s1; rho[2] = s0; rho[3] = s1; rho[4] = s2;",
                                "rho[0] = s0; rho[1] = s1; rho[2] = s2; rho[3] = s1; rho[4] = s0;"),
    "sep5_outer_taps_at_offset_one": ("hu += delta[b] * (img[k][2 + b] - img[k][2 - b]);",
                                      "hu += delta[b] * (img[k][3] - img[k][1]);"),
    "sep5_norm_drops_d2": ("*norm = 2 * (d1 + 2 * d2) *", "*norm = 2 * (d1 + d2) *"),
    "sep5_outer_taps_not_required": ("(rho[a] != 0 && du != 0 && delta[abs(du)] != 0)",
                                     "(rho[a] != 0 && abs(du) == 1 && delta[abs(du)] != 0)"),
    "no_candidate_not_special": ("    if (m == 0) { /* reading R6: every valid neighbour at the centre's depth */\n        n0[idx] = 0.0; n1[idx] = 0.0; n2[idx] = -1.0;\n        return;\n    }",
                                 "    if (m == 0) { c[m++] = 0.0; }"),
    "points_keep_holes": ("double X = 0, Y = 0, Z = 0;\n            if (ok) {", "double X = 0, Y = 0, Z = 0;\n            if (1) {"),
}


def _pins_fail(lib):
    if pins.check_golden(lib):
        return True
    if point_pins.check_points(lib):
        return True
    if weighted_pins.check_weighted(lib):
        return True
    if sep5_pins.check_sep5(lib):
        return True
    for grad in pins.GRADS:
        for phi in pins.PHIS:
            if not (pins.plane_max_error(grad, phi, lib, H=16, W=20) < 1e-9):
                return True
    for phi in pins.PHIS:
        o = pins.sphere_orders(phi, lib)
        if not all(1.8 <= x <= 2.3 for x in o):
            return True
    return False


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = oracle.open_library(oracle.compile_to(str(mutant), str(tmp_path / "libmutant.so")))
    with np.errstate(all="ignore"):
        assert _pins_fail(lib), f"mutant {name} passes every pin"


def test_unmutated_copy_passes(tmp_path):
    lib = oracle.open_library(oracle.compile_to(SRC, str(tmp_path / "libsame.so")))
    assert not _pins_fail(lib)
