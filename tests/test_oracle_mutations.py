"""The pins catch plausible mistakes in the oracle.  Each case builds the
oracle with one mistake planted at a test-only mutation point of the C
source (ORC_MUTATION = k; the default build has none), routes the oracle's
wrappers to that build and checks that a pin of tests/test_oracle_pins.py
fails; the default build is restored afterwards.
"""
import pytest

import oracle
import test_oracle_pins as pins

# k: (the planted mistake, the pin that must catch it, its arguments)
MUTANTS = {
    1: ("projection without the z term", "test_bin_contract_brute_force_rational", {}),
    2: ("contract bins one bin low", "test_bin_closed_forms", {"m": 8}),
    3: ("DFT at frequency k + 1 instead of k", "test_spectrum_closed_forms", {}),
    4: ("Eq. 1 without the pad bin dR", "test_bin_eq1_matches_exact_eq1_and_contract_moves_only_boundary_atoms", {}),
    5: ("Eq. 3 with |difference| instead of its square", "test_match_recovers_planted_orientation", {}),
    6: ("membership test with the y coordinate in place of x", "test_gather_matches_kdtree_ball", {}),
    7: ("Eq. 2 with the k_x and k_y roles swapped", "test_fsp_matches_brute_force_and_lattice_peaks", {}),
    8: ("band maximum keeping the highest k on ties", "test_signature_is_band_max_with_lowest_argk", {}),
    9: ("refinement Jacobian with the wrong sign", "test_refine_gradient_matches_finite_differences", {}),
    10: ("strongest nodes with equal values in descending index order", "test_top_nodes_order_and_ties", {}),
    11: ("look-up table holding the farthest node instead of the nearest", "test_lut_is_nearest_node", {}),
    12: ("disorientation over 23 of the 24 proper cubic rotations", "test_disorientation_textbook_values", {}),
    13: ("normalisation by the row sum instead of the row maximum",
         "test_normalise_divides_each_row_by_its_maximum", {}),
    14: ("rotation matrix transposed", "test_quat_to_matrix_matches_axis_angle_rodrigues", {}),
    15: ("bilinear weights of the two image columns swapped",
         "test_bilinear_reproduces_grid_values_and_is_linear_inside_cells", {}),
    16: ("band edges rounded outwards", "test_band_interval_reproduces_paper_al_200", {}),
    17: ("Eq. 2 grid spacing 2 k_max / L instead of 2 k_max / (L - 1)", "test_fsp_closed_forms", {}),
    18: ("Gauss-Newton step with the wrong sign", "test_refine_converges_to_truth", {}),
    19: ("atom type bits read one position off", "test_gather_type_mask", {}),
    20: ("reference nodes rotated by the transposed matrix", "test_lut_is_nearest_node", {}),
    21: ("DFT twiddle angles over N_b - 1 instead of N_b", "test_spectrum_matches_numpy_rfft", {"m": 8}),
    22: ("candidate score summed over its channels instead of averaged",
         "test_match_phase_reduces_to_eq3_and_averages_channels", {}),
    23: ("every channel of a candidate reads the measured signature of its first channel",
         "test_match_phase_recovers_planted_candidate", {}),
    24: ("channel differences not divided by the reference's energy",
         "test_match_phase_empty_signature_scores_one", {}),
}


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_pins_catch_planted_mistake(k):
    what, pin, kw = MUTANTS[k]
    oracle.use_library(oracle.build_mutant(k))
    try:
        with pytest.raises(AssertionError):
            getattr(pins, pin)(**kw)
    finally:
        oracle.use_library(None)
    getattr(pins, pin)(**kw)          # and the default build passes it
