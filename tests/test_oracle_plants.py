"""The oracle's pins must catch plausible mistakes: each planted variant of the oracle (a
compile-time switch in the oracle source, built only here) has to fail at least one pin."""
import pytest

import oracle
import test_oracle_categorical as cat
import test_oracle_evolve as evo
import test_oracle_pins as pins

# plant id -> (description, pin calls that must not all pass)
PLANTS = {
    1: ("zero margin counted as true", [lambda o: pins.test_fig1b_points(o, 0),
                                        lambda o: pins.test_dense_form_agrees_on_boundaries(o, 0)]),
    2: ("'<' evaluated as a negated '>'", [lambda o: pins.test_nan_and_inf_compare_false(o),
                                           lambda o: pins.test_dense_form_agrees_on_boundaries(o, 1)]),
    3: ("pair condition reads the wrong feature", [lambda o: pins.test_fig1b_points(o, 0),
                                                   lambda o: pins.test_dense_form_agrees_on_boundaries(o, 2)]),
    4: ("last firing rule wins", [lambda o: pins.test_fig1b_points(o, 0)]),
    5: ("later rules not discounted", [lambda o: pins.test_soft_probabilities_sum_to_one(o)]),
    6: ("threshold gradient sign", [lambda o: pins.test_one_rule_one_condition_is_logistic_regression(o, 0, False)]),
    7: ("S used where 1 - S belongs in the adjoint", [lambda o: pins.test_adjoint_matches_central_differences(o, 0)]),
    8: ("a fractional category value keeps its code",
        [lambda o: cat.test_membership_edge_values(o, range(64), [1, 1, 1, 0, 1, 0, 0, 0, 0, 0, 0, 1, 1, 1, 0]),
         lambda o: cat.test_mixed_rulesets_match_isin_formulation(o, 0)]),
    9: ("category bits read in the wrong order", [lambda o: cat.test_membership_bit_order(o),
                                                   lambda o: cat.test_single_code_equals_band(o)]),
    10: ("evolution never adds a condition", [lambda o: evo.check_operator_mix(o)]),
    11: ("threshold drawn from the wrong feature", [lambda o: evo.check_thresholds_from_data(o)]),
    12: ("1 - q taken from log q alone at large margins",
         [lambda o: pins.test_large_margin_single_condition_closed_form(o, 0, False),
          lambda o: pins.test_large_margins_match_arbitrary_precision(o, 0)]),
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_pins_catch_planted_mistake(plant):
    desc, calls = PLANTS[plant]
    o = oracle.planted(plant)
    caught = 0
    for call in calls:
        try:
            call(o)
        except AssertionError:
            caught += 1
    assert caught == len(calls), f"plant {plant} ({desc}) escaped {len(calls) - caught} pin(s)"
