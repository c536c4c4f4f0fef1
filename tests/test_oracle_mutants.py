"""Planted mistakes in the oracle are caught by its pins.

The oracle source carries a few compile-time switches (OR_MUTANT = m) that each
plant one plausible mistake: a dropped term, a wrong sign, a transposed
operand, a wrong stencil or coefficient. Each mutant is built on the CPU and
the pins that target it must fail, which shows the pins are sharp enough.
"""
import pytest

import oracle_pins as P

MUTANTS = {
    1: ("feq: -u^2 term dropped", [P.check_feq_moments, P.check_cs_exact_rational, P.check_fd_high_precision]),
    2: ("feq: sign of v.u flipped", [P.check_feq_moments, P.check_cs_exact_rational, P.check_fd_high_precision]),
    3: ("CS: streams to x - c_k", [P.check_cs_streaming_direction, P.check_cs_exact_rational]),
    4: ("velocity components transposed", [P.check_set_ordering, P.check_cs_exact_rational,
                                           P.check_fd_high_precision]),
    5: ("WENO: mirrored third candidate", [P.check_weno_quadratic_exact, P.check_fd_high_precision]),
    6: ("RK3: wrong second-stage weights", [P.check_fd_rk3_relaxation, P.check_fd_high_precision]),
    7: ("WENO: downwind stencil for v > 0", [P.check_fd_linear_advection, P.check_fd_linear_modes,
                                            P.check_fd_high_precision]),
    8: ("WENO: wrong beta_2 coefficient", [P.check_weno_beta, P.check_fd_high_precision]),
    9: ("FD: BGK moments of every stage taken from f^n", [P.check_fd_high_precision, P.check_fd_linear_modes,
                                                          P.check_fd_decay_closed_form]),
    10: ("IMEX: implicit stages relax to the equilibrium of f^n", [P.check_imex_linear_modes,
                                                                   P.check_imex_high_precision]),
    11: ("IMEX: wrong gamma of the implicit tableau", [P.check_imex_relaxation, P.check_imex_linear_modes,
                                                       P.check_imex_high_precision]),
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_mutant_is_caught(mutant):
    what, checks = MUTANTS[mutant]
    for check in checks:
        with pytest.raises(AssertionError):
            check(mutant)
