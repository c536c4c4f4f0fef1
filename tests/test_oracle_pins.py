"""The FP64 oracle against what the paper and the mathematics fix (CPU only).

Each check is documented in tests/oracle_pins.py; together they cover every
routine of oracle/lbm_oracle.c and the host helpers in oracle/__init__.py.
"""
import pytest

import oracle_pins as P


@pytest.mark.parametrize("check", P.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(check):
    check(0)
