"""Oracle for Blocked Bloom filters with choices (arXiv 2501.18977).

TEST INFRASTRUCTURE ONLY. A plain, slow, single-threaded CPU statement of the
method (C, bit by bit, costs in double) plus the closed forms the paper prints.
Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import it; the product library never does, and this package never imports the
product.

Every oracle function is pinned by a test against something other than
itself (printed values, closed forms, invariants, brute force); see
``tests/test_oracle_pins.py``.
"""
from .oracle import (OracleFilter, COST_MIX, COST_LA, COST_EXP, COST_TABLE, derive_multipliers,
                     hash_lin, cost, bit_positions, splitmix64_next)
from . import closed_forms

__all__ = ["OracleFilter", "COST_MIX", "COST_LA", "COST_EXP", "COST_TABLE", "derive_multipliers",
           "hash_lin", "cost", "bit_positions", "splitmix64_next", "closed_forms"]
