import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libpdot.so")
    config.addinivalue_line("markers", "slow: long-running test")


MUTANT_ENV = "PDOT_ORACLE_MUTANT"


@pytest.fixture(scope="session")
def ora():
    import oracle
    mutant = os.environ.get(MUTANT_ENV)
    if mutant:
        # Mutation check of the pins (tests/test_oracle_mutations.py): run them
        # against a prebuilt copy of the oracle with one planted mistake, and cap
        # every solve's pass budget (the unmodified oracle needs < 3000 passes in
        # any pin) so a mutant that stops converging fails fast.
        oracle._SRC, oracle._LIB, oracle._lib = mutant + ".c", mutant + ".so", None
        solve = oracle.solve

        def capped(C, f, g, opts=None, *a, **kw):
            import dataclasses
            opts = dataclasses.replace(opts or oracle.Options())
            opts.max_passes = min(opts.max_passes, 50_000)
            return solve(C, f, g, opts, *a, **kw)

        oracle.solve = capped
        return oracle
    oracle.build()
    return oracle
