"""The stored expected values under tests/golden/ (written by
tests/golden/make_golden.py from the oracle alone) still come out of the
oracle: a regression pin on the oracle itself, and the fixed numbers the GPU
tests compare against."""
import numpy as np

from tests.golden import make_golden as mg


def test_full8_lowest4_reproduced():
    assert np.allclose(mg.full8_lowest4(), mg.read_full8(), rtol=0, atol=1e-12)


def test_h2o29_tables_reproduced():
    ref = mg.read_tables()
    got = mg.h2o29_tables()
    for kind, name in ((1, "singles"), (2, "doubles")):
        for key, val in got[kind].items():
            assert ref["%s.%s" % (name, key)] == val, (name, key)
