"""The paper's printed values (tests/golden/paper_values.txt) against the oracle's
data and against their own closed forms."""
import math

import numpy as np
import pytest

import oracle as O
from tests.helpers import golden


@pytest.mark.parametrize("name", ["A", "B", "C"])
def test_oracle_tableaux_are_the_printed_ones(name):
    t = O.SCHEMES[name]
    A = t["A"]
    assert A[1, 0] == pytest.approx(golden("scheme_%s_a21" % name), abs=1e-15)
    assert A[2, 0] == pytest.approx(golden("scheme_%s_a31" % name), abs=1e-15)
    assert A[2, 1] == pytest.approx(golden("scheme_%s_a32" % name), abs=1e-15)
    assert np.allclose(t["b"], golden("scheme_%s_b" % name), atol=1e-15)
    assert np.allclose(t["c"], golden("scheme_%s_c" % name), atol=1e-15)
    # strictly lower triangular, rows summing to the nodes (the paper's tableaux are consistent)
    assert np.allclose(np.triu(A), 0.0) and np.allclose(A.sum(1), t["c"], atol=1e-15)


def test_saffman_beta0_closed_form():
    g = golden("euler_gamma")
    assert g == pytest.approx(np.euler_gamma, abs=1e-6)
    assert golden("saffman_beta0") == pytest.approx(0.5 * (1 - np.euler_gamma + math.log(2)), abs=1e-6)
