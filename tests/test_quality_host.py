"""RelMSE as the quality harness computes it (no GPU)."""
import numpy as np


def test_relmse_definition():
    from paper_2607_23122_gb300 import quality as Q
    ref = np.array([[0.5, 0.0], [1.0, 0.2]])
    est = np.array([[0.4, 0.1], [1.0, 0.2]])
    valid = np.array([[True, True], [True, False]])
    want = np.mean([0.01 / (0.25 + 1e-3), 0.01 / (0.0 + 1e-3), 0.0])
    assert abs(Q.relmse(est, ref, valid) - want) < 1e-12
