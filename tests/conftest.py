import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long statistical run")


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")


def read_golden_numbers(path):
    out = {}
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()[:2]
                out[k] = float(v)
    return out


# Populations of the FP32 path against the oracle: the error of population a is measured
# against its scale w_a rho (rho the node's density), the size of the Hermite terms its value
# is summed from; a small population is a difference of such terms, so its own relative error
# is not the measure of the arithmetic. FP32 populations are held to 1e-5 of that scale.
LB_TOL_FP32 = 1e-5
LB_TOL_FP64 = 1e-12


def lb_err(gf, of, w):
    """Largest |gf - of| / (w_a rho) over populations a and nodes (rho = sum_a of)."""
    import numpy as np
    gf = np.asarray(gf, np.float64)
    of = np.asarray(of, np.float64)
    shape = (len(w),) + (1,) * (of.ndim - 1)
    rho = of.sum(0, keepdims=True)
    return float((np.abs(gf - of) / (np.asarray(w).reshape(shape) * np.abs(rho))).max())
