import os
import sys
import warnings

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    # scipy's quad emits IntegrationWarning on the kinked piecewise EOS; the
    # results are checked against tolerances in the tests themselves.
    warnings.filterwarnings("ignore", message=".*roundoff error.*")
    warnings.filterwarnings("ignore", message=".*extrapolation table.*")
