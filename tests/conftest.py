import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# BO_ORACLE_PATH names a directory holding an altered copy of the oracle
# package, imported in place of the repository's (planted-mistake checks)
if os.environ.get("BO_ORACLE_PATH"):
    sys.path.insert(0, os.environ["BO_ORACLE_PATH"])


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled solver library")
    config.addinivalue_line("markers", "slow: larger CPU cases")
