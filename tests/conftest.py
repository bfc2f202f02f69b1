import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built fg21 library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


import json as _json


def report(name: str, **vals):
    """Append measured error statistics to $FG21_PARITY_REPORT (if set)."""
    path = os.environ.get("FG21_PARITY_REPORT")
    if not path:
        return
    rec = {"test": name}
    for k, v in vals.items():
        try:
            rec[k] = float(v)
        except (TypeError, ValueError):
            rec[k] = str(v)
    with open(path, "a") as fh:
        fh.write(_json.dumps(rec) + "\n")


@pytest.fixture(scope="session")
def fg21lib():
    """The built library on a GPU machine (GPU tests only)."""
    from paper_2603_13196_gb300 import fg21
    import __graft_entry__
    __graft_entry__.build()
    if fg21.fg21_device_count() < 1:
        pytest.fail("GPU test collected on a machine without a CUDA device")
    return fg21
