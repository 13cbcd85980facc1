import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running test")


@pytest.fixture
def parity_log():
    """record(name, entry): add an entry to the JSON file MBS_PARITY_OUT names
    (no-op when unset) -- the per-result errors against the oracle and the
    FP64 path that the bench line and the design notes quote."""
    import json

    def record(name, entry):
        path = os.environ.get("MBS_PARITY_OUT")
        if not path:
            return
        d = {}
        if os.path.exists(path):
            try:
                d = json.load(open(path))
            except ValueError:
                d = {}
        d[name] = entry
        with open(path, "w") as f:
            json.dump(d, f, indent=0)

    return record
