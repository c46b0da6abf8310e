import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session", autouse=True)
def _checked_build_records_nothing():
    """With BS_LIBRARY=checked (the -DBS_CHECKED library, whose device bounds
    checks record a violation and skip the access) the whole session must end
    with no recorded violation.  test_gpu_checked.py plants violations on
    purpose in its own child processes; run it without this variable."""
    yield
    if os.environ.get("BS_LIBRARY") != "checked":
        return
    import torch
    import paper_2506_10526_gb300 as bs
    if bs._lib is None or not torch.cuda.is_available():  # nothing ran on a GPU
        return
    st = bs.checked_status(reset=False)
    assert st["violations"] == 0, f"checked build recorded out-of-range accesses: {st}"
