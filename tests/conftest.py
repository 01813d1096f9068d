import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session", autouse=True)
def _build_oracle():
    import oracle
    oracle.build()


GOLDEN_DIR = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    """Values printed in the paper, from tests/golden/<name>.txt ("key = value" lines,
    whitespace-separated numbers become lists; '#' starts a comment)."""
    out = {}
    with open(os.path.join(GOLDEN_DIR, name + ".txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (x.strip() for x in line.split("=", 1))
            parts = v.split()
            try:
                nums = [float(x) for x in parts]
                nums = [int(x) if x.is_integer() else x for x in nums]
                out[k] = nums[0] if len(nums) == 1 else nums
            except ValueError:
                out[k] = parts if len(parts) > 1 else v
    return out
