import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def read_golden(name):
    """Parse a tests/golden fixture: '#' comments, 'key value' scalars, and blocks of
    numbers introduced by a bare key line."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out, cur = {}, None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            try:
                nums = [float(x) for x in parts]
            except ValueError:
                nums = None
            if nums is None:
                if len(parts) == 2:
                    out[parts[0]] = float(parts[1])
                    cur = None
                else:
                    cur = parts[0]
                    out[cur] = []
            else:
                out[cur].append(nums)
    return out


@pytest.fixture
def golden():
    return read_golden
