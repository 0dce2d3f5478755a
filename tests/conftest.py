"""Shared test configuration.

Markers: ``gpu`` -- needs a CUDA device (GB300); everything else runs on CPU.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: test needs a CUDA GPU (sm_103a)")


def load_golden(name: str) -> dict:
    """Parse a tests/golden/*.txt fixture: `key = v1, v2, ...` lines, '#' comments.
    Values are Python numeric literals (complex with j)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, vals = line.split("=", 1)
            items = [complex(v.strip().replace(" ", "")) for v in vals.split(",")]
            arr = np.array(items)
            if np.all(arr.imag == 0):
                arr = arr.real
            out[key.strip()] = arr
    return out


@pytest.fixture
def golden():
    return load_golden
