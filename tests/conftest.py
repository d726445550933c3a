"""Test configuration.

Markers: `gpu` tests need a CUDA device and the compiled library; everything
else runs on the CPU (oracle pins, host logic, library export checks).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libhr")
    config.addinivalue_line("markers", "slow: long-running CPU statistical test")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    """Rows of whitespace-separated tokens from tests/golden/<name>, skipping
    comment lines that start with '#'."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows
