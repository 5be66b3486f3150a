import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: oracle pins that take minutes; run with LBM_SLOW_PINS=1")


def pytest_collection_modifyitems(config, items):
    import pytest

    if os.environ.get("LBM_SLOW_PINS"):
        return
    skip = pytest.mark.skip(reason="slow oracle pin: set LBM_SLOW_PINS=1 to run it")
    for item in items:
        if "slow" in item.keywords:
            item.add_marker(skip)


def golden(name):
    """Parse a tests/golden text fixture into {key: [rows of floats]}."""
    out = {}
    from fractions import Fraction

    with open(os.path.join(HERE, "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out.setdefault(key, []).append([float(Fraction(v)) for v in vals])
    return out
