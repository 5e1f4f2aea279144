import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the CUDA library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~20 s")


def golden(name):
    return os.path.join(ROOT, "tests", "golden", name)


def paper_values():
    out = {}
    with open(golden("paper_values.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            out[parts[0]] = (float(parts[1]), float(parts[2]))
    return out
