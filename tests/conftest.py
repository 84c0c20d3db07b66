import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running oracle comparison")


def golden_path(name: str) -> str:
    return os.path.join(ROOT, "tests", "golden", name)


def read_golden_kv(name: str) -> dict:
    out = {}
    with open(golden_path(name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = [s.strip() for s in line.split("=", 1)]
            try:
                out[k] = float(v) if "." in v else int(v)
            except ValueError:
                out[k] = v  # text values (digests)
    return out


@pytest.fixture(scope="session")
def orc16():
    import oracle

    o = oracle.Oracle(4)
    o.keygen(7)
    return o


@pytest.fixture(scope="session")
def orc4096():
    import oracle

    o = oracle.Oracle(12)
    o.keygen(2024)
    return o
