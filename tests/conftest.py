import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (runs the CUDA library)")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def gmco_mod():
    from paper_1904_01567_b300.build import build
    build()
    import paper_1904_01567_b300 as g
    return g


def read_fstar(name):
    path = os.path.join(ROOT, "tests", "golden", f"fstar_{name}.txt")
    out = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                continue
            a = line.split()
            out[int(a[0])] = float(a[1])
    return out
