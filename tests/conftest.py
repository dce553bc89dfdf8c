import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")
    config.addinivalue_line("markers", "run_last: run after every other collected test")


def pytest_collection_modifyitems(session, config, items):
    """Tests marked run_last go to the end of the run (stable otherwise), so that a run that
    stops at the first failure has already run everything else when one of them fails."""
    items[:] = [i for i in items if i.get_closest_marker("run_last") is None] + \
               [i for i in items if i.get_closest_marker("run_last") is not None]


def read_golden(name):
    """Rows of a whitespace-separated golden fixture, comments stripped."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O

    O.build()
    return O
