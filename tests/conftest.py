import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libmot.so")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def pr1_ops():
    """PR1: icosphere level 1, eps_r = 2, c dt = 0.2."""
    from paper_2510_07989_gb300.inputs.meshes import icosphere
    from paper_2510_07989_gb300.inputs.assemble import assemble
    return assemble(icosphere(1), 2.0, 1.0, 0.2)


@pytest.fixture(scope="session")
def pr1_system(pr1_ops):
    from oracle import mot as O
    return O.build_system(pr1_ops)


def _golden_rows(name):
    path = os.path.join(ROOT, "tests", "golden", name)
    return [ln.split() for ln in open(path) if ln.strip() and not ln.lstrip().startswith("#")]


def golden_table(name):
    """Rows of a table the paper prints, from tests/golden/<name> (the file cites its passage)."""
    return _golden_rows(name)


def golden_values(name):
    """key -> value (float, or tuple of floats) from tests/golden/<name> (the file cites its passage)."""
    out = {}
    for r in _golden_rows(name):
        vals = tuple(float(x) for x in r[1:])
        out[r[0]] = vals[0] if len(vals) == 1 else vals
    return out
