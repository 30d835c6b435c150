import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libfcs")


@pytest.fixture(scope="session")
def geo():
    from paper_2103_14737_gb300 import synth
    return synth.geometry()


@pytest.fixture(scope="session")
def prm(geo):
    from paper_2103_14737_gb300 import synth
    return synth.params(geo)


@pytest.fixture(scope="session")
def ogeo(geo):
    from oracle import oracle as O
    return O.OracleGeometry(geo)


@pytest.fixture(scope="session")
def oprm(prm):
    from oracle import oracle as O
    return O.OracleParams(prm)
