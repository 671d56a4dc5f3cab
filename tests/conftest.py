import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running check")


@pytest.fixture(scope="session")
def mechdir(tmp_path_factory):
    return str(tmp_path_factory.mktemp("mech"))


@pytest.fixture(scope="session")
def mech_path(mechdir):
    from paper_2411_02640_gb300 import synth

    def get(name):
        return synth.mechanism_file(name, mechdir)
    return get


@pytest.fixture(scope="session")
def oracle_for(mech_path):
    import oracle
    cache = {}

    def get(name):
        if name not in cache:
            cache[name] = oracle.Oracle(mech_path(name), nthreads=min(8, os.cpu_count() or 1))
        return cache[name]
    return get
