import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")
    # temporary files of the tests stay inside the repository (git-ignored _build/)
    if not config.option.basetemp:
        config.option.basetemp = os.path.join(ROOT, "_build", "pytest_tmp")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
