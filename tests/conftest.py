import os
import re
import shutil
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libtsqbx")


def pytest_collection_modifyitems(config, items):
    # a file of its own runs last (kept last regardless of -p ordering plugins)
    last = [i for i in items if "test_zz_" in i.nodeid]
    rest = [i for i in items if "test_zz_" not in i.nodeid]
    items[:] = rest + last


@pytest.fixture(scope="session")
def rng():
    return np.random.default_rng(12345)


@pytest.fixture
def scratch(request):
    """A fresh working directory inside the repository (git-ignored), removed
    after the test: builds of planted-mistake copies and result files."""
    name = re.sub(r"[^A-Za-z0-9_.-]+", "_", request.node.nodeid)[-120:]
    d = os.path.join(ROOT, "tests", "native", "_build", "scratch", name)
    shutil.rmtree(d, ignore_errors=True)
    os.makedirs(d)
    yield __import__("pathlib").Path(d)
    shutil.rmtree(d, ignore_errors=True)
