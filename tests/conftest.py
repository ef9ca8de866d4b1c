import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300) and the built CUDA library")


@pytest.fixture(scope="session")
def model_dir(tmp_path_factory):
    return str(tmp_path_factory.mktemp("models"))


@pytest.fixture(scope="session")
def tiny_model_path(model_dir):
    from paper_2511_11337_b300 import synth
    return synth.make_model_file(os.path.join(model_dir, "tiny.boaw"), synth.TINY, seed=1)


@pytest.fixture(scope="session")
def uniform_model_path(model_dir):
    from paper_2511_11337_b300 import synth
    return synth.make_model_file(os.path.join(model_dir, "uniform.boaw"), synth.TINY, seed=2, zero_head=True)


@pytest.fixture(scope="session")
def peaked_model_path(model_dir):
    from paper_2511_11337_b300 import synth
    return synth.make_model_file(os.path.join(model_dir, "peaked.boaw"), synth.TINY, seed=3, head_scale=50.0)
