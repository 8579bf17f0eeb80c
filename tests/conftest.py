import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")
    config.addinivalue_line("markers", "emulation: the CUDA sources run on the CPU under the threaded emulator "
                                       "(opt-in: MBICG_EMULATION_TESTS=1)")


def pytest_collection_modifyitems(config, items):
    """The host-emulation layer (tests/test_host_emulation*.py: the library's
    CUDA sources compiled for the host and run one host thread per CUDA
    thread, also under the sanitizers) is a pre-check for machines without a
    GPU that takes tens of minutes; it runs when MBICG_EMULATION_TESTS=1 and
    is skipped otherwise, so that the default CPU suite stays within minutes."""
    on = os.environ.get("MBICG_EMULATION_TESTS", "") not in ("", "0")
    skip = pytest.mark.skip(reason="host emulation: set MBICG_EMULATION_TESTS=1 to run it")
    for item in items:
        if os.path.basename(str(item.fspath)).startswith("test_host_emulation"):
            item.add_marker(pytest.mark.emulation)
            if not on:
                item.add_marker(skip)


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def emulated_library(tmp_path_factory):
    """The test-only emulated library (tests/emulated_library.py), built once."""
    import emulated_library as el

    if not el.available():
        pytest.skip("g++ or the CUDA headers are missing")
    return el.build(str(tmp_path_factory.mktemp("library_emulation")))
