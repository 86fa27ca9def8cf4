import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter):
    """The parity log names the oracle's join path: the nested loop below its
    cap, its own sort-merge join above it."""
    mod = sys.modules.get("oracle.oracle")
    if mod is not None and any(mod.JOIN_PATHS.values()):
        terminalreporter.write_line(
            "oracle joins: {nested} nested-loop, {sortmerge} sort-merge".format(**mod.JOIN_PATHS))
