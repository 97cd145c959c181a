import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~20 s")


@pytest.fixture(scope="session")
def oracle_cfg1():
    from oracle.pipeline import OracleRun
    from paper_1812_07437_gb300 import workloads
    return OracleRun(workloads.get("cfg1_1bin"))


@pytest.fixture(scope="session")
def oracle_tiny():
    from oracle.pipeline import OracleRun
    from paper_1812_07437_gb300 import workloads
    return OracleRun(workloads.get("tiny_2bin"))
