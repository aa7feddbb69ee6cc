import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")


@pytest.fixture(scope="session")
def oracle():
    # The mutation tests point RESAMPLE_ORACLE_PY at a copy of oracle.py with
    # a planted mistake (and RESAMPLE_ORACLE_LIB at the built C library).
    path = os.environ.get("RESAMPLE_ORACLE_PY")
    if path:
        import importlib.util
        spec = importlib.util.spec_from_file_location("oracle_mutant", path)
        o = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(o)
        return o
    from oracle import oracle as o
    o.build()
    return o
