import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def ensure_library():
    """Build the CUDA library in-tree if needed and return the imported package."""
    import importlib.util
    path = os.path.join(ROOT, "paper_1502_03391_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("fjofc_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_1502_03391_gb300
    return paper_1502_03391_gb300
