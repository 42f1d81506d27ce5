import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def build_library():
    """Compile libadc_gb300.so if needed (build.py loaded by path, not via the package)."""
    import importlib.util
    path = os.path.join(ROOT, "paper_2511_21640_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("_adc_gb300_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()
