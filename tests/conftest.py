import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_cuda = torch.cuda.is_available()
    except Exception:
        have_cuda = False
    if have_cuda:
        return
    skip = pytest.mark.skip(reason="no CUDA device in this process")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(autouse=True)
def _checked_build_status():
    """Under the checked build (SAS_CHECKED=1) every handle's status word is
    read before the handle is destroyed, so an index check that fired in any
    launch fails the test that made it, whether or not the test synchronised."""
    if os.environ.get("SAS_CHECKED") != "1":
        yield
        return
    import paper_2101_05888_gb300 as sas
    orig = sas.Geometry.close

    def close(self):
        if getattr(self, "h", None):
            sas.sas_sync_status(self.h)
        orig(self)

    sas.Geometry.close = close
    try:
        yield
    finally:
        sas.Geometry.close = orig
