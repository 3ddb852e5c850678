"""Shared pytest set-up: the ``gpu`` marker and the repository root on sys.path."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (the sm_103a library)")


@pytest.fixture(autouse=True)
def _restore_library_options(request):
    """GPU tests may set process-wide library options (directly or through the
    autotuner); put them back afterwards so no test depends on another's settings."""
    if "gpu" not in request.keywords:
        yield
        return
    saved, m = None, None
    try:
        from paper_1604_06697_gb300 import build
        build.build()
        import paper_1604_06697_gb300 as m
        saved = {k: m.get_option(k) for k in m.OPTIONS}
    except Exception:
        saved = None
    yield
    if saved:
        for k, v in saved.items():
            m.set_option(k, v)


def pytest_collection_modifyitems(config, items):
    has_gpu = None
    for item in items:
        if "gpu" in item.keywords:
            if has_gpu is None:
                try:
                    import torch
                    has_gpu = torch.cuda.is_available()
                except Exception:
                    has_gpu = False
            if not has_gpu:
                item.add_marker(pytest.mark.skip(reason="no CUDA device"))
