import os
import sys

# triton is only used as an independent CPU implementation of Philox (interpreter mode);
# the flag must be set before anything imports triton.
os.environ.setdefault("TRITON_INTERPRET", "1")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def rsctx():
    """One library context on cuda:0 for the GPU tests (fails loudly without the built library)."""
    import torch
    from paper_1602_02350_gb300 import Context, lib
    lib()
    ctx = Context(0)
    yield ctx
    torch.cuda.synchronize()
    ctx.close()
