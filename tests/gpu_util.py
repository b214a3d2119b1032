"""Shared helpers for the GPU tests (skip cleanly without a GPU; never fall back)."""
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_05134_gb300 as kep
    kep.lib()
    return kep
