"""md_set_allocator wired to PyTorch's caching allocator (needs a GB300): the
library's buffers come from torch's pool, results are unchanged, and the blocks go
back to the pool when the context is freed."""
import numpy as np
import pytest

from paper_1212_0262_gb300 import System
from paper_1212_0262_gb300.allocator import use_cuda_allocator, use_torch_allocator

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model,eps", [(0, 0.0), (1, 0.01), (2, 1e-3)])
def test_torch_allocator_gives_the_same_results(model, eps):
    import torch

    torch.cuda.init()
    ref = System(model, 5000, eps, 0.05, 3, precision="mixed")
    ref.step(10)
    qr, pr = ref.get_state()
    ref.close()
    base = torch.cuda.memory_allocated()
    use_torch_allocator()
    try:
        s = System(model, 5000, eps, 0.05, 3, precision="mixed")
        s.step(10)
        q, p = s.get_state()
        assert torch.cuda.memory_allocated() > base  # the buffers live in torch's pool
        s.close()
        assert torch.cuda.memory_allocated() == base  # and went back to it
    finally:
        use_cuda_allocator()
    assert np.array_equal(q, qr) and np.array_equal(p, pr)
