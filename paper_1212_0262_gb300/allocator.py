"""Route libmd's device allocations through PyTorch's caching allocator
(md_set_allocator), so the library shares the framework's memory pool instead of
calling cudaMalloc / cudaFree itself.

Only marshalling: the callbacks call torch.cuda.caching_allocator_alloc /
caching_allocator_delete.  Blocks come back 512-byte aligned, which meets the
library's 256-byte requirement; the library synchronises the device before it
hands a block back.
"""
from __future__ import annotations

import ctypes

from . import binding as B

_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_callbacks = None  # kept alive while installed


def use_torch_allocator(device: int | None = None) -> None:
    """Make libmd allocate device memory from torch's caching allocator (for
    allocations made after this call)."""
    import torch

    global _callbacks
    dev = torch.cuda.current_device() if device is None else int(device)

    def _alloc(nbytes, _user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev))
        except Exception:  # out of memory: the library reports MD_ENOMEM
            return None

    def _free(ptr, _user):
        torch.cuda.caching_allocator_delete(int(ptr))

    cbs = (_ALLOC_T(_alloc), _FREE_T(_free))
    rc = B.load().md_set_allocator(ctypes.cast(cbs[0], ctypes.c_void_p), ctypes.cast(cbs[1], ctypes.c_void_p), None)
    B.check(rc)
    _callbacks = cbs


def use_cuda_allocator() -> None:
    """Back to cudaMalloc / cudaFree for later allocations.  Blocks made through
    torch stay valid: each is freed by the allocator that made it."""
    rc = B.load().md_set_allocator(None, None, None)
    B.check(rc)
