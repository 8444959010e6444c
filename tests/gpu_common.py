"""Helpers shared by the GPU tests."""
import numpy as np
import pytest
import torch

from paper_2609_19116_b300 import build

_built = False


def lib_ready():
    global _built
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not _built:
        if build.needs_build():
            build.build()
        _built = True
    import paper_2609_19116_b300 as q
    return q


def dev_shots(shots):
    return torch.tensor(np.asarray(shots, dtype=np.int64), dtype=torch.int64, device="cuda")


def kept_bits(mask_words, nshots):
    w = mask_words.cpu().numpy().view(np.uint64)
    bits = np.unpackbits(w.view(np.uint8), bitorder="little")
    return bits[:nshots].astype(bool)
