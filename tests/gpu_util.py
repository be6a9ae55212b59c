"""Helpers shared by the GPU tests: device tensors in, numpy out."""
import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()
