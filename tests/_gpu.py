"""GPU-test helpers: build/load libadcomb and move numpy arrays to and from the device."""
import numpy as np
import torch

from paper_2310_03568_gb300 import adcomb
from paper_2310_03568_gb300.build import build

_built = False


def ensure_lib():
    global _built
    if not _built:
        build()
        adcomb.lib()
        _built = True
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()
