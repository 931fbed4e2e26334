"""GPU test helpers: move synthetic numpy TTs to the device and back."""
import numpy as np
import torch


def dev():
    return torch.device("cuda:0")


def to_dev(tt):
    return [torch.from_numpy(np.ascontiguousarray(c, dtype=np.float64)).to(dev()) for c in tt]


def to_host(tt):
    torch.cuda.synchronize()
    return [c.detach().cpu().numpy().astype(np.float64) for c in tt]


def const_ranks(N, r):
    return [1] + [r] * (N - 1) + [1]
