"""Small helpers shared by the tests: moving numpy arrays to and from torch
device tensors without changing their bits."""
import numpy as np


def to_dev(a, device="cuda"):
    import torch

    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32).copy()).to(device)
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64).copy()).to(device)
    raise TypeError(a.dtype)


def to_np(t, dt):
    return t.detach().cpu().numpy().view(dt)


def header_functions(path):
    """Names of the functions a C header declares (ISORT_API prototypes)."""
    import re

    txt = open(path).read()
    return sorted(set(re.findall(r"ISORT_API\s+[\w\s\*]+?\b(isort_\w+)\s*\(", txt)))
