"""Helpers shared by the GPU tests (marshalling only)."""
import numpy as np
import torch

import paper_1909_09825_gb300 as fgt


def gpu_transform(plan, x, y, a, dev="cuda:0"):
    d = torch.device(dev)
    u = fgt.transform(plan, torch.from_numpy(np.ascontiguousarray(x)).to(d),
                      torch.from_numpy(np.ascontiguousarray(y)).to(d),
                      torch.from_numpy(np.ascontiguousarray(a)).to(d))
    return u.cpu().numpy()


def rel_inf(u, ref, a):
    """||u - ref||_inf / sum_j |alpha_j| (the tolerance metric of the transform)."""
    s = np.sum(np.abs(a))
    return float(np.max(np.abs(u - ref)) / s) if len(u) else 0.0
