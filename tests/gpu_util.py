"""Helpers for the GPU tests: move seeded inputs to the device, build plans."""
import numpy as np
import torch

from paper_1306_0612_gb300 import lbfmm as L

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(DEV)


def host(t):
    return t.detach().cpu().numpy()


def plan_for(g, rotation=None, **opt):
    o = L.lbf_default_options(**opt)
    return L.lbf_plan_create(g.island_ptr, dev(g.x), dev(g.dx), dev(g.d2x), dev(g.centres),
                             pole_rotation=rotation, opt=o)


def zeros(n):
    return torch.zeros(n, dtype=torch.float64, device=DEV)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))
