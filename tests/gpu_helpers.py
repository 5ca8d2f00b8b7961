"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
binding and compute the oracle's answer on the same seeded inputs."""
import numpy as np

import oracle


def torch_mod():
    import torch
    return torch


def run_gpu(g, shape, precision, soft=False, width=0.5, q_list=None, want_A=False):
    torch = torch_mod()
    import paper_2202_03411_gb300 as sm
    h = sm.scatman_create(g, precision, soft=soft, soft_width=width, q_list=q_list)
    n = sm.scatman_n_pix(h)
    f64 = precision == "fp64"
    I = torch.empty(n, dtype=torch.float64 if f64 else torch.float32, device="cuda")
    A = torch.empty(n, dtype=torch.complex128 if f64 else torch.complex64, device="cuda")
    sm.scatman_voxelise(h, shape)
    sm.scatman_forward(h, I, A)
    sm.scatman_sync(h)
    out = (I.cpu().double().numpy(), A.cpu().numpy().astype(np.complex128))
    if want_A:
        return out[0], out[1], h
    h.close()
    return out


def oracle_field(g, shape, q=None, soft=False, width=0.5, sample=None):
    """Oracle I and A on all pixels (or on the pixel indices in `sample`)."""
    if q is None:
        q = oracle.detector_q(g)
    if sample is not None:
        q = q[sample]
    chi, _ = oracle.voxelise(shape, g, soft, width)
    rho = oracle.slices(chi, g, shape.delta, shape.beta)
    A = oracle.msft(rho, q, g.voxel)
    return np.abs(A) ** 2, A


def rel_l2(x, ref):
    return oracle.relative_l2(x, ref)
