"""Shared helpers for the GPU tests: upload synthetic meshes, run the oracle on the same inputs."""
import numpy as np

import synthetic
from oracle import fem

RULES = {"gll": 0, "gauss": 1}


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_mesh(ceed, m, qkind="gll", ncomp=1, dirichlet=True, device="cuda", coords=None):
    import torch
    return ceed.ceed_setup_mesh(m.n_elem, m.n_ldof, m.p, torch.from_numpy(m.elem_dofs).to(device),
                                torch.from_numpy(m.vertices).to(device),
                                torch.from_numpy(m.boundary).to(device) if dirichlet else None,
                                q_rule=RULES[qkind], ncomp=ncomp,
                                coords=None if coords is None else torch.from_numpy(coords).to(device))


def curved_coords(m, amplitude=0.05):
    """Node positions [n_ldof, 3] of a curved mesh: the trilinear nodes moved by the bubble warp (oracle side)."""
    return synthetic.bubble_warp(fem.global_node_points(m.p, m.vertices, m.elem_dofs, m.n_ldof), amplitude)


def oracle_qdata(m, qkind, op, coeff):
    sp_ = fem.Space(m.p, qkind)
    if op == "mass":
        rho = None
        if coeff == "sine":
            X, _ = fem.trilinear_map(m.vertices, sp_.XI)
            rho = fem.coeff_sine(X)
        elif isinstance(coeff, np.ndarray):
            rho = coeff
        return sp_, fem.qdata_mass(sp_, m.vertices, rho)
    return sp_, fem.qdata_diffusion(sp_, m.vertices, coeff)
