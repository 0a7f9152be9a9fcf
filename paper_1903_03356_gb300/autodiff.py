"""A capsule objective after T steps (the case's scheme, Kinematic or Dynamic) as a
differentiable torch function of the membrane constants and the driving force.

``CapsuleObjective.apply(k_s, k_b, g_x, case, nsteps, objective, storage, ckpt_every)``
returns J = D(T) (Taylor deformation) or a centroid coordinate of the case's first
capsule (Section 3.1) as a float64 tensor; its backward pass returns dJ/dk_s, dJ/dk_b,
dJ/dg_x from the library's reverse sweep (lbmib_adjoint). The initial state (the case's
fields and ring) does not depend on the parameters.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbmib


def context_for(case, ks: float, kb: float, gx: float, storage: str = "fp32"):
    """Context of ``case`` with capsule 0's k_s, k_b and the body force g_x replaced; the
    initial fields are the case's own."""
    cap = case.capsules[0]
    ctx = lbmib.Context(case.nx, case.ny, case.tau, case.walls, case.u_bottom, case.u_top, gx, case.gy,
                        storage=storage, max_capsules=len(case.capsules), max_nodes=case.n_nodes)
    ctx.init_fields(*case.fields())
    ctx.add_capsule(cap.xy, ks, kb, cap.ka, cap.mass)
    for other in case.capsules[1:]:
        ctx.add_capsule(other.xy, other.ks, other.kb, other.ka, other.mass)
    return ctx


class CapsuleObjective(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ks, kb, gx, case, nsteps, objective=lbmib.OBJ_TAYLOR_D, storage="fp32", ckpt_every=200):
        c = context_for(case, float(ks), float(kb), float(gx), storage)
        J, grad = c.adjoint(int(nsteps), objective=objective, capsule=0, ckpt_every=int(ckpt_every),
                            scheme=case.scheme)
        nc = len(case.capsules)
        g = torch.tensor([grad[0], grad[nc], grad[2 * nc]], dtype=torch.float64)
        fctx.save_for_backward(g)
        c.close()
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(fctx, gJ):
        (g,) = fctx.saved_tensors
        return gJ * g[0], gJ * g[1], gJ * g[2], None, None, None, None, None
