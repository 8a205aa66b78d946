"""``torch.autograd.Function`` over a differentiable run of the terrain.

The forward records a run through ``crm_adjoint_forward`` (checkpoints every
``every`` steps); the backward hands the incoming gradients of the per-step
body wrench and centre and of the final SPH state to ``crm_adjoint_backward``
(recompute of each segment, then the hand-derived reverse sweep in the CUDA
library).  Tensors here are
FP64 host tensors: the run itself stays on the device inside the library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import GRAD_NAMES, from_scene


class TerrainRun(torch.autograd.Function):
    """(wrench, centre, x, u, sig, rho) = TerrainRun.apply(params, x0, u0, sig0, rho0,
    scene, n_steps, every).

    params: FP64 tensor in GRAD_NAMES order (E, nu, rho0, mu_s, cohesion,
    av_gamma, mu_2, I0, grain_d; mu_2 = mu_s turns mu(I) off, and then the
    gradient for mu_s is the one with mu_2 moving along); x0, u0, sig0, rho0: the
    initial SPH state
    (n, 3), (n, 3), (n, 6), (n,); scene: the ``scenes.Scene`` that supplies
    the walls, bodies and the other constants.  Returns the soil wrench
    (n_steps, n_bodies, 6) and the body centres (n_steps, n_bodies, 3) after
    each step, and the final SPH state.  Every tensor input receives its
    gradient."""

    @staticmethod
    def forward(ctx, params, x, u, sig, rho, scene, n_steps: int, every: int):
        sc = scene.copy()
        p = params.detach().cpu().double().numpy()
        for k, name in enumerate(GRAD_NAMES):
            sc.params[name] = float(p[k])
        sc.x = x.detach().cpu().double().numpy().copy()
        sc.u = u.detach().cpu().double().numpy().copy()
        sc.sig = sig.detach().cpu().double().numpy().copy()
        sc.rho = rho.detach().cpu().double().numpy().copy()
        t = from_scene(sc, skin=0.0)
        w, q = t.adjoint_forward(sc.dt, int(n_steps), int(every))
        xT, uT, sT, rT = t.particles()
        ctx.terrain = t
        out = [w, q[..., :3], xT, uT, sT, rT]
        return tuple(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)) for a in out)

    @staticmethod
    def backward(ctx, g_wrench, g_centre, g_x, g_u, g_sig, g_rho):
        t = ctx.terrain

        def host(g):
            return None if g is None else g.detach().cpu().double().numpy()
        g = t.adjoint_backward(host(g_wrench), host(g_centre), host(g_x), host(g_u), host(g_sig),
                               host(g_rho))
        ctx.terrain = None
        t.close()
        return (torch.from_numpy(g["params"].copy()), torch.from_numpy(g["xyz"].copy()),
                torch.from_numpy(g["vel"].copy()), torch.from_numpy(g["stress"].copy()),
                torch.from_numpy(g["rho"].copy()), None, None, None)


def scene_params(scene) -> torch.Tensor:
    """The scene's differentiable constants as a tensor in GRAD_NAMES order."""
    return torch.tensor([float(scene.params[n]) for n in GRAD_NAMES], dtype=torch.float64)
