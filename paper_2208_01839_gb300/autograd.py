"""torch.autograd bridge for the discrete adjoint of a SEIRD run.

``misfit(solver, u0, rates, beta_field, spec)`` returns the misfit of a run of
``spec['n_steps']`` backward-Euler steps from ``u0`` as a 0-d tensor; its
gradients with respect to ``rates`` (10 values, order ``seird.PARAM_NAMES``) and
``beta_field`` (per node) come from ``seird_adjoint``: the library computes
them together with the forward run, and backward only scales them.
"""
import numpy as np
import torch

from . import seird as S


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rates, beta_field, solver, u0, base_params, spec):
        vals = rates.detach().cpu().double().numpy()
        p = dict(base_params.as_dict() if hasattr(base_params, "as_dict") else base_params)
        for k, name in enumerate(S.PARAM_NAMES[:6]):
            p[name] = float(vals[k])
        p["nu"] = tuple(float(v) for v in vals[6:10])
        bf = None if beta_field is None else beta_field.detach().cpu().double().numpy()
        solver.set_params(p, beta_field=bf)
        solver.set_state(u0)
        j, g, gf = solver.adjoint(spec["n_steps"], spec["obs_nodes"], spec["obs_steps"], spec["I_hat"],
                                  spec["D_hat"], checkpoint_every=spec.get("checkpoint_every", 1),
                                  lin_rtol=spec.get("lin_rtol", 0.0), field=beta_field is not None)
        ctx.save_for_backward(torch.tensor(g, dtype=rates.dtype, device=rates.device),
                              torch.tensor(np.zeros(1) if gf is None else gf, dtype=rates.dtype,
                                           device=rates.device))
        ctx.has_field = beta_field is not None
        return torch.tensor(j, dtype=rates.dtype, device=rates.device)

    @staticmethod
    def backward(ctx, grad_out):
        g, gf = ctx.saved_tensors
        return grad_out * g, (grad_out * gf if ctx.has_field else None), None, None, None, None


def misfit(solver, u0, rates, beta_field, base_params, spec):
    return _Misfit.apply(rates, beta_field, solver, u0, base_params, spec)
