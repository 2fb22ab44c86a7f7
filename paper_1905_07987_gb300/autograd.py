"""torch.autograd bridge for the receiver misfit of the linear-elastic solver.

``receiver_misfit(mat, M, run, u0, t0, dt, steps, k_ckpt, obs)`` returns the scalar misfit
J = 1/2 dt sum |v_rec - obs|^2 as a differentiable function of the per-cell material ``mat``
[cells, 3] (rho, lambda, mu) and the moment tensor ``M`` [6].  The forward pass calls the
library's checkpointed forward + adjoint sweep (ader_misfit_gradient) once and keeps the
gradients; backward only scales them.  Argument marshalling only: every step runs in libader.
"""
import torch


class ReceiverMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mat, M, run, u0, t0, dt, steps, k_ckpt, obs):
        run.set_material(mat.detach().contiguous().view(-1))
        run.set_point_source(run.src_x0, M.detach().double().cpu().numpy(), run.src_f0, run.src_t0)
        need = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
        gm = torch.empty(mat.numel(), dtype=torch.float64, device=mat.device) if need else None
        gM = torch.empty(6, dtype=torch.float64, device=mat.device) if need else None
        J = run.misfit_gradient(u0.contiguous().view(-1), t0, dt, steps, k_ckpt,
                                obs.contiguous().view(-1), gm, gM)
        if need:
            ctx.save_for_backward(gm.view_as(mat), gM)
        ctx.M_device = M.device
        return torch.tensor(J, dtype=torch.float64, device=mat.device)

    @staticmethod
    def backward(ctx, gJ):
        gm, gM = ctx.saved_tensors
        return gJ * gm, (gJ * gM).to(ctx.M_device), None, None, None, None, None, None, None


def receiver_misfit(mat, M, run, u0, t0, dt, steps, k_ckpt, obs):
    return ReceiverMisfit.apply(mat, M, run, u0, t0, dt, steps, k_ckpt, obs)
