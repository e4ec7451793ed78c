"""torch.autograd form of the grand potential (the differentiated form of the path).

``grand_potential(plan, rho, V, rho_bath)`` returns Omega/kT as a 0-d float64 tensor.  Its
backward is the library's hand-written gradient pass (dft_grad): the back-convolution
dOmega/drho = h^3 ln(rho/G(rho)), dOmega/dV = h^3 rho and dOmega/drho_bath, with the weighted
densities recomputed rather than stored.  Forward and backward run in the CUDA library; this
module only marshals tensors (and scales by the incoming gradient, as autograd requires).

The plan fixes the bath: ``rho_bath`` (nm^-3, shape (S,)) must equal the plan's bath densities;
it is an input only so that autograd can return dOmega/drho_bath.
"""
import numpy as np
import torch


class GrandPotential(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, V, rho_bath, plan):
        bath = plan.bulk()["rho"]
        if not np.allclose(rho_bath.detach().cpu().numpy(), bath, rtol=1e-12, atol=0.0):
            raise ValueError("rho_bath differs from the plan's bath densities")
        omega, _, _, _ = plan.grad(rho, V, want_rho=False, want_V=False, want_bulk=False)
        ctx.plan = plan
        ctx.save_for_backward(rho, V)
        ctx.bath_device = rho_bath.device
        return torch.tensor(omega, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, grad_omega):
        rho, V = ctx.saved_tensors
        need_rho, need_V, need_bath = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        _, d_rho, d_V, d_bath = ctx.plan.grad(rho, V, want_rho=need_rho, want_V=need_V, want_bulk=need_bath)
        g = grad_omega.detach()
        out_rho = d_rho * g.to(d_rho.dtype) if need_rho else None
        out_V = d_V * g.to(d_V.dtype) if need_V else None
        out_bath = (torch.tensor(d_bath, dtype=torch.float64, device=ctx.bath_device) * g.to(ctx.bath_device)
                    if need_bath else None)
        return out_rho, out_V, out_bath, None


def grand_potential(plan, rho, V, rho_bath=None):
    """Omega/kT of the plan's state point at (rho, V); differentiable in rho, V and rho_bath."""
    if rho_bath is None:
        rho_bath = torch.tensor(plan.bulk()["rho"], dtype=torch.float64)
    return GrandPotential.apply(rho, V, rho_bath, plan)
