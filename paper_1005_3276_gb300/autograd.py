"""torch.autograd.Function over the library's hand-written adjoint force kernel.

PseudofermionAction.apply(lat, phi, eta) returns S = S_pf (+ S_B) at phi; its
backward returns grad_output * dS/dphi as one complex tensor whose real and
imaginary parts are dS/dphi_R and dS/dphi_I -- the convention PyTorch uses for
the gradient of a real function of a complex tensor.  The force comes from
wz_force (the adjoint kernel of the fermion matrix plus the bosonic force of
Eq. acws); no FFT intermediates are stored: forward computes the action and
the force together and keeps only the force (one complex number per site).
"""

import torch

from . import binding


class PseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lat, phi, eta, tol=1e-10, bosonic=False):
        if phi.dtype != torch.complex128:
            raise TypeError("phi must be complex128")
        lat.set_phi(phi.detach().contiguous())
        grad = torch.empty_like(phi, memory_format=torch.contiguous_format)
        parts = binding.WZ_FORCE_FERMION | (binding.WZ_FORCE_BOSON if bosonic else 0)
        sb, spf, _ = lat.force(eta.detach().contiguous(), grad, tol=tol, parts=parts)
        ctx.save_for_backward(grad)
        return torch.tensor(spf + (sb if bosonic else 0.0), dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return None, grad_out.to(grad.device) * grad, None, None, None
