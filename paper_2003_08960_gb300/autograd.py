"""torch.autograd front end of the aberration path.

``Sharpness.apply(coeffs, z, plan, frames)`` returns the sharpness loss
L = -sum P^2 / (sum P)^2 of the pupil-corrected volume as a float64 scalar
tensor; its backward pass hands back dL/dc_1..dL/dc_15 and dL/dz.  Both the
loss and the gradient come from one call of the C ABI (``ssoct_sharpness``: a
forward pass and a hand-written adjoint pass on the device), so backward does
no further device work.
"""

import torch


class Sharpness(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coeffs, z, plan, frames):
        c = coeffs.detach().to("cpu", torch.float64)
        loss, grad, _ = plan.sharpness(frames, c.tolist(), float(z))
        ctx.save_for_backward(torch.from_numpy(grad[1:].copy()), torch.tensor(grad[0], dtype=torch.float64))
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, g):
        gc, gz = ctx.saved_tensors
        return g * gc, g * gz, None, None


def sharpness(plan, frames, coeffs, z):
    """L(coeffs, z) with autograd support; coeffs (15,) and z () are float64 CPU tensors."""
    return Sharpness.apply(coeffs, z, plan, frames)
