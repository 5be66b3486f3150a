"""Differentiable drainage: the saturation after n steps as a PyTorch
function of the per-voxel wettability field and the inlet density.

Forward runs the lattice through ``lbm_record`` (checkpoints every ``every``
steps); backward runs ``lbm_adjoint`` (the discrete adjoint of the step, with
each segment recomputed from its checkpoint).  Both run entirely in liblbm's
CUDA kernels; this module only moves tensors across the C ABI.
"""
import torch


class SaturationFunction(torch.autograd.Function):
    """J = smooth non-wetting saturation of the sample slab (mean of
    rho1 / (rho1 + rho2), Section 4.1) after ``nsteps`` steps from the initial
    densities ``rho_init``, as a function of ``xi_field`` (CUDA float32, the
    grid's shape; used on wall voxels, Eq. 15) and ``rho_in1`` (a 0-d tensor,
    the prescribed inlet density of component 1)."""

    @staticmethod
    def forward(ctx, xi_field, rho_in1, lattice, rho_init, nsteps, every):
        lattice.set_xi_field(xi_field.detach().contiguous())
        lattice.set_inlet(float(rho_in1))
        lattice.init_densities(*rho_init)
        lattice.record(int(nsteps), int(every))
        ctx.lattice = lattice
        ctx.recording = lattice.recordings
        ctx.rin_dtype = rho_in1.dtype if torch.is_tensor(rho_in1) else torch.float64
        J = lattice.saturation()[1]
        return torch.tensor(J, dtype=torch.float64, device=xi_field.device)

    @staticmethod
    def backward(ctx, grad_out):
        lat = ctx.lattice
        if getattr(lat, "recordings", None) != ctx.recording:
            # the lattice recorded another trajectory since this forward: its
            # adjoint would be the gradient of that one
            raise RuntimeError("the lattice was recorded again after this forward; run backward before the next "
                               "forward on the same lattice")
        gxi = torch.empty(lat.shape, dtype=torch.float32, device=grad_out.device)
        _, grin = lat.adjoint(float(grad_out), gxi)
        return gxi, torch.tensor(grin, dtype=ctx.rin_dtype, device=grad_out.device), None, None, None, None


def saturation(lattice, rho_init, xi_field, rho_in1, nsteps, every=50):
    """Differentiable J(xi_field, rho_in1); see SaturationFunction."""
    if not torch.is_tensor(rho_in1):
        rho_in1 = torch.tensor(float(rho_in1), dtype=torch.float64)
    return SaturationFunction.apply(xi_field, rho_in1, lattice, rho_init, nsteps, every)
