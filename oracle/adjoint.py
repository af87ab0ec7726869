"""FP64 reference gradients of the step and of a rollout loss, by reverse-mode differentiation
of the population-form oracle (oracle.lbm) with torch.autograd on the CPU.

TEST INFRASTRUCTURE (oracle). The paper has no adjoint; the gradient is defined here as the
exact transpose Jacobian of the oracle's own forward map, which the tests pin independently
with central finite differences of that forward map.

Conventions: the state is the public moment state (p*, u, A) of oracle.lbm; a cotangent of a
state has the same (10, nz, ny, nx) layout and holds dL/d(component) for the stored component
(the off-diagonal entries A_xy, A_xz, A_yz are single stored numbers).
"""
import torch

from . import lbm


def step_vjp(lat, M_t, tau, force, lam_next, solid=None, rho=1.0):
    """lambda_t = (dM^{t+1}/dM^t)^T lam_next and g_F = (dM^{t+1}/dF)^T lam_next for one step
    with a time-constant force (uniform 3-vector or field (3, nz, ny, nx))."""
    M = torch.as_tensor(M_t, dtype=torch.float64).clone().requires_grad_(True)
    F = torch.as_tensor(force, dtype=torch.float64).clone().requires_grad_(True)
    out = lbm.step_moments(lat, M, tau, F, F, solid, rho, rho)
    (out * torch.as_tensor(lam_next, dtype=torch.float64)).sum().backward()
    return M.grad.detach(), F.grad.detach()


def velocity_mismatch_loss(M, u_target, fluid):
    """L = (1/N_fluid) sum over fluid sites of |u - u_target|^2."""
    d = (M[1:4] - u_target) * fluid.unsqueeze(0)
    return (d * d).sum() / fluid.sum()


def rollout_gradient(lat, M0, force, steps, tau, u_target, solid=None, rho=1.0):
    """Loss of a `steps`-step rollout and its gradients with respect to the initial public
    moments M0 and the per-site force field. Returns (L, dL/dM0, dL/dF)."""
    M0 = torch.as_tensor(M0, dtype=torch.float64).clone().requires_grad_(True)
    F = torch.as_tensor(force, dtype=torch.float64).clone().requires_grad_(True)
    shape = M0.shape[1:]
    fluid = torch.ones(shape, dtype=torch.float64)
    if solid is not None:
        fluid = (~torch.as_tensor(solid, dtype=torch.bool)).to(torch.float64)
    MT = lbm.run(lat, M0, steps, tau, F, solid, rho)
    L = velocity_mismatch_loss(MT, torch.as_tensor(u_target, dtype=torch.float64), fluid)
    L.backward()
    return L.detach(), M0.grad.detach(), F.grad.detach()


def rollout_loss(lat, M0, force, steps, tau, u_target, solid=None, rho=1.0):
    with torch.no_grad():
        shape = M0.shape[1:]
        fluid = torch.ones(shape, dtype=torch.float64)
        if solid is not None:
            fluid = (~torch.as_tensor(solid, dtype=torch.bool)).to(torch.float64)
        MT = lbm.run(lat, M0, steps, tau, force, solid, rho)
        return velocity_mismatch_loss(MT, torch.as_tensor(u_target, dtype=torch.float64), fluid)
