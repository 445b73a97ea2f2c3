"""torch.autograd.Functions over libpmgb's hand-written reverse mode.

* ``simulate(pm, noise)``: Zel'dovich ICs + all DKD steps; backward runs the
  adjoint method (Sec. 2.7, Table 5) through ``pm_adjoint`` and the IC pullback
  through ``pm_ic_adjoint``.  Only the final state is kept for the backward
  pass, so memory does not grow with the number of steps (the primal state is
  reintegrated backwards alongside the cotangents).
* ``density(pm, disp, n_mesh, order)``: CIC/TSC density contrast; backward is
  the scatter VJP w.r.t. positions (App. C), ``pm_density_vjp``.

sigma8 enters the ICs as an overall factor of the displacement field, so a
differentiable sigma8 is obtained by feeding noise * (sigma8 / cfg.sigma8).
"""
import torch


class _Simulate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, noise, pm):
        disp, vel = pm.ic_zeldovich(noise.contiguous())
        pm.run(disp, vel)
        ctx.pm = pm
        ctx.save_for_backward(noise, disp, vel)
        return disp.clone(), vel.clone()

    @staticmethod
    def backward(ctx, g_disp, g_vel):
        pm = ctx.pm
        noise, disp, vel = ctx.saved_tensors
        d, v = disp.clone(), vel.clone()
        ad = g_disp.contiguous().clone() if g_disp is not None else torch.zeros_like(d)
        av = g_vel.contiguous().clone() if g_vel is not None else torch.zeros_like(v)
        pm.adjoint(d, v, ad, av)
        anoise, _ = pm.ic_adjoint(noise.contiguous(), ad, av, with_sigma8=False)
        return anoise, None


class _Density(torch.autograd.Function):
    @staticmethod
    def forward(ctx, disp, pm, n_mesh, order):
        ctx.pm, ctx.n_mesh, ctx.order = pm, n_mesh, order
        ctx.save_for_backward(disp)
        return pm.density(disp, n_mesh, order)

    @staticmethod
    def backward(ctx, g):
        (disp,) = ctx.saved_tensors
        return ctx.pm.density_vjp(disp, g.contiguous(), ctx.n_mesh, ctx.order), None, None, None


def simulate(pm, noise):
    """Final (disp, vel) of a full run from white noise [B, N]; differentiable in noise."""
    return _Simulate.apply(noise, pm)


def density(pm, disp, n_mesh=None, order=None):
    """delta = rho M / N - 1 of X = q + disp; differentiable in disp."""
    return _Density.apply(disp, pm, n_mesh or pm.cfg.n_mesh, order or pm.cfg.order)
