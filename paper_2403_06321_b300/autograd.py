"""torch.autograd wrapper around the C ABI: positions after S VBD steps as a
differentiable function of per-tet log Young's moduli and initial velocities.

Forward runs vbd_set_log_young, vbd_set_state and S x vbd_step with the
tape on; backward calls vbd_backward, which treats every recorded step as
converged (the paper has no derivatives; the adjoint follows from dG/dx = 0
of Eq. 2).  Only argument marshalling and stream ordering happen here.
"""
from __future__ import annotations

import torch

from . import vbd


class VBDFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_young: torch.Tensor, v0: torch.Tensor, sim: "vbd.Sim", x0: torch.Tensor,
                h: float, iters: int, steps: int, adj_iters: int) -> torch.Tensor:
        if steps > sim.tape_steps:
            raise ValueError("the Sim was bound with tape_steps=%d < steps=%d" % (sim.tape_steps, steps))
        dev = sim.workspace.device
        le = log_young.detach().to(device=dev, dtype=torch.float32).contiguous()
        vv = v0.detach().to(device=dev, dtype=torch.float32).contiguous().reshape(-1)
        xx = x0.detach().to(device=dev, dtype=torch.float32).contiguous().reshape(-1)
        out = torch.empty(3 * sim.n_verts, dtype=torch.float32, device=dev)
        s = sim.stream
        s.wait_stream(torch.cuda.current_stream(dev))
        vbd.vbd_set_log_young(sim.ctx, le)
        vbd.vbd_set_state(sim.ctx, xx, vv, None)
        for _ in range(steps):
            vbd.vbd_step(sim.ctx, h, iters)
        vbd.vbd_get_state(sim.ctx, out, None)
        torch.cuda.current_stream(dev).wait_stream(s)
        for t in (le, vv, xx, out):
            t.record_stream(s)
        ctx.sim, ctx.adj_iters = sim, adj_iters
        return out.view(-1, 3)

    @staticmethod
    def backward(ctx, grad_x: torch.Tensor):
        sim = ctx.sim
        dev = sim.workspace.device
        gx = grad_x.detach().to(device=dev, dtype=torch.float32).contiguous().reshape(-1)
        g_logE = torch.empty(sim.n_tets, dtype=torch.float32, device=dev)
        g_v0 = torch.empty(3 * sim.n_verts, dtype=torch.float32, device=dev)
        s = sim.stream
        s.wait_stream(torch.cuda.current_stream(dev))
        vbd.vbd_backward(sim.ctx, gx, g_logE, g_v0, ctx.adj_iters)
        torch.cuda.current_stream(dev).wait_stream(s)
        for t in (gx, g_logE, g_v0):
            t.record_stream(s)
        return g_logE, g_v0.view(-1, 3), None, None, None, None, None, None


def simulate(log_young, v0, sim, x0, h, iters, steps, adj_iters=100):
    """x(T) after `steps` VBD steps; differentiable in log_young and v0."""
    return VBDFunction.apply(log_young, v0, sim, x0, h, iters, steps, adj_iters)
