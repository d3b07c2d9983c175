"""Shared helpers for the GPU parity tests: run the same seeded workload
through the C ABI (CUDA path) and through the FP64 oracle."""
from __future__ import annotations

import numpy as np

from paper_2403_06321_b300 import synth, vbd


def params_of(cfg: synth.SimConfig, **over) -> dict:
    d = dict(gravity=cfg.gravity, ground_on=cfg.ground_on, ground_height=cfg.ground_height,
             ground_normal=cfg.ground_normal, k_c=cfg.k_c, cheby_rho=cfg.cheby_rho,
             init_mode=cfg.init_mode, det_eps=cfg.det_eps, k_d=cfg.k_d, mu_c=cfg.mu_c, eps_v=cfg.eps_v,
             line_search=cfg.line_search, jacobi=cfg.jacobi, self_collision=cfg.self_collision,
             dcd_radius=cfg.dcd_radius, walls=cfg.walls, ccd_interval=cfg.ccd_interval,
             ccd_edges=cfg.ccd_edges)
    d.update(over)
    return d


def bbox_diag(x: np.ndarray) -> float:
    return float(np.linalg.norm(x.max(0) - x.min(0)))


def gpu_run(mesh, pdict: dict, colors, h, iters, steps, x0=None, v0=None, vprev0=None,
            lanes=None, block=None, graph=True, vert_offset=None, tet_offset=None, variant=-1):
    """Returns (x, v) as float64 numpy arrays in caller order."""
    if variant == 3:
        pdict = dict(pdict, scatter_sweep=True)
    if variant == 7:
        pdict = dict(pdict, warp_rows=True)
    sim = vbd.Sim(mesh, vbd.make_params(**pdict), colors=colors,
                  vert_offset=vert_offset, tet_offset=tet_offset)
    try:
        if lanes or block or variant >= 0:
            vbd.vbd_set_launch(sim.ctx, lanes or 0, block or 0, variant)
        vbd.vbd_set_graph(sim.ctx, graph)
        x0 = mesh.rest if x0 is None else x0
        v0 = np.zeros_like(mesh.rest) if v0 is None else v0
        sim.set_state(x0, v0, vprev0)
        for _ in range(steps):
            sim.step(h, iters)
        sim.sync_status()
        x, v = sim.get_state()
        return x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    finally:
        sim.close()


def oracle_run(orc, mesh, pdict: dict, colors, h, iters, steps, x0=None, v0=None, vprev0=None):
    model = orc.Model.from_mesh(mesh)
    p = orc.Params.make(**pdict)
    nc = int(np.max(colors)) + 1
    x0 = mesh.rest if x0 is None else x0
    v0 = np.zeros_like(mesh.rest) if v0 is None else v0
    x, v, _ = orc.run(model, p, colors, nc, h, iters, steps, x0, v0, vprev0)
    return x, v
