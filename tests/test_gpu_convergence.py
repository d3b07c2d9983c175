"""Convergence reports (no paper counterpart; they state how far the fixed
iteration counts leave the solves):

* vbd_gradient_norm: max_i |dG/dx_i| of Eq. 2 (inertia, elasticity, plane
  penalties of Eq. 12) at the current iterate, checked against the oracle's
  FP64 gradient at the same positions and inertia target;
* vbd_adjoint_residuals: max |r - H lam| / max |r| of each recorded step
  after vbd_backward's block Gauss-Seidel sweeps.  For the last step with a
  single sweep (lam = 0 before it, r = dL/dx_T) the oracle replays that one
  sweep on its dense FP64 Hessian in the same colour order and computes the
  residual itself; with more sweeps the residual must fall."""
import numpy as np
import pytest
import torch

from paper_2403_06321_b300 import synth, vbd
from gpu_util import params_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_06321_b300.build import build
    build()


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def test_gradient_norm_matches_the_oracle_gradient(orc):
    m, cfg = synth.large_cube(6, drop_height=0.0)  # lowest vertex on the ground
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(cfg, k_c=1e5)
    rng = np.random.default_rng(81)
    x0 = _f32(m.rest + rng.uniform(-1e-3, 1e-3, m.rest.shape))
    v0 = _f32(rng.normal(0, 0.2, m.rest.shape))
    sim = vbd.Sim(m, vbd.make_params(**pd), colors=colors)
    try:
        sim.set_state(x0, v0)
        vbd.vbd_begin_step(sim.ctx, cfg.h)
        results = []
        for sweeps in (0, 2, 8, 40):
            for k in range(sweeps):
                vbd.vbd_sweep_color(sim.ctx, k % 4)
            g_gpu, scale = vbd.vbd_gradient_norm(sim.ctx)
            x, _ = sim.get_state()
            results.append((g_gpu, x.cpu().numpy().astype(np.float64)))
        vbd.vbd_end_step(sim.ctx)
        sim.sync_status()
    finally:
        sim.close()
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(**pd)
    y = model.inertia_target(p, cfg.h, x0, v0)
    M = np.repeat(model.mass(), 3)
    assert scale == pytest.approx(model.mass().max() * 9.8, rel=1e-6)
    first = None
    for g_gpu, x in results:
        g = M / cfg.h ** 2 * (x - y).reshape(-1) + model.elastic_grad(x)
        for n, d, act in model._plane_terms(p, x):
            for i in np.nonzero(act)[0]:
                g[3 * i:3 * i + 3] -= p.k_c * d[i] * n
        g_orc = float(np.abs(g).max())
        print("sweeps: |dG/dx|_inf gpu %.6e oracle %.6e" % (g_gpu, g_orc))
        # FP32 terms against FP64 at the same x; the residual shrinks while
        # its terms (m/h^2 |x - y|, elastic forces) do not, so the bar is
        # relative to the force scale, not to the residual
        assert abs(g_gpu - g_orc) <= 1e-4 * max(g_orc, scale)
        first = g_orc if first is None else first
    assert g_orc < 0.1 * first  # 50 sweeps later the residual has fallen


def _dense_block_gs_residual(orc, m, p, h, x_T, r, colors):
    """One block Gauss-Seidel sweep on H lam = r from lam = 0 (colours in
    ascending order, pinned vertices excluded) with the oracle's dense FP64
    Hessian of G at x_T; returns max |r - H lam| / max |r| over free DoFs."""
    model = orc.Model.from_mesh(m)
    _, H = model.global_grad_hess(p, h, x_T, x_T)  # y does not enter the Hessian
    free = model.free
    lam = np.zeros(3 * m.n_verts)
    for c in range(int(colors.max()) + 1):
        for i in np.nonzero((colors == c) & free)[0]:
            sl = slice(3 * i, 3 * i + 3)
            b = r[sl] - H[sl] @ lam + H[sl, sl] @ lam[sl]
            lam[sl] = np.linalg.solve(H[sl, sl], b)
    fd = np.repeat(free, 3)
    res = (r - H @ lam)[fd]
    return float(np.abs(res).max() / np.abs(r[fd]).max())


def test_adjoint_residuals_one_sweep_matches_oracle_and_more_sweeps_converge(orc):
    m = synth.beam(5, 2, 2, E=1e5, nu=0.4, jitter_frac=0.05, seed=61)
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(synth.SimConfig(), ground_on=True, ground_height=m.rest[:, 2].min() + 0.02, k_c=1e5)
    h, steps = 1 / 60, 3
    rng = np.random.default_rng(62)
    gx = rng.normal(0, 1.0, m.rest.shape) * (1 - m.pinned[:, None])
    sim = vbd.Sim(m, vbd.make_params(tape_steps=steps, **pd), colors=colors)
    try:
        sim.set_state(m.rest, np.zeros_like(m.rest))
        for _ in range(steps):
            sim.step(h, 30)
        x, _ = sim.get_state()
        x_T = x.cpu().numpy().astype(np.float64)
        dev = sim.workspace.device
        gxt = torch.tensor(gx.reshape(-1), dtype=torch.float32, device=dev)
        gE = torch.empty(m.n_tets, dtype=torch.float32, device=dev)
        gv = torch.empty(3 * m.n_verts, dtype=torch.float32, device=dev)
        rel = {}
        for it in (1, 4, 16, 64, 256):
            vbd.vbd_backward(sim.ctx, gxt, gE, gv, it)
            rel[it] = vbd.vbd_adjoint_residuals(sim.ctx, steps)
        sim.sync_status()
    finally:
        sim.close()
    p = orc.Params.make(**pd)
    r = _f32(gx).reshape(-1)
    want = _dense_block_gs_residual(orc, m, p, h, x_T, r, colors)
    print("one sweep, last step: gpu %.6e oracle %.6e; last step by sweeps %s" % (
        rel[1][-1], want, {k: "%.2e" % v[-1] for k, v in rel.items()}))
    assert rel[1][-1] == pytest.approx(want, rel=2e-3)
    lasts = [rel[k][-1] for k in (1, 4, 16, 64, 256)]
    assert all(b < a for a, b in zip(lasts, lasts[1:]))
    assert max(rel[256]) < 1e-4


def test_report_calls_refuse_what_they_cannot_answer():
    m = synth.beam(3, 2, 2, jitter_frac=0.05, seed=63)
    sim = vbd.Sim(m, vbd.make_params(tape_steps=2), colors=synth.kuhn_coloring(m.grid_ijk))
    try:
        with pytest.raises(vbd.VbdError) as e:
            vbd.vbd_gradient_norm(sim.ctx)  # no step yet: y is undefined
        assert e.value.status == "VBD_ERR_STATE"
        with pytest.raises(vbd.VbdError) as e:
            vbd.vbd_adjoint_residuals(sim.ctx, 2)  # no vbd_backward yet
        assert e.value.status == "VBD_ERR_NO_TAPE"
        sim.set_state(m.rest, np.zeros_like(m.rest))
        for _ in range(2):
            sim.step(1 / 60, 5)
        g, w = vbd.vbd_gradient_norm(sim.ctx)
        assert np.isfinite(g) and g >= 0.0 and w > 0.0
        dev = sim.workspace.device
        gx = torch.ones(3 * m.n_verts, dtype=torch.float32, device=dev)
        vbd.vbd_backward(sim.ctx, gx, None, None, 3)
        with pytest.raises(vbd.VbdError) as e:
            vbd.vbd_adjoint_residuals(sim.ctx, 1)  # two recorded steps need two entries
        assert e.value.status == "VBD_ERR_INVALID_ARG"
        r = vbd.vbd_adjoint_residuals(sim.ctx, 2)
        assert r.shape == (2,) and np.all(np.isfinite(r)) and np.all(r >= 0.0)
        sim.sync_status()
    finally:
        sim.close()
