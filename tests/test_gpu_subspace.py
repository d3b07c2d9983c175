"""Subspace constraints (Sec. 3.4, bilateral: a vertex moves within
x^t + span(Q), L = 1 a line, L = 2 a plane) on the GPU against the FP64
oracle: a beam on tilted rollers on every sweep variant and with each option
of the sweep, constrained vertices in the self-collision slab scene, the
vertices staying on their subspaces, the adjoint through constrained steps,
and the entry point's errors.
Tolerance 1e-5 of the bounding-box diagonal."""
import numpy as np
import pytest
import torch

from paper_2403_06321_b300 import synth, vbd
from gpu_util import bbox_diag, gpu_run, oracle_run, params_of

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_06321_b300.build import build
    build()
    assert torch.cuda.is_available()


def _rollers(seed=91):
    """Beam pinned at x = 0 whose far face slides in a tilted plane and whose
    top edge moves along a tilted line."""
    m = synth.beam(6, 3, 3, edge=0.05, E=1e5, nu=0.4, jitter_frac=0.08, seed=seed)
    ijk = m.grid_ijk
    m.sub_dim = np.full(m.n_verts, 3, np.int32)
    m.sub_dir = np.zeros((m.n_verts, 3))
    far = ijk[:, 0] == 6
    m.sub_dim[far] = 2
    m.sub_dir[far] = (1.0, 0.1, -0.2)
    edge = (ijk[:, 1] == 0) & (ijk[:, 2] == 3) & (ijk[:, 0] > 0) & (ijk[:, 0] < 6)
    m.sub_dim[edge] = 1
    m.sub_dir[edge] = (0.6, 0.3, -0.74)
    return m


def _on_subspaces(m, x, rel, x0=None):
    d = x - (m.rest if x0 is None else x0)
    scale = np.abs(d).max()
    for i in np.nonzero(m.sub_dim < 3)[0]:
        e = m.sub_dir[i] / np.linalg.norm(m.sub_dir[i])
        off = abs(d[i] @ e) if m.sub_dim[i] == 2 else np.linalg.norm(d[i] - (d[i] @ e) * e)
        assert off <= rel * scale, (i, off, scale)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7])
def test_rollers_match_oracle_on_every_variant(orc, variant):
    m = _rollers()
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(synth.SimConfig(), gravity=(1.5, -1.0, -9.8), cheby_rho=0.6)
    xg, _ = gpu_run(m, pd, colors, 1 / 60, 15, 12, variant=variant, lanes=None if variant == 1 else 4)
    xo, _ = oracle_run(orc, m, pd, colors, 1 / 60, 15, 12)
    err = float(np.abs(xg - xo).max() / bbox_diag(m.rest))
    print("rollers, variant %d: err/bbox %.2e" % (variant, err))
    assert err <= TOL
    _on_subspaces(m, xg, 1e-5)
    assert np.abs(xo[m.sub_dim == 2] - m.rest[m.sub_dim == 2]).max() > 1e-3  # the rollers move


@pytest.mark.parametrize("opts", [dict(line_search=True), dict(jacobi=True), dict(k_d=1e-5),
                                  dict(ground_on=True, ground_height=0.02, k_c=1e5, mu_c=0.3, eps_v=1e-2),
                                  dict(init_mode=0), dict(init_mode=1)],
                         ids=["line_search", "jacobi", "damping", "ground_friction", "init_previous",
                              "init_inertia"])
def test_rollers_with_each_option_match_oracle(orc, opts):
    m = _rollers(seed=92)
    m.rest[:, 2] += 0.03
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(synth.SimConfig(), gravity=(1.5, -1.0, -9.8), **opts)
    iters, steps = (5, 8) if opts.get("jacobi") else (15, 12)
    xg, _ = gpu_run(m, pd, colors, 1 / 60, iters, steps)
    xo, _ = oracle_run(orc, m, pd, colors, 1 / 60, iters, steps)
    err = float(np.abs(xg - xo).max() / bbox_diag(m.rest))
    print("rollers %s: err/bbox %.2e" % (opts, err))
    assert err <= TOL
    _on_subspaces(m, xg, 1e-5)


def test_constrained_vertices_in_the_self_collision_scene(orc):
    """The upper slab's top vertices may only move vertically (L = 1) and a
    row of its side only within a vertical plane (L = 2) while the slabs push
    each other apart."""
    from test_gpu_collision import _trajectory
    m, cfg, u0 = synth.colliding_slabs(seed=7)
    m.sub_dim = np.full(m.n_verts, 3, np.int32)
    m.sub_dir = np.zeros((m.n_verts, 3))
    upper = np.arange(m.n_verts) >= u0
    top = upper & (m.rest[:, 2] > m.rest[upper, 2].max() - 0.02)
    m.sub_dim[top] = 1
    m.sub_dir[top] = (0.0, 0.0, 1.0)
    side = upper & ~top & (m.rest[:, 0] < m.rest[upper, 0].min() + 0.02)
    m.sub_dim[side] = 2
    m.sub_dir[side] = (1.0, 0.2, 0.0)
    assert top.sum() > 50 and side.sum() > 5
    err, x, counts = _trajectory(orc, m, params_of(cfg), cfg.h, cfg.iters, cfg.steps)
    print("slabs with subspaces: err/bbox %.2e, pairs %s" % (err, counts))
    assert min(counts) > 20
    assert err <= TOL
    _on_subspaces(m, x, 1e-12, x0=np.asarray(m.rest, np.float32).astype(np.float64))  # the start positions


def test_subspace_entry_point_errors():
    m = _rollers()
    arr = vbd.MeshArrays(m.rest, m.tets, m.young, m.poisson, m.density, m.pinned)
    ctx = vbd.vbd_create_mesh(arr.desc(), vbd.make_params())
    try:
        pinned = int(np.nonzero(m.pinned)[0][0])
        free = int(np.nonzero(m.pinned == 0)[0][0])
        for vertex, dim, d in (([m.n_verts], [1], [(1, 0, 0)]), ([pinned], [1], [(1, 0, 0)]),
                               ([free, free], [1, 2], [(1, 0, 0), (0, 1, 0)]), ([free], [3], [(1, 0, 0)]),
                               ([free], [2], [(0, 0, 0)]), ([free], [1], [(np.nan, 0, 0)])):
            with pytest.raises(vbd.VbdError) as e:
                vbd.vbd_set_subspaces(ctx, vertex, dim, d)
            assert e.value.status == "VBD_ERR_INVALID_ARG"
        vbd.vbd_set_subspaces(ctx, [free], [2], [(0, 0, 1)])
        vbd.vbd_color(ctx, None)
        ws = torch.empty(vbd.vbd_workspace_size(ctx), dtype=torch.uint8, device="cuda")
        stream = torch.cuda.Stream()
        vbd.vbd_bind(ctx, ws, ws.numel(), stream.cuda_stream)
        with pytest.raises(vbd.VbdError) as e:
            vbd.vbd_set_subspaces(ctx, [], [], np.zeros((0, 3)))
        assert e.value.status == "VBD_ERR_STATE"
        stream.synchronize()
    finally:
        vbd.vbd_destroy(ctx)


def test_adjoint_through_constrained_steps_matches_oracle(orc):
    """Converged steps of the rollers beam (4 steps, 400 iterations on the
    GPU, dense Newton in the oracle): the reduced adjoint blocks and the
    r - H lam part of xbar give dL/dlogE and dL/dv0 within 1e-3 relative of
    the oracle's dense adjoint."""
    from test_gpu_adjoint import _check, _gpu_grads, _oracle_grads
    m = synth.beam(6, 2, 2, edge=0.05, E=1e5, nu=0.4, jitter_frac=0.05, seed=95)
    ijk = m.grid_ijk
    m.sub_dim = np.full(m.n_verts, 3, np.int32)
    m.sub_dir = np.zeros((m.n_verts, 3))
    far = ijk[:, 0] == 6
    m.sub_dim[far] = 2
    m.sub_dir[far] = (1.0, 0.1, -0.2)
    edge = (ijk[:, 1] == 0) & (ijk[:, 2] == 2) & (ijk[:, 0] > 0) & (ijk[:, 0] < 6)
    m.sub_dim[edge] = 1
    m.sub_dir[edge] = (0.6, 0.3, -0.74)
    colors, _ = orc.color_greedy(m.n_verts, m.tets)
    pd = params_of(synth.SimConfig(), gravity=(1.0, -0.5, -9.8))
    Bm = orc.Model.from_mesh(m).reduced_basis()
    rng = np.random.default_rng(96)
    v0 = (Bm @ (Bm.T @ rng.normal(0, 0.2, 3 * m.n_verts))).reshape(-1, 3)  # admissible
    v0 = np.asarray(v0, np.float32).astype(np.float64)
    v0 = (Bm @ (Bm.T @ v0.reshape(-1))).reshape(-1, 3)
    tip = np.nonzero(ijk[:, 0] >= 5)[0]
    target = m.rest[tip] + np.array([0.02, -0.01, 0.03])
    h, steps = 1 / 60, 4
    gE, gv, xg = _gpu_grads(m, pd, colors, h, 400, steps, v0, tip, target, adj_iters=300)
    oE, ov, xo = _oracle_grads(orc, m, pd, colors, h, 0, steps, v0, tip, target, newton=True)
    print("constrained adjoint: |x|err %.2e" % np.abs(xg - xo).max())
    assert np.abs(xg - xo).max() < 1e-5
    _check("constrained adjoint", gE, oE, gv, ov)
