"""World-box walls (Sec. 3.4: unilateral constraints as penalty potentials)
on the GPU against the FP64 oracle: a block thrown about a box with friction
on every sweep variant, tilted walls with Chebyshev, damping, line search and
block Jacobi, the energy with wall penalties, and the adjoint with the wall
Hessians.  Tolerance 1e-5 of the bounding-box diagonal, as for the ground."""
import numpy as np
import pytest
import torch

from paper_2403_06321_b300 import synth, vbd
from gpu_util import bbox_diag, gpu_run, oracle_run, params_of

pytestmark = pytest.mark.gpu

BOX = synth.world_box((-0.3, -0.3, 0.0), (0.5, 0.4, 0.4))
TILTED = [(1.0, 0.2, 0.1, 0.0), (0.1, 1.0, -0.2, 0.0), (0.0, 0.0, 1.0, 0.0), (-0.3, -0.2, -1.0, -0.35)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_06321_b300.build import build
    build()
    assert torch.cuda.is_available()


def _block(jitter=0.05, seed=61, origin=(0.05, 0.05, 0.05)):
    return synth.beam(4, 3, 2, edge=0.05, E=1e5, nu=0.35, pin_face=None, jitter_frac=jitter, seed=seed,
                      origin=origin)


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7])
def test_block_thrown_about_a_box_matches_oracle(orc, variant):
    """30 steps: the block hits the +x, +y and floor walls with friction on."""
    m = _block()
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(synth.SimConfig(), walls=BOX, k_c=1e5, mu_c=0.3, eps_v=1e-2)
    v0 = _f32(np.broadcast_to([3.0, 2.0, -1.0], m.rest.shape))
    xg, vg = gpu_run(m, pd, colors, 1 / 60, 12, 30, v0=v0, variant=variant,
                     lanes=None if variant == 1 else 4)
    xo, vo = oracle_run(orc, m, pd, colors, 1 / 60, 12, 30, v0=v0)
    err = float(np.abs(xg - xo).max() / bbox_diag(m.rest))
    print("box, variant %d: err/bbox %.2e" % (variant, err))
    assert err <= 1e-5
    # free flight would carry it 1.5 m along +x: the +x wall turned it back
    assert xo[:, 0].max() < 0.5 + 0.01 and vo[:, 0].mean() < 0.5


@pytest.mark.parametrize("opts", [dict(cheby_rho=0.8), dict(k_d=1e-5), dict(line_search=True),
                                  dict(jacobi=True), dict(mu_c=0.4, eps_v=1e-2, ground_on=True,
                                                          ground_height=-0.01)],
                         ids=["chebyshev", "damping", "line_search", "jacobi", "friction_and_ground"])
def test_tilted_corner_matches_oracle(orc, opts):
    """A block pushed into a corner of tilted walls under a slanted gravity:
    contact with up to three walls at once, each option of the sweep."""
    m = _block(origin=(0.01, 0.01, 0.02))
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(synth.SimConfig(), gravity=(-3.0, -3.0, -9.8), walls=TILTED, k_c=1e5, **opts)
    v0 = _f32(np.broadcast_to([-0.5, -0.4, -0.3], m.rest.shape))
    iters, steps = (5, 10) if opts.get("jacobi") else (15, 20)
    xg, _ = gpu_run(m, pd, colors, 1 / 60, iters, steps, v0=v0)
    xo, _ = oracle_run(orc, m, pd, colors, 1 / 60, iters, steps, v0=v0)
    err = float(np.abs(xg - xo).max() / bbox_diag(m.rest))
    print("tilted corner %s: err/bbox %.2e" % (opts, err))
    assert err <= 1e-5
    pressed = 0
    for w in TILTED[:3]:
        nh = np.array(w[:3]) / np.linalg.norm(w[:3])
        pressed += bool((xo @ nh < w[3]).any())
    assert pressed >= 2


def test_energy_with_wall_penalties_matches_oracle(orc):
    m = _block(origin=(-0.02, -0.01, -0.015))
    pd = params_of(synth.SimConfig(), walls=TILTED, k_c=1e5)
    x = _f32(m.rest)
    v = _f32(np.broadcast_to([0.2, -0.1, -0.4], m.rest.shape))
    sim = vbd.Sim(m, vbd.make_params(**pd))
    try:
        sim.set_state(x, v)
        vbd.vbd_begin_step(sim.ctx, 1 / 60)
        G_gpu = sim.energy()
        xg, _ = sim.get_state()
        xg = xg.cpu().numpy().astype(np.float64)
        vbd.vbd_end_step(sim.ctx)
    finally:
        sim.close()
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(**pd)
    y = model.inertia_target(p, 1 / 60, x, v)
    G0 = model.energy_G(p, 1 / 60, xg, y)
    G_nw = model.energy_G(orc.Params.make(**dict(pd, walls=())), 1 / 60, xg, y)
    assert G0 - G_nw > 1e-3 * abs(G0)  # the wall terms matter here
    assert G_gpu == pytest.approx(G0, rel=1e-5)


def test_adjoint_with_wall_contact(orc):
    """Converged steps of a block sliding into a tilted corner: the adjoint
    includes k_c n n^T of every wall a vertex presses into."""
    from test_gpu_adjoint import _check, _gpu_grads, _oracle_grads
    m = synth.beam(4, 3, 2, edge=0.05, E=1e5, nu=0.4, pin_face=None, jitter_frac=0.05, seed=63,
                   origin=(0.002, 0.002, 0.0))
    colors, _ = orc.color_greedy(m.n_verts, m.tets)
    pd = params_of(synth.SimConfig(), gravity=(-2.0, -2.0, -9.8), walls=TILTED[:3], k_c=1e5)
    rng = np.random.default_rng(64)
    v0 = rng.normal(0, 0.05, m.rest.shape)
    v0 += np.array([-0.2, -0.2, -0.3])
    top = np.nonzero(m.grid_ijk[:, 2] == 2)[0]
    target = m.rest[top] + np.array([0.01, -0.02, -0.01])
    h, steps = 1 / 60, 6
    gE, gv, xg = _gpu_grads(m, pd, colors, h, 600, steps, v0, top, target, adj_iters=400)
    oE, ov, xo = _oracle_grads(orc, m, pd, colors, h, 0, steps, v0, top, target, newton=True)
    walls_hit = sum(bool((xo @ (np.array(w[:3]) / np.linalg.norm(w[:3])) < w[3]).any()) for w in TILTED[:3])
    print("wall contact: |x|err %.2e  walls %d" % (np.abs(xg - xo).max(), walls_hit))
    assert walls_hit >= 2
    assert np.abs(xg - xo).max() < 1e-5
    _check("wall contact", gE, oE, gv, ov)
