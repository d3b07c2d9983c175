"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs and the same colouring.  Tolerance: FP32 positions
within 1e-5 of the bounding-box diagonal of the FP64 oracle's, the bar the
method's FP32 GPU / FP64 CPU comparison is held to."""
import numpy as np
import pytest
import torch

from paper_2403_06321_b300 import synth, vbd
from gpu_util import bbox_diag, gpu_run, oracle_run, params_of

pytestmark = pytest.mark.gpu

TOL = 1e-5  # x bbox diagonal


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_06321_b300.build import build
    build()
    assert torch.cuda.is_available()


def _err(xg, xo, ref):
    return float(np.abs(xg - xo).max() / bbox_diag(ref))


@pytest.mark.parametrize("coloring", ["kuhn", "greedy"])
def test_cantilever_beam_100_steps(orc, coloring):
    """10x3x3 beam, x=0 face pinned, E=1e5, nu=0.4, h=1/60, 20 iters, 100 steps."""
    m, cfg = synth.cantilever_beam()
    colors = synth.kuhn_coloring(m.grid_ijk) if coloring == "kuhn" else orc.color_greedy(m.n_verts, m.tets)[0]
    pd = params_of(cfg)
    xg, vg = gpu_run(m, pd, colors, cfg.h, cfg.iters, cfg.steps)
    xo, vo = oracle_run(orc, m, pd, colors, cfg.h, cfg.iters, cfg.steps)
    err = _err(xg, xo, m.rest)
    print("cantilever %s: max |x_gpu - x_oracle| / bbox = %.3e" % (coloring, err))
    assert err <= TOL
    assert np.abs(xo - m.rest).max() > 0.01  # the beam really sags
    assert np.abs(vg - vo).max() <= TOL * bbox_diag(m.rest) / cfg.h * 10


def test_one_iteration_from_perturbed_state_ragged(orc):
    """13x5x3 jittered beam (several blocks, ragged colour ranges), seeded
    deformed state and velocities: one iteration of every colour."""
    m = synth.beam(13, 5, 3, edge=0.05, E=3e5, nu=0.42, jitter_frac=0.1, seed=11)
    x0, v0 = synth.perturbed_state(m.rest, 0.004, 0.3, seed=12)
    x0[m.pinned == 1] = m.rest[m.pinned == 1]
    colors, _ = orc.color_greedy(m.n_verts, m.tets)
    pd = params_of(synth.SimConfig())
    xo, vo = oracle_run(orc, m, pd, colors, 1 / 60, 1, 1, x0, v0)
    shapes = [dict(variant=1, block=128), dict(variant=1, block=256)] + \
             [dict(variant=0, lanes=l) for l in (4, 8, 16, 32)] + \
             [dict(variant=2, lanes=4), dict(variant=2, lanes=8, block=256), dict(variant=3, lanes=4),
              dict(variant=3, lanes=8), dict(variant=4, lanes=4), dict(variant=4, lanes=8),
              dict(variant=5, lanes=4), dict(variant=5, lanes=8, block=128),
              dict(variant=6, lanes=4), dict(variant=6, lanes=8, block=128), dict(variant=6, lanes=16),
              dict(variant=7)]
    results = []
    for sh in shapes:
        xg, vg = gpu_run(m, pd, colors, 1 / 60, 1, 1, x0, v0, **sh)
        assert _err(xg, xo, m.rest) <= 1e-6, sh
        results.append(xg)
    # same lanes-per-vertex reduction order: pipelined and plain 8-lane sweeps agree bit for bit
    assert np.array_equal(results[0], results[3]) and np.array_equal(results[1], results[3])
    # the persistent form is the plain kernel on another grid
    assert np.array_equal(results[6], results[2]) and np.array_equal(results[7], results[3])
    # the scatter form sums the same per-slot terms in the same order, but each
    # term is rounded before it is added (no fused multiply-add into the sum)
    for a, b in ((results[8], results[2]), (results[9], results[3])):
        assert _err(a, b, m.rest) <= 1e-7
    # the fused cluster loop runs the same passes inside one launch
    assert np.array_equal(results[10], results[2]) and np.array_equal(results[11], results[3])
    # warp rows: the same slots per lane in the same order as 4 lanes, streamed through shared memory
    assert np.array_equal(results[17], results[2])


def test_ground_contact_and_chebyshev(orc):
    """Jittered 4x4x3 block falling onto the ground (k_c = 1e5), Chebyshev
    rho = 0.9 with the colliding-vertex skip, 30 steps of 15 iterations."""
    m = synth.beam(4, 4, 3, edge=0.05, E=2e5, nu=0.4, pin_face=None, jitter_frac=0.1, seed=13,
                   origin=(0.0, 0.0, 0.02))
    colors, _ = orc.color_greedy(m.n_verts, m.tets)
    for rho in (0.0, 0.9):
        pd = params_of(synth.SimConfig(), ground_on=True, k_c=1e5, cheby_rho=rho)
        xg, _ = gpu_run(m, pd, colors, 1 / 60, 15, 30)
        xo, _ = oracle_run(orc, m, pd, colors, 1 / 60, 15, 30)
        assert xo[:, 2].min() < 0.0  # contact happened
        err = _err(xg, xo, m.rest)
        print("contact rho=%.1f: err/bbox = %.3e" % (rho, err))
        assert err <= TOL


def test_init_modes_and_damping(orc):
    m = synth.beam(6, 2, 2, edge=0.1, E=1e5, nu=0.4, jitter_frac=0.05, seed=14)
    colors, _ = orc.color_greedy(m.n_verts, m.tets)
    rng = np.random.default_rng(15)
    v0 = rng.normal(0, 0.2, m.rest.shape)
    for mode in (0, 1, 2, 3):
        for kd in (0.0, 1e-3):
            pd = params_of(synth.SimConfig(), init_mode=mode, k_d=kd)
            xg, _ = gpu_run(m, pd, colors, 1 / 60, 10, 10, None, v0)
            xo, _ = oracle_run(orc, m, pd, colors, 1 / 60, 10, 10, None, v0)
            assert _err(xg, xo, m.rest) <= TOL, (mode, kd)


def test_batched_union_equals_individual_meshes(orc):
    meshes = [synth.beam(a, b, c, E=E, nu=nu, pin_face=f) for a, b, c, E, nu, f in
              [(5, 2, 2, 2e4, 0.3, "x-"), (8, 3, 2, 3e5, 0.45, "y+"), (4, 2, 3, 1e5, 0.4, "z-")]]
    cat, voff, toff = synth.concat(meshes)
    cat_colors = np.concatenate([orc.color_greedy(mm.n_verts, mm.tets)[0] for mm in meshes])
    pd = params_of(synth.SimConfig())
    xb, _ = gpu_run(cat, pd, cat_colors, 1 / 60, 10, 8, vert_offset=voff, tet_offset=toff)
    for b, mm in enumerate(meshes):
        xi, _ = gpu_run(mm, pd, cat_colors[voff[b]:voff[b + 1]], 1 / 60, 10, 8)
        assert np.array_equal(xb[voff[b]:voff[b + 1]], xi)  # bit-identical
    xo, _ = oracle_run(orc, cat, pd, cat_colors, 1 / 60, 10, 8)
    assert _err(xb, xo, cat.rest) <= TOL


def test_graph_replay_equals_eager():
    m, cfg = synth.cantilever_beam()
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(cfg, cheby_rho=0.8)
    out = {}
    for pipe in (1, 0, 2, 3, 4, 5):
        xa, va = gpu_run(m, pd, colors, cfg.h, 7, 5, graph=True, variant=pipe)
        xb, vb = gpu_run(m, pd, colors, cfg.h, 7, 5, graph=False, variant=pipe)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        out[pipe] = xa
    # persistent and fused (with its in-kernel Chebyshev update) equal the plain launches
    assert np.array_equal(out[2], out[0]) and np.array_equal(out[4], out[0])


def test_energy_fp64_matches_oracle(orc):
    m = synth.beam(6, 3, 2, edge=0.1, E=1e5, nu=0.4, jitter_frac=0.1, seed=16)
    x0, v0 = synth.perturbed_state(m.rest, 0.01, 0.2, seed=17)
    pd = params_of(synth.SimConfig(), ground_on=True, ground_height=0.05, k_c=1e4)
    # float32-representable inputs so that both sides start from the same numbers
    x0, v0 = x0.astype(np.float32).astype(np.float64), v0.astype(np.float32).astype(np.float64)
    sim = vbd.Sim(m, vbd.make_params(**pd))
    try:
        sim.set_state(x0, v0)
        vbd.vbd_begin_step(sim.ctx, 1 / 60)
        G_gpu = sim.energy()
    finally:
        sim.close()
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(**pd)
    y = model.inertia_target(p, 1 / 60, x0, v0)
    xi = model.initial_guess(p, 1 / 60, x0, v0, v0)
    G_orc = model.energy_G(p, 1 / 60, xi, y)
    assert G_gpu == pytest.approx(G_orc, rel=1e-5)


def test_nonfinite_update_is_reported():
    m, cfg = synth.cantilever_beam()
    x0 = m.rest.copy()
    free = np.nonzero(m.pinned == 0)[0]
    x0[free[5]] = np.nan
    sim = vbd.Sim(m, vbd.make_params(**params_of(cfg)), colors=synth.kuhn_coloring(m.grid_ijk))
    try:
        sim.set_state(x0, np.zeros_like(x0))
        sim.step(cfg.h, 3)
        with pytest.raises(vbd.VbdError) as e:
            sim.sync_status()
        assert e.value.status == "VBD_ERR_NONFINITE"
        sim.set_state(m.rest, np.zeros_like(x0))  # the context stays usable
        sim.step(cfg.h, 3)
        sim.sync_status()
    finally:
        sim.close()


def test_ground_friction_sliding_and_sticking(orc):
    """Jittered 4x4x2 block on the ground with friction (Eqs. 13-16): sliding
    at 1 m/s (Coulomb regime) and at rest on a slope below the friction angle
    (static regime, |u| < eps_v h)."""
    m = synth.beam(4, 4, 2, edge=0.05, E=2e5, nu=0.35, pin_face=None, jitter_frac=0.1, seed=81)
    colors, _ = orc.color_greedy(m.n_verts, m.tets)
    v0 = np.zeros_like(m.rest)
    v0[:, 0] = 1.0
    th = np.arctan(0.2)
    slope = (9.8 * np.sin(th), 0.0, -9.8 * np.cos(th))
    for gravity, vinit in [((0, 0, -9.8), v0), (slope, np.zeros_like(m.rest))]:
        pd = params_of(synth.SimConfig(), gravity=gravity, ground_on=True, k_c=1e6, mu_c=0.4, eps_v=1e-3)
        xg, vg = gpu_run(m, pd, colors, 1 / 60, 25, 20, None, vinit)
        xo, vo = oracle_run(orc, m, pd, colors, 1 / 60, 25, 20, None, vinit)
        err = _err(xg, xo, m.rest)
        print("friction g=%s: err/bbox = %.3e, mean vx gpu %.5f oracle %.5f" % (
            np.round(gravity, 2), err, vg[:, 0].mean(), vo[:, 0].mean()))
        assert err <= TOL


def test_line_search_with_hard_contact(orc):
    """Soft block hitting the ground at 5 m/s (k_c = 1e6): full Newton steps
    overshoot into the penalty, and the local line search (Sec. 3.2) changes
    the result (by ~8e-3 of the bbox); both variants match the oracle, whose
    search evaluates G_i literally.  (At k_c = 1e8 vertices come to rest at
    d ~ 1e-6 after one pass and the contact branch d > 0 is then decided by
    rounding: FP32 and FP64 runs take different branches there.)"""
    m = synth.beam(4, 3, 2, edge=0.05, E=1e4, nu=0.4, pin_face=None, jitter_frac=0.1, seed=73,
                   origin=(0, 0, 0.004))
    colors, _ = orc.color_greedy(m.n_verts, m.tets)
    v0 = np.zeros_like(m.rest)
    v0[:, 2] = -5.0
    out = {}
    for ls in (False, True):
        pd = params_of(synth.SimConfig(), ground_on=True, k_c=1e6, line_search=ls)
        xg, _ = gpu_run(m, pd, colors, 1 / 60, 12, 6, None, v0)
        xo, _ = oracle_run(orc, m, pd, colors, 1 / 60, 12, 6, None, v0)
        err = _err(xg, xo, m.rest)
        print("line search %s: err/bbox = %.3e" % (ls, err))
        assert err <= TOL
        out[ls] = xo
    assert _err(out[True], out[False], m.rest) > 1e-3


def test_block_jacobi(orc):
    """Block Jacobi (all vertices against the previous iterate, x^new and
    copy-back), with and without the line search, on a soft beam where Jacobi
    converges; the GPU ignores the colouring in this mode."""
    m = synth.beam(6, 2, 2, edge=0.1, E=2e3, nu=0.4, jitter_frac=0.05, seed=82)
    colors, _ = orc.color_greedy(m.n_verts, m.tets)
    for ls in (False, True):
        pd = params_of(synth.SimConfig(), jacobi=True, line_search=ls)
        xg, _ = gpu_run(m, pd, colors, 1 / 60, 30, 10)
        xo, _ = oracle_run(orc, m, pd, colors, 1 / 60, 30, 10)
        assert _err(xg, xo, m.rest) <= TOL
    xk, _ = gpu_run(m, params_of(synth.SimConfig(), jacobi=True), synth.kuhn_coloring(m.grid_ijk), 1 / 60, 30, 10)
    xg, _ = gpu_run(m, params_of(synth.SimConfig(), jacobi=True), colors, 1 / 60, 30, 10)
    assert np.array_equal(xk, xg)


@pytest.mark.parametrize("variant", [1, 7])
def test_pipeline_wait_time_out_is_reported_and_recoverable(variant):
    """A bounded wait of the TMA-staged sweep that runs out (the test hook
    makes each CTA's first chunk also wait on a barrier at which nothing
    arrives) is reported as VBD_ERR_TIMEOUT; the context then runs normally
    and gives the same result as a context that never timed out."""
    m, cfg = synth.cantilever_beam()
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(cfg)
    ref, _ = gpu_run(m, pd, colors, cfg.h, 5, 3, variant=variant)
    sim = vbd.Sim(m, vbd.make_params(warp_rows=variant == 7, **pd), colors=colors)
    try:
        vbd.vbd_set_launch(sim.ctx, 0, 0, variant)
        sim.set_state(m.rest, np.zeros_like(m.rest))
        vbd.vbd_debug_stall_pipeline(sim.ctx, True)
        vbd.vbd_begin_step(sim.ctx, cfg.h)
        vbd.vbd_sweep_color(sim.ctx, 0)
        vbd.vbd_end_step(sim.ctx)
        with pytest.raises(vbd.VbdError) as e:
            sim.sync_status()
        assert e.value.status == "VBD_ERR_TIMEOUT"
        vbd.vbd_debug_stall_pipeline(sim.ctx, False)
        sim.set_state(m.rest, np.zeros_like(m.rest))
        for _ in range(3):
            sim.step(cfg.h, 5)
        sim.sync_status()
        x, _ = sim.get_state()
        assert np.array_equal(x.cpu().numpy().astype(np.float64), ref)
    finally:
        sim.close()
