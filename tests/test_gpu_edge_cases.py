"""Degenerate and edge inputs through the C ABI against the FP64 oracle:
no free vertex, one tet with one free vertex, empty colours, zero
iterations, heterogeneous per-tet materials, a single colour pass called
by hand.  Tolerance: 1e-5 of the bounding-box diagonal (1e-6 for one pass)."""
import numpy as np
import pytest
import torch

from paper_2403_06321_b300 import synth, vbd
from gpu_util import bbox_diag, gpu_run, oracle_run, params_of

pytestmark = pytest.mark.gpu

H = 1.0 / 60.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_06321_b300.build import build
    build()
    assert torch.cuda.is_available()


def _err(a, b, ref):
    return float(np.abs(a - b).max() / bbox_diag(ref))


def test_every_vertex_pinned_is_a_no_op(orc):
    m = synth.beam(3, 2, 2, jitter_frac=0.1, seed=81)
    m.pinned[:] = 1
    v0 = np.random.default_rng(82).normal(0, 0.5, m.rest.shape)
    xg, vg = gpu_run(m, params_of(synth.SimConfig()), None, H, 10, 3, v0=v0)
    assert np.array_equal(xg, m.rest.astype(np.float32).astype(np.float64))
    assert np.all(vg == 0.0)


def test_single_tet_single_free_vertex(orc):
    """One tet, three corners pinned: every step is the exact minimiser of a
    quadratic in the free corner (J is affine in one vertex)."""
    rest = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0], [0.02, 0.03, 0.1]], np.float64)
    m = synth.MeshInput(rest=rest, tets=np.array([[0, 1, 2, 3]], np.int32),
                        young=np.array([1e5], np.float32), poisson=np.array([0.4], np.float32),
                        density=np.array([1000.0], np.float32), pinned=np.array([1, 1, 1, 0], np.uint8))
    colors = np.array([0, 1, 2, 3], np.int32)
    pd = params_of(synth.SimConfig())
    xg, _ = gpu_run(m, pd, colors, H, 3, 20)
    xo, _ = oracle_run(orc, m, pd, colors, H, 3, 20)
    assert np.abs(xo[3] - rest[3]).max() > 1e-4  # it sags
    assert _err(xg, xo, rest) <= 1e-5


def test_empty_colours_are_skipped(orc):
    """A caller colouring with unused ids (1 and 4 empty of 0..5)."""
    m = synth.beam(4, 3, 2, jitter_frac=0.1, seed=83)
    base = synth.kuhn_coloring(m.grid_ijk)
    colors = np.array([0, 2, 3, 5], np.int32)[base]
    pd = params_of(synth.SimConfig())
    xg, _ = gpu_run(m, pd, colors, H, 10, 5)
    xo, _ = oracle_run(orc, m, pd, colors, H, 10, 5)
    assert _err(xg, xo, m.rest) <= 1e-5


def test_zero_iterations_keep_the_initial_guess(orc):
    m = synth.beam(4, 2, 2, jitter_frac=0.1, seed=84)
    v0 = np.random.default_rng(85).normal(0, 0.3, m.rest.shape)
    v0[m.pinned == 1] = 0
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(synth.SimConfig())
    xg, vg = gpu_run(m, pd, colors, H, 0, 2, v0=v0)
    xo, vo = oracle_run(orc, m, pd, colors, H, 0, 2, v0=v0)
    assert _err(xg, xo, m.rest) <= 1e-6
    assert np.abs(vg - vo).max() <= 1e-4


def test_heterogeneous_per_tet_materials(orc):
    """E and nu differ per tet, so every vertex reads its tets' own mu and
    lambda (the per-tet material path of the sweep)."""
    m = synth.beam(6, 3, 3, edge=0.05, jitter_frac=0.1, seed=86)
    rng = np.random.default_rng(87)
    m.young = np.exp(rng.uniform(np.log(1e4), np.log(1e6), m.n_tets)).astype(np.float32)
    m.poisson = rng.uniform(0.2, 0.48, m.n_tets).astype(np.float32)
    m.density = rng.uniform(500, 2000, m.n_tets).astype(np.float32)
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(synth.SimConfig(), ground_on=True, ground_height=-0.02, k_c=1e6)
    xg, _ = gpu_run(m, pd, colors, H, 20, 40)
    xo, _ = oracle_run(orc, m, pd, colors, H, 20, 40)
    assert np.abs(xo - m.rest).max() > 1e-2
    assert _err(xg, xo, m.rest) <= 1e-5


def test_manual_colour_passes_equal_iterate(orc):
    """vbd_sweep_color over the colours, then vbd_accelerate, is the same
    iteration as vbd_iterate (bit for bit), with Chebyshev on."""
    m = synth.beam(5, 3, 2, jitter_frac=0.1, seed=88)
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(synth.SimConfig(), cheby_rho=0.9)
    out = []
    for manual in (False, True):
        sim = vbd.Sim(m, vbd.make_params(**pd), colors=colors)
        try:
            sim.set_state(m.rest, np.zeros_like(m.rest))
            for _ in range(3):
                vbd.vbd_begin_step(sim.ctx, H)
                if manual:
                    for n in range(1, 8):
                        for c in range(4):
                            vbd.vbd_sweep_color(sim.ctx, c)
                        vbd.vbd_accelerate(sim.ctx, n)
                else:
                    vbd.vbd_iterate(sim.ctx, 7)
                vbd.vbd_end_step(sim.ctx)
            sim.sync_status()
            out.append(sim.get_state()[0].cpu().numpy())
        finally:
            sim.close()
    assert np.array_equal(out[0], out[1])


def test_in_place_writes_equal_xnew_copy_back(orc):
    """Algorithm 1 writes x^new and copies it back after each colour; with
    tets and ground contact no two vertices of one colour interact, so the
    library's in-place writes give the same positions bit for bit (here with
    ground contact, friction and Chebyshev on)."""
    m = synth.beam(5, 4, 3, edge=0.05, pin_face=None, jitter_frac=0.1, seed=89, origin=(0, 0, 0.01))
    colors = synth.kuhn_coloring(m.grid_ijk)
    v0 = np.zeros_like(m.rest)
    v0[:, 2] = -1.0
    pd = params_of(synth.SimConfig(), ground_on=True, k_c=1e5, mu_c=0.3, cheby_rho=0.8)
    xa, va = gpu_run(m, pd, colors, H, 10, 10, v0=v0)
    xb, vb = gpu_run(m, dict(pd, xnew_copy_back=True), colors, H, 10, 10, v0=v0)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert xa[:, 2].min() < 0.01  # it reached the ground


def test_warp_rows_with_per_tet_materials_run_the_persistent_pass():
    """The warp-row records carry no per-tet material index, so with
    per-tet materials (here after vbd_set_log_young) variant 7's passes run
    variant 2 with 4 lanes: the same positions bit for bit, and the same as
    variant 7 gives once the materials are uniform again."""
    m = synth.beam(8, 3, 3, edge=0.05, E=2e5, nu=0.4, jitter_frac=0.1, seed=77)
    colors = synth.kuhn_coloring(m.grid_ijk)
    rng = np.random.default_rng(78)
    logE = (np.log(2e5) + rng.uniform(-0.5, 0.5, m.n_tets)).astype(np.float32)
    out = {}
    for variant in (2, 7):
        sim = vbd.Sim(m, vbd.make_params(warp_rows=True), colors=colors)
        try:
            vbd.vbd_set_launch(sim.ctx, 4, 256, variant)
            vbd.vbd_set_log_young(sim.ctx, logE)
            sim.set_state(m.rest, np.zeros_like(m.rest))
            for _ in range(4):
                sim.step(1 / 60, 10)
            sim.sync_status()
            out[variant] = sim.get_state()[0].cpu().numpy()
        finally:
            sim.close()
    assert np.array_equal(out[2], out[7])
    assert np.abs(out[7] - m.rest).max() > 1e-4  # it moved
