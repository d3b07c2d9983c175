"""Vertex-triangle CCD (Sec. 3.5: before every n_col-th iteration, along the
straight paths from x^t to the current iterate) on the GPU against the FP64
oracle: blocks thrown at a pinned block fast enough to pass its top face
within one step, with CCD every 1, 3 or 5 iterations, alone and with
Chebyshev, damping and friction.  The pairs of the last CCD of every step are
compared exactly; positions within 1e-5 of the bounding-box diagonal."""
import numpy as np
import pytest
import torch

from paper_2403_06321_b300 import synth, vbd
from gpu_util import bbox_diag, params_of

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_06321_b300.build import build
    build()
    assert torch.cuda.is_available()


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def _scene(seed=131, origin=(0.02, 0.03, 0.13), upper_dims=(2, 2, 1)):
    lower = synth.beam(3, 3, 1, edge=0.1, E=1e5, nu=0.4, pin_face="z-", jitter_frac=0.03, seed=seed)
    upper = synth.beam(*upper_dims, edge=0.1, E=1e5, nu=0.4, pin_face=None, jitter_frac=0.03, seed=seed + 1,
                       origin=origin)
    cat, voff, _ = synth.concat([lower, upper])
    cat.grid_ijk = None
    return cat, voff


def _run(orc, m, pd, v0, h, iters, steps):
    """Step by step on both sides with the library's colouring; returns the
    worst position error (/ bbox), the oracle's final state and the number
    of CCD pairs after each step."""
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(**pd)
    sim = vbd.Sim(m, vbd.make_params(**pd))
    counts = []
    try:
        colors = vbd.vbd_get_colors(sim.ctx, m.n_verts)
        nc = int(colors.max()) + 1
        x = _f32(m.rest)
        v = _f32(v0)
        vp = v.copy()
        sim.set_state(x, v)
        worst = 0.0
        for step in range(steps):
            sim.step(h, iters)
            model.step(p, colors, nc, h, iters, x, v, vp)
            got = vbd.vbd_get_contacts(sim.ctx, m.n_verts)
            want = model.contacts()
            _, is_ccd = model.contact_weights()
            bad = np.nonzero(got != want)[0]
            assert bad.size == 0, (step, bad, got[bad], want[bad])
            counts.append(int(is_ccd.sum()))
            xg, _ = sim.get_state()
            worst = max(worst, float(np.abs(xg.cpu().numpy() - x).max()))
        sim.sync_status()
    finally:
        sim.close()
    return worst / bbox_diag(m.rest), x, v, counts


@pytest.mark.parametrize("interval", [1, 3, 5])
def test_fast_block_matches_oracle(orc, interval):
    m, voff = _scene()
    pd = params_of(synth.SimConfig(k_c=1e5, self_collision=True, dcd_radius=0.05, ccd_interval=interval))
    v0 = np.zeros_like(m.rest)
    v0[voff[1]:, 2] = -6.0
    err, x, v, counts = _run(orc, m, pd, v0, 1 / 60, 30, 12)
    print("fast block, CCD every %d: err/bbox %.2e, CCD pairs %s" % (interval, err, counts))
    assert max(counts) >= 4  # the bottom vertices were caught by CCD
    top = m.rest[:voff[1], 2].max()
    assert x[voff[1]:, 2].min() > top - 0.02  # and the block stayed on top
    assert err <= TOL


@pytest.mark.parametrize("extra", [dict(cheby_rho=0.7), dict(k_d=1e-5), dict(mu_c=0.3, eps_v=1e-2)],
                         ids=["chebyshev", "damping", "friction"])
def test_oblique_throw_with_options_matches_oracle(orc, extra):
    """A block thrown down and sideways: it lands on the pinned block and
    slides (with friction, stops) while CCD runs every 2 iterations."""
    m, voff = _scene(seed=141, origin=(0.03, 0.02, 0.12))
    pd = params_of(synth.SimConfig(k_c=1e5, self_collision=True, dcd_radius=0.05, ccd_interval=2), **extra)
    v0 = np.zeros_like(m.rest)
    v0[voff[1]:] = (0.8, 0.3, -5.0)
    err, x, v, counts = _run(orc, m, pd, v0, 1 / 60, 20, 12)
    print("oblique throw %s: err/bbox %.2e, CCD pairs %s" % (extra, err, counts))
    assert max(counts) >= 4
    assert err <= TOL


@pytest.mark.parametrize("seed", range(4))
def test_seeded_throws_match_oracle(orc, seed):
    rng = np.random.default_rng(150 + seed)
    dims = (int(rng.integers(1, 3)), int(rng.integers(1, 3)), 1)
    origin = (float(rng.uniform(0.01, 0.09)), float(rng.uniform(0.01, 0.09)), float(rng.uniform(0.105, 0.14)))
    m, voff = _scene(seed=160 + seed, origin=origin, upper_dims=dims)
    interval = int(rng.integers(1, 6))
    pd = params_of(synth.SimConfig(k_c=1e5, self_collision=True, dcd_radius=0.05, ccd_interval=interval))
    v0 = np.zeros_like(m.rest)
    v0[voff[1]:] = (rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(-7.0, -3.0))
    err, x, v, counts = _run(orc, m, pd, v0, 1 / 60, 25, 10)
    print("seed %d (dims %s, CCD every %d): err/bbox %.2e, CCD pairs %s" % (seed, dims, interval, err, counts))
    assert max(counts) >= 1
    assert err <= TOL


# ---- edge-edge pairs ----------------------------------------------------------

def _run_ee(orc, m, pd, v0, h, iters, steps):
    """Like _run, comparing the edge-edge pairs (partner per boundary edge)
    as well; returns the worst error (/ bbox), the final positions and the
    edge-edge pair count after each step."""
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(**pd)
    sim = vbd.Sim(m, vbd.make_params(**pd))
    counts = []
    try:
        edges, _ = vbd.vbd_get_edge_pairs(sim.ctx, with_partners=False)
        assert np.array_equal(edges, model.edges())  # same boundary edges, same order
        colors = vbd.vbd_get_colors(sim.ctx, m.n_verts)
        nc = int(colors.max()) + 1
        x = _f32(m.rest)
        v = _f32(v0)
        vp = v.copy()
        sim.set_state(x, v)
        worst = 0.0
        for step in range(steps):
            sim.step(h, iters)
            model.step(p, colors, nc, h, iters, x, v, vp)
            got = vbd.vbd_get_contacts(sim.ctx, m.n_verts)
            assert np.array_equal(got, model.contacts()), step
            _, partner = vbd.vbd_get_edge_pairs(sim.ctx)
            want = model.ee_pairs()[0]
            bad = np.nonzero(partner != want)[0]
            assert bad.size == 0, (step, bad, partner[bad], want[bad])
            counts.append(int((want >= 0).sum()))
            xg, _ = sim.get_state()
            worst = max(worst, float(np.abs(xg.cpu().numpy() - x).max()))
            print("  step %d: err/bbox %.2e, edge-edge pairs %d" % (step, worst / bbox_diag(m.rest), counts[-1]))
        sim.sync_status()
    finally:
        sim.close()
    return worst / bbox_diag(m.rest), x, counts


def _ridges():
    rest = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, -1], [0, 1, -1],
                     [0, -1, 0.3], [0, 1, 0.3], [-1, 0, 1.3], [1, 0, 1.3]], float) * 0.1
    return synth.MeshInput(rest=rest, tets=np.array([[0, 1, 2, 3], [4, 5, 6, 7]], np.int32),
                           young=np.full(2, 1e5, np.float32), poisson=np.full(2, 0.3, np.float32),
                           density=np.full(2, 1000.0, np.float32),
                           pinned=np.array([1, 1, 1, 1, 0, 0, 0, 0], np.uint8))


@pytest.mark.parametrize("interval", [1, 4])
def test_crossing_ridges_match_oracle(orc, interval):
    """Two tets meeting ridge to ridge (no vertex ever meets a face): only
    edge-edge pairs act.  A ridge balanced on a ridge then tips over (an
    unstable rest), so the comparison stops after 5 steps."""
    m = _ridges()
    pd = params_of(synth.SimConfig(k_c=1e5, self_collision=True, dcd_radius=0.01, ccd_interval=interval,
                                   ccd_edges=True))
    v0 = np.zeros_like(m.rest)
    v0[4:, 2] = -1.5
    err, x, counts = _run_ee(orc, m, pd, v0, 1 / 60, 20, 5)
    print("ridges, CCD every %d: err/bbox %.2e, edge-edge pairs %s" % (interval, err, counts))
    assert max(counts) >= 1
    assert err <= TOL


def test_crossed_bars_match_oracle(orc):
    """A bar thrown crosswise onto a pinned bar: vertex-triangle and
    edge-edge pairs together, with Chebyshev."""
    lower = synth.beam(6, 1, 1, edge=0.05, E=1e5, nu=0.4, pin_face="z-", jitter_frac=0.03, seed=181)
    upper = synth.beam(1, 6, 1, edge=0.05, E=1e5, nu=0.4, pin_face=None, jitter_frac=0.03, seed=182,
                       origin=(0.12, -0.12, 0.07))
    cat, voff, _ = synth.concat([lower, upper])
    cat.grid_ijk = None
    pd = params_of(synth.SimConfig(k_c=1e5, self_collision=True, dcd_radius=0.02, ccd_interval=2,
                                   ccd_edges=True), cheby_rho=0.6)
    v0 = np.zeros_like(cat.rest)
    v0[voff[1]:, 2] = -3.0
    err, x, counts = _run_ee(orc, cat, pd, v0, 1 / 60, 20, 10)
    print("crossed bars: err/bbox %.2e, edge-edge pairs %s" % (err, counts))
    assert err <= TOL


def test_interpenetrating_slabs_with_vertex_ccd_match_oracle(orc):
    """The slab scene pushing apart with vertex-triangle CCD every 3
    iterations beside the step-start DCD: DCD pairs for the vertices inside
    the other slab, CCD pairs for those that cross a face during a step;
    every pair compared exactly after every step."""
    m, cfg, _ = synth.colliding_slabs(n=8, seed=43)
    pd = params_of(cfg, ccd_interval=3)
    err, x, v, counts = _run(orc, m, pd, np.zeros_like(m.rest), cfg.h, cfg.iters, 6)
    print("slabs with vertex CCD: err/bbox %.2e, CCD pairs %s" % (err, counts))
    assert max(counts) >= 2
    assert err <= TOL


def test_interpenetrating_slabs_edge_pairs_match_oracle(orc):
    """The self-collision slab scene (two jittered slabs sunk into each
    other, 936 boundary edges) with vertex-triangle and edge-edge CCD every 5
    iterations: about a hundred edge pairs held at once, compared exactly
    after every step, positions within 1e-5 of the bounding box."""
    m, cfg, _ = synth.colliding_slabs(n=8, seed=41)
    pd = params_of(cfg, ccd_interval=5, ccd_edges=True)
    err, x, counts = _run_ee(orc, m, pd, np.zeros_like(m.rest), cfg.h, cfg.iters, 6)
    print("slabs with edge pairs: err/bbox %.2e, edge-edge pairs %s" % (err, counts))
    assert min(counts) >= 50
    assert err <= TOL


def test_large_slabs_ccd_sampled(orc):
    """The slab scene at bench size (900,010 vertices, 734,352 boundary
    triangles) with the upper slab thrown down at 3 m/s (one edge per step)
    and one CCD per step: after the step-start DCD and the CCD before the
    first iteration (paths x^t -> initial guess), the pairs of sampled
    boundary vertices without a step-start pair, each recomputed alone by
    the oracle (brute force over every triangle)."""
    m, cfg, u0 = synth.colliding_slabs(n=300, layers=4, seed=31)
    pd = params_of(cfg, ccd_interval=cfg.iters)
    x = _f32(m.rest)
    v0 = np.zeros_like(x)
    v0[u0:, 2] = -3.0
    sim = vbd.Sim(m, vbd.make_params(**pd), colors=synth.kuhn_coloring(m.grid_ijk))
    try:
        tris = vbd.vbd_get_surface(sim.ctx)
        sim.set_state(x, v0)
        vbd.vbd_begin_step(sim.ctx, cfg.h)
        dcd = vbd.vbd_get_contacts(sim.ctx, m.n_verts)
        xg, _ = sim.get_state()  # the initial guess
        x0 = xg.cpu().numpy().astype(np.float64)
        vbd.vbd_iterate(sim.ctx, 1)  # the CCD runs before iteration 1
        got = vbd.vbd_get_contacts(sim.ctx, m.n_verts)
        vbd.vbd_end_step(sim.ctx)
        sim.sync_status()
    finally:
        sim.close()
    model = orc.Model.from_mesh(m)
    assert np.array_equal(tris, model.tris())
    surf = np.unique(tris)
    free = surf[dcd[surf] < 0]  # swept by the CCD
    caught = free[got[free] >= 0]
    print("large slabs: %d step-start pairs, %d CCD pairs" % ((dcd >= 0).sum(), caught.size))
    assert caught.size > 1000
    rng = np.random.default_rng(33)
    sample = np.concatenate([rng.choice(caught, 30, replace=False), rng.choice(free, 30, replace=False)])
    want = np.array([model.ccd_vertex(x, x0, a)[0] for a in sample])
    bad = np.nonzero(got[sample] != want)[0]
    assert bad.size == 0, (sample[bad], got[sample][bad], want[bad])


def test_large_slabs_edge_ccd_sampled(orc):
    """Edge-edge CCD at bench size (1.1M boundary edges) with the upper slab
    thrown down at 3 m/s: each sampled edge's first hit, recomputed alone by
    the oracle (brute force over every edge), is the edge's partner or, for
    a pair found from both sides, held by the partner (lower index)."""
    m, cfg, u0 = synth.colliding_slabs(n=300, layers=4, seed=31)
    pd = params_of(cfg, ccd_interval=cfg.iters, ccd_edges=True)
    x = _f32(m.rest)
    v0 = np.zeros_like(x)
    v0[u0:, 2] = -3.0
    sim = vbd.Sim(m, vbd.make_params(**pd), colors=synth.kuhn_coloring(m.grid_ijk))
    try:
        edges, _ = vbd.vbd_get_edge_pairs(sim.ctx, with_partners=False)
        sim.set_state(x, v0)
        vbd.vbd_begin_step(sim.ctx, cfg.h)
        xg, _ = sim.get_state()  # the initial guess
        x0 = xg.cpu().numpy().astype(np.float64)
        vbd.vbd_iterate(sim.ctx, 1)  # the CCD runs before iteration 1
        _, partner = vbd.vbd_get_edge_pairs(sim.ctx)
        vbd.vbd_end_step(sim.ctx)
        sim.sync_status()
    finally:
        sim.close()
    model = orc.Model.from_mesh(m)
    assert np.array_equal(edges, model.edges())
    held = np.nonzero(partner >= 0)[0]
    print("large slabs: %d of %d edges hold an edge-edge pair" % (held.size, partner.size))
    assert held.size > 1000
    rng = np.random.default_rng(34)
    sample = np.concatenate([rng.choice(held, 12, replace=False), rng.choice(partner.size, 12, replace=False)])
    for e in sample:
        f, _, _ = model.ee_first_hit(x, x0, e)
        if partner[e] >= 0:
            assert f == partner[e], (e, f, partner[e])
        else:
            assert f < 0 or (f < e and partner[f] == e), (e, f, partner[f] if f >= 0 else None)
