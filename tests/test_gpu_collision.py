"""Self-collision (Sec. 3.5, vertex-triangle pairs with the penalty of Eq. 12)
on the GPU against the FP64 oracle: the pairs the detection finds (index
work, compared exactly where the choice is unique), the energy with contact
terms, and whole trajectories with the same colouring (positions within
1e-5 of the bounding-box diagonal)."""
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


def _pairs_agree(orc, model, p, x, tris, got, want):
    """Exact agreement, except where the oracle's decision is not unique at
    FP32 resolution: two triangles equally near (within 1e-5 r), or a vertex
    that is paired on one side only and sits on the penetration boundary (its
    nearest triangle within 1e-5 r) or at the detection distance."""
    bad = np.nonzero(got != want)[0]
    for a in bad:
        dist = {}
        for T in (got[a], want[a]):
            if T >= 0:
                q, _ = orc.closest_point_tri(x[a], *x[tris[T]])
                dist[T] = np.linalg.norm(q - x[a])
        if got[a] >= 0 and want[a] >= 0:
            assert abs(dist[got[a]] - dist[want[a]]) <= 1e-5 * p.dcd_radius, a
        else:
            dT = dist[got[a] if got[a] >= 0 else want[a]]
            assert min(dT, abs(dT - p.dcd_radius)) <= 1e-5 * p.dcd_radius, a
    return len(bad)


def _sim(m, pd, colors):
    return vbd.Sim(m, vbd.make_params(**pd), colors=colors)


@pytest.mark.parametrize("angle,sink", [(0.15, 0.1), (0.6, 0.35)])
def test_detection_matches_oracle(orc, angle, sink):
    m, cfg, _ = synth.colliding_slabs(n=14, angle=angle, sink=sink, seed=21)
    pd = params_of(cfg)
    x = _f32(m.rest)  # positions both sides hold exactly
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(**pd)
    want = model.dcd(p, x)
    sim = _sim(m, pd, None)
    try:
        tris = vbd.vbd_get_surface(sim.ctx)
        assert np.array_equal(tris, model.tris())
        sim.set_state(x, np.zeros_like(x))
        vbd.vbd_begin_step(sim.ctx, cfg.h)  # detection on x^t
        got = vbd.vbd_get_contacts(sim.ctx, m.n_verts)
        vbd.vbd_end_step(sim.ctx)
        _, n_pairs = vbd.vbd_sync_status(sim.ctx, with_contacts=True)
    finally:
        sim.close()
    assert (want >= 0).sum() > 100
    assert n_pairs == int((got >= 0).sum())
    n_bad = _pairs_agree(orc, model, p, x, tris, got, want)
    print("detection angle %.2f sink %.2f: %d pairs, %d differ (ties)" % (angle, sink, (want >= 0).sum(), n_bad))
    assert n_bad <= 2


def test_energy_with_contacts_matches_oracle(orc):
    m, cfg, u0 = synth.colliding_slabs(n=10, seed=22)
    pd = params_of(cfg)
    x = _f32(m.rest)
    v = np.zeros_like(x)
    v[u0:, 2] = -0.5
    v = _f32(v)
    sim = _sim(m, pd, None)
    try:
        sim.set_state(x, v)
        vbd.vbd_begin_step(sim.ctx, cfg.h)
        G_gpu = sim.energy()
        xg, _ = sim.get_state()
        xg = xg.cpu().numpy().astype(np.float64)
        vbd.vbd_end_step(sim.ctx)
    finally:
        sim.close()
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(**pd)
    model.dcd(p, x)
    y = model.inertia_target(p, cfg.h, x, v)
    G0 = model.energy_G(p, cfg.h, xg, y)
    G_nc = model.energy_G(orc.Params.make(**params_of(cfg, self_collision=False)), cfg.h, xg, y)
    assert G0 - G_nc > 1e-3 * abs(G0)  # the contact terms matter here
    assert G_gpu == pytest.approx(G0, rel=1e-5)


def _trajectory(orc, m, pd, h, iters, steps, v0=None):
    """Step by step on both sides with the library's colouring; returns the
    worst position error over the steps (/ bbox), the oracle's final
    positions, and the pair count of each step."""
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(**pd)
    sim = _sim(m, pd, None)
    counts = []
    try:
        colors = vbd.vbd_get_colors(sim.ctx, m.n_verts)
        nc = int(colors.max()) + 1
        tris = vbd.vbd_get_surface(sim.ctx)
        x = _f32(m.rest)
        v = np.zeros_like(x) if v0 is None else _f32(v0)
        vp = v.copy()
        sim.set_state(x, v)
        worst = 0.0
        for step in range(steps):
            vbd.vbd_begin_step(sim.ctx, h)
            got = vbd.vbd_get_contacts(sim.ctx, m.n_verts)
            vbd.vbd_iterate(sim.ctx, iters)
            vbd.vbd_end_step(sim.ctx)
            xt = x.copy()
            model.step(p, colors, nc, h, iters, x, v, vp)  # DCD on x^t, then the iterations
            want = model.contacts()
            assert _pairs_agree(orc, model, p, xt, tris, got, want) == 0, step
            counts.append(int((want >= 0).sum()))
            xg, _ = sim.get_state()
            worst = max(worst, float(np.abs(xg.cpu().numpy() - x).max()))
        sim.sync_status()
    finally:
        sim.close()
    return worst / bbox_diag(m.rest), x, counts


@pytest.mark.parametrize("extra", [dict(), dict(cheby_rho=0.8), dict(k_d=1e-5), dict(mu_c=0.3, eps_v=1e-2)],
                         ids=["plain", "chebyshev", "damping", "friction"])
def test_slabs_trajectory_matches_oracle(orc, extra):
    """10 steps x 20 iterations of the slab scene (870 vertices, about 220
    pairs per step); pairs compared at every step start; self-contact alone,
    with Chebyshev and with Rayleigh damping."""
    m, cfg, u0 = synth.colliding_slabs(seed=7)
    err, x, counts = _trajectory(orc, m, params_of(cfg, **extra), cfg.h, cfg.iters, cfg.steps)
    print("slabs %s: max |x_gpu - x_oracle| / bbox = %.3e, pairs %s" % (extra, err, counts))
    assert min(counts) > 20
    assert np.abs(x - m.rest).max() > 1e-3  # the contact pushed the slabs apart
    assert err <= TOL


def test_blocks_sliding_on_the_ground_with_self_contact(orc):
    """A free 3x3x1 block resting on the ground and a 2x2x1 block sunk 4 mm
    into it, both sliding at 0.3 m/s: ground penalty, ground friction
    (mu = 0.3) and self-contact together, 10 steps x 20 iterations."""
    lower = synth.beam(3, 3, 1, edge=0.1, E=1e5, nu=0.4, pin_face=None, jitter_frac=0.02, seed=111)
    lower.rest[:, 2] -= lower.rest[:, 2].min() - 0.001
    upper = synth.beam(2, 2, 1, edge=0.1, E=1e5, nu=0.4, pin_face=None, jitter_frac=0.02, seed=112,
                       origin=(0.03, 0.04, 0.096))
    cat, voff, _ = synth.concat([lower, upper])
    pd = params_of(synth.SimConfig(k_c=1e5, self_collision=True, dcd_radius=0.05), ground_on=True, mu_c=0.3)
    v0 = np.zeros_like(cat.rest)
    v0[:, 0] = 0.3
    err, x, counts = _trajectory(orc, cat, pd, 1 / 60, 20, 10, v0)
    print("blocks on ground: err / bbox = %.3e, pairs %s" % (err, counts))
    assert min(counts) > 0 and x[:voff[1], 2].min() < 0.0  # both kinds of contact act
    assert err <= TOL


def test_block_sliding_on_a_rigid_block_with_friction(orc):
    """The oracle's Coulomb pin on the GPU: a block sliding at 2 m/s on a
    fully pinned block, friction mu_c = 0.3 on the self-contact pairs; the
    trajectories agree and the GPU's deceleration is mu g."""
    lower = synth.beam(6, 3, 1, edge=0.1, E=1e6, nu=0.3, pin_face="z-")
    lower.pinned[:] = 1
    upper = synth.beam(2, 2, 1, edge=0.1, E=1e6, nu=0.3, pin_face=None, origin=(0.03, 0.04, 0.1 - 5e-5))
    cat, voff, _ = synth.concat([lower, upper])
    pd = params_of(synth.SimConfig(k_c=1e6, self_collision=True, dcd_radius=0.05), mu_c=0.3, eps_v=1e-3)
    v0 = np.zeros_like(cat.rest)
    v0[voff[1]:, 0] = 2.0
    err, x, counts = _trajectory(orc, cat, pd, 1 / 60, 200, 10, v0)
    print("block on rigid block with friction: err / bbox = %.3e, pairs %s" % (err, counts))
    assert min(counts) >= 9 and err <= TOL


def test_jacobi_with_self_contact_first_iterations(orc):
    """Block Jacobi with self-contact (every vertex against the previous
    iterate).  It diverges on this scene after a few steps, as Jacobi does on
    stiff settings, so one step of 3 iterations is compared."""
    m, cfg, u0 = synth.colliding_slabs(seed=7)
    err, x, counts = _trajectory(orc, m, params_of(cfg, jacobi=True), cfg.h, 3, 1)
    print("jacobi + self-contact: err / bbox = %.3e" % err)
    assert counts[0] > 100 and err <= 1e-6


def test_block_rests_on_block_and_falls_through_without_contact(orc):
    """The oracle's drop pin, on the GPU: with self-collision the upper block
    comes to rest on the lower one; without it, it falls through."""
    lower = synth.beam(3, 3, 1, edge=0.1, E=1e5, nu=0.4, pin_face="z-", jitter_frac=0.05, seed=102)
    upper = synth.beam(2, 2, 1, edge=0.1, E=1e5, nu=0.4, pin_face=None, jitter_frac=0.05, seed=103,
                       origin=(0.05, 0.05, 0.102))
    cat, voff, _ = synth.concat([lower, upper])
    v0 = np.zeros_like(cat.rest)
    v0[voff[1]:, 2] = -1.0
    for collide in (True, False):
        pd = params_of(synth.SimConfig(k_c=1e5), self_collision=collide, dcd_radius=0.05)
        sim = _sim(cat, pd, None)
        try:
            sim.set_state(cat.rest, v0)
            for _ in range(20):
                sim.step(1 / 60, 40)
            sim.sync_status()
            x, _ = sim.get_state()
            zmin = float(x.cpu().numpy()[voff[1]:, 2].min())
        finally:
            sim.close()
        if collide:
            assert zmin > 0.1 - 0.01
        else:
            assert zmin < 0.0


def test_self_collision_arguments(orc):
    m, cfg, _ = synth.colliding_slabs(n=6)
    sim = _sim(m, params_of(cfg, self_collision=False), None)
    try:
        with pytest.raises(vbd.VbdError) as e:  # the workspace has no contact arrays
            vbd.vbd_set_params(sim.ctx, vbd.make_params(**params_of(cfg)))
        assert e.value.status == "VBD_ERR_STATE"
        with pytest.raises(vbd.VbdError) as e:
            vbd.vbd_get_contacts(sim.ctx, m.n_verts)
        assert e.value.status == "VBD_ERR_STATE"
    finally:
        sim.close()


def test_large_slabs_detection_sampled(orc):
    """The slab scene at bench size (300x300x4 and 298x298x4 cubes: 900,010
    vertices, 4,291,296 tets, 367,180 boundary vertices): the pairs of sampled
    boundary vertices, each recomputed alone by the oracle (brute force over
    every tet and triangle); then three steps stay finite and lift the
    upper slab's penetrating vertices."""
    m, cfg, u0 = synth.colliding_slabs(n=300, layers=4, seed=31)
    pd = params_of(cfg)
    x = _f32(m.rest)
    sim = _sim(m, pd, synth.kuhn_coloring(m.grid_ijk))
    try:
        tris = vbd.vbd_get_surface(sim.ctx)
        sim.set_state(x, np.zeros_like(x))
        vbd.vbd_begin_step(sim.ctx, cfg.h)
        got = vbd.vbd_get_contacts(sim.ctx, m.n_verts)
        vbd.vbd_iterate(sim.ctx, cfg.iters)
        vbd.vbd_end_step(sim.ctx)
        for _ in range(2):
            sim.step(cfg.h, cfg.iters)
        sim.sync_status()
        xg, _ = sim.get_state()
        xg = xg.cpu().numpy().astype(np.float64)
    finally:
        sim.close()
    model = orc.Model.from_mesh(m)
    assert np.array_equal(tris, model.tris())
    p = orc.Params.make(**pd)
    surf = np.unique(tris)
    rng = np.random.default_rng(32)
    paired = np.nonzero(got >= 0)[0]
    assert paired.size > 1000
    sample = np.concatenate([rng.choice(paired, 30, replace=False), rng.choice(surf, 30, replace=False)])
    want = got.copy()
    for a in sample:
        want[a] = model.dcd_vertex(p, x, a)
    assert _pairs_agree(orc, model, p, x, tris, got[sample], want[sample]) == 0
    assert np.isfinite(xg).all()
    # the overlap shrinks: the upper slab's penetrating vertices rise on average
    sunk = paired[paired >= u0]
    assert sunk.size > 1000 and xg[sunk, 2].mean() > x[sunk, 2].mean()


def test_positions_beyond_the_grid_range_are_reported(orc):
    """The detection grid is exact while positions stay within 65536 cells of
    the origin; a scene moved 1e5 m away is detected safely (coordinates are
    clamped) and vbd_sync_status reports VBD_ERR_RANGE."""
    m, cfg, _ = synth.colliding_slabs(n=6)
    m.rest = m.rest + np.array([1e5, 0.0, 0.0])
    sim = _sim(m, params_of(cfg), None)
    try:
        sim.set_state(m.rest, np.zeros_like(m.rest))
        sim.step(cfg.h, 2)
        with pytest.raises(vbd.VbdError) as e:
            sim.sync_status()
        assert e.value.status == "VBD_ERR_RANGE"
        sim.sync_status()  # the counter was cleared by the report
    finally:
        sim.close()


def _random_blocks(seed: int):
    rng = np.random.default_rng(2000 + seed)
    e = 0.05
    nl = [int(v) for v in rng.integers(3, 7, 2)] + [int(rng.integers(1, 3))]
    nu = [int(v) for v in rng.integers(2, 5, 2)] + [int(rng.integers(1, 3))]
    lower = synth.beam(*nl, edge=e, E=float(np.exp(rng.uniform(np.log(3e4), np.log(3e5)))), nu=0.4,
                       pin_face="z-", jitter_frac=float(rng.uniform(0.0, 0.06)), seed=int(rng.integers(1 << 30)))
    upper = synth.beam(*nu, edge=e, E=float(np.exp(rng.uniform(np.log(3e4), np.log(3e5)))), nu=0.4,
                       pin_face=None, jitter_frac=float(rng.uniform(0.0, 0.06)), seed=int(rng.integers(1 << 30)))
    ang = float(rng.uniform(-0.4, 0.4))
    c, s_ = np.cos(ang), np.sin(ang)
    R = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])
    top = nl[2] * e
    sink = float(rng.uniform(0.02, 0.3)) * e
    centre = upper.rest.mean(axis=0)
    target = np.array([0.5 * nl[0] * e + rng.uniform(-0.1, 0.1) * e, 0.5 * nl[1] * e + rng.uniform(-0.1, 0.1) * e,
                       top + 0.5 * nu[2] * e - sink])
    upper.rest = (upper.rest - centre) @ R.T + target
    cat, voff, _ = synth.concat([lower, upper])
    pd = params_of(synth.SimConfig(k_c=float(rng.choice([3e4, 1e5, 3e5])), self_collision=True,
                                   dcd_radius=float(rng.uniform(0.3, 0.6)) * e),
                   cheby_rho=float(rng.choice([0.0, 0.0, 0.7])), k_d=float(rng.choice([0.0, 1e-6])),
                   mu_c=float(rng.choice([0.0, 0.2, 0.5])), eps_v=float(rng.choice([1e-3, 1e-2])))
    v0 = np.zeros_like(cat.rest)
    v0[voff[1]:] = rng.normal(0.0, 0.2, 3)
    return cat, pd, v0, int(rng.integers(5, 20)), int(rng.integers(3, 7))


@pytest.mark.parametrize("seed", range(8))
def test_random_block_pairs_match_oracle(orc, seed):
    """Seeded random pairs of blocks (sizes, materials, jitter, a turned and
    sunk upper block, radius, k_c, friction, Chebyshev, damping, velocity):
    pairs equal at every step start, positions within 1e-5 of the bbox."""
    cat, pd, v0, iters, steps = _random_blocks(seed)
    err, x, counts = _trajectory(orc, cat, pd, 1 / 60, iters, steps, v0)
    print("random blocks %d: %d verts, pairs %s, err / bbox %.2e" % (seed, cat.n_verts, counts, err))
    assert max(counts) > 0 and err <= TOL
