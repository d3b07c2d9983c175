"""Pins of the oracle's world-box walls.  Sec. 3.4 treats unilateral
constraints as potentials; here each wall is one more static half-space
{x : x.n/|n| >= offset} carrying the ground's penalty (Eq. 12, stiffness
k_c) and friction (Eqs. 13-16).  CPU only."""
import numpy as np
import pytest

from paper_2403_06321_b300 import synth

H = 1.0 / 60.0
BOX = [(1, 0, 0, -0.3), (-1, 0, 0, -0.5), (0, 1, 0, -0.3), (0, -1, 0, -0.4), (0, 0, 1, 0.0), (0, 0, -1, -0.4)]


def _rot(a, b, c):
    ca, sa, cb, sb, cc, sc = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(c), np.sin(c)
    rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1]])
    ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    rx = np.array([[1, 0, 0], [0, cc, -sc], [0, sc, cc]])
    return rz @ ry @ rx


def _simulate(orc, m, p, v0, steps, iters, record=False):
    model = orc.Model.from_mesh(m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    x = m.rest.copy()
    v = np.broadcast_to(np.asarray(v0, np.float64), x.shape).copy()
    vp = v.copy()
    xs, vs = [], []
    for _ in range(steps):
        model.step(p, colors, nc, H, iters, x, v, vp)
        if record:
            xs.append(x.copy())
            vs.append(v.copy())
    return (x, v, xs, vs) if record else (x, v)


def test_a_wall_is_the_ground_plane(orc):
    """One wall with the ground's normal and height (non-unit normal) gives
    the ground's trajectory bit for bit, friction included; so does the
    floor given as the last of six walls whose other five are never reached,
    which checks that every wall is visited with its own normal."""
    m = synth.beam(2, 2, 1, edge=0.1, E=1e5, nu=0.3, pin_face=None, origin=(0.0, 0.0, 0.03))
    common = dict(gravity=(0.0, 0.0, -9.8), k_c=1e5, mu_c=0.3, eps_v=1e-2)
    v0 = (0.8, -0.3, -1.0)
    xg, vg = _simulate(orc, m, orc.Params.make(ground_on=True, ground_height=0.01, ground_normal=(0, 0, 2),
                                                **common), v0, 25, 10)
    xw, vw = _simulate(orc, m, orc.Params.make(walls=[(0, 0, 2, 0.01)], **common), v0, 25, 10)
    far = [(1, 0, 0, -9.0), (0, 1, 0, -9.0), (-1, 0, 0, -9.0), (0, -1, 0, -9.0), (0, 0, -1, -9.0)]
    xl, vl = _simulate(orc, m, orc.Params.make(walls=far + [(0, 0, 2, 0.01)], **common), v0, 25, 10)
    assert np.array_equal(xg, xw) and np.array_equal(vg, vw)
    assert np.array_equal(xg, xl) and np.array_equal(vg, vl)
    assert xg[:, 2].min() < 0.01  # the block reached the plane
    assert abs(vg[:, 0].mean()) < 0.8 - 0.1  # and friction slowed it


def test_rotated_scene_gives_the_rotated_motion(orc):
    """Block thrown about a six-wall box with gravity and friction: rotating
    the mesh, gravity and wall normals (offsets unchanged) rotates the
    trajectory."""
    m = synth.beam(2, 2, 1, edge=0.1, E=1e5, nu=0.35, pin_face=None, origin=(0.05, 0.05, 0.05))
    R = _rot(0.4, -0.7, 1.1)
    common = dict(k_c=1e5, mu_c=0.2, eps_v=1e-2)
    g = np.array([0.0, 0.0, -9.8])
    v0 = np.array([3.0, 2.0, 1.0])
    xa, va = _simulate(orc, m, orc.Params.make(gravity=g, walls=BOX, **common), v0, 30, 15)
    mr = synth.beam(2, 2, 1, edge=0.1, E=1e5, nu=0.35, pin_face=None, origin=(0.05, 0.05, 0.05))
    mr.rest = m.rest @ R.T
    walls_r = [tuple(R @ np.array(w[:3], float)) + (w[3],) for w in BOX]
    xb, vb = _simulate(orc, mr, orc.Params.make(gravity=R @ g, walls=walls_r, **common), R @ v0, 30, 15)
    bbox = np.linalg.norm(m.rest.max(0) - m.rest.min(0))
    assert np.abs(xb - xa @ R.T).max() <= 1e-8 * bbox
    assert np.abs(vb - va @ R.T).max() <= 1e-6


def test_block_thrown_in_a_box_bounces_and_stays_in(orc):
    """The block crosses the box and comes back from the +x wall; no vertex
    ever goes further out than one penalty term could with all the initial
    energy, 1/2 k_c d^2 <= E0 (implicit Euler only removes energy)."""
    m = synth.beam(2, 2, 1, edge=0.1, E=1e5, nu=0.35, pin_face=None, origin=(0.05, 0.05, 0.05))
    k_c = 1e5
    v0 = np.array([3.0, 2.0, 1.0])
    _, _, xs, vs = _simulate(orc, m, orc.Params.make(gravity=(0, 0, -9.8), walls=BOX, k_c=k_c), v0, 40, 15,
                             record=True)
    M = float(orc.Model.from_mesh(m).mass().sum())
    E0 = 0.5 * M * float(v0 @ v0) + M * 9.8 * float(m.rest[:, 2].max())
    dmax = np.sqrt(2 * E0 / k_c)
    for x in xs:
        for w in BOX:
            n = np.array(w[:3], float)
            assert (w[3] - x @ n).max() <= dmax
    vx = np.array([v[:, 0].mean() for v in vs])
    assert vx[0] > 2.0 and vx.min() < -0.2  # turned back by the +x wall (implicit Euler damps the bounce)
    assert max(x[:, 0].max() for x in xs) > 0.5  # and pressed into it


def test_weight_on_a_tilted_wall_is_carried_by_its_penalty(orc):
    """A block at rest on a tilted wall, gravity along -n: at steady state
    x = x^t the inertia force is -m g per vertex, elastic forces cancel over
    the body, so the penalty forces add up to the weight, sum k_c d = M |g|,
    and only the face on the wall is pressed in.  The wall is the second of
    two; the first is never reached."""
    m = synth.beam(1, 2, 2, edge=0.1, E=1e6, nu=0.3, pin_face=None)
    R = _rot(0.3, 0.5, -0.2)
    m.rest = m.rest @ R.T
    n = R @ np.array([1.0, 0.0, 0.0])
    k_c = 1e5
    walls = [tuple(-n) + (-5.0,), tuple(3.0 * n) + (0.0,)]
    x, v = _simulate(orc, m, orc.Params.make(gravity=-9.8 * n, walls=walls, k_c=k_c), (0, 0, 0), 40, 300)
    M = float(orc.Model.from_mesh(m).mass().sum())
    d = -(x @ n)
    assert k_c * d[d > 0].sum() == pytest.approx(M * 9.8, rel=1e-4)
    face = np.abs(m.rest @ n) < 1e-12
    assert np.array_equal(d > 0, face)
    assert np.abs(v).max() < 1e-4


def test_block_in_a_tilted_corner_converges_to_dense_newton(orc):
    """Many VBD iterations on a block pressed into a corner of the floor and
    two tilted walls reach the dense global Newton minimiser of Eq. 2 with
    the wall penalties (computed by separate code)."""
    m = synth.beam(2, 1, 1, edge=0.1, E=1e5, nu=0.4, pin_face=None, origin=(-0.01, -0.01, -0.02))
    model = orc.Model.from_mesh(m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    walls = [(1.0, 0.2, 0.1, 0.0), (0.1, 1.0, -0.2, 0.0), (0.0, 0.0, 1.0, 0.0)]
    p = orc.Params.make(gravity=(-2.0, -2.0, -9.8), walls=walls, k_c=1e5)
    xt = m.rest.copy()
    v = np.zeros_like(xt)
    x_vbd, _, _ = orc.run(model, p, colors, nc, H, 4000, 1, xt, v)
    y = model.inertia_target(p, H, xt, v)
    x_nt = model.newton_solve(p, H, xt, y)
    assert np.abs(x_vbd - x_nt).max() <= 1e-9
    for w in walls:  # every wall is pressed
        nh = np.array(w[:3]) / np.linalg.norm(w[:3])
        assert (x_nt @ nh < w[3]).any()


def test_wall_energy_is_the_penalty_and_local_energy_agrees(orc):
    """The walls add sum_i sum_k 1/2 k_c max(0, c_k - x_i.n_k)^2 over the free
    vertices to G (Eq. 12 per half-space), and moving one vertex changes G
    and its G_i by the same amount (Sec. 3.1)."""
    m = synth.beam(3, 2, 2, jitter_frac=0.1, seed=74)
    model = orc.Model.from_mesh(m)
    walls = [(1.0, 0.3, 0.0, 0.2), (0.0, -2.0, 0.5, -0.15), (0.2, 0.1, 1.0, 0.06)]
    p = orc.Params.make(walls=walls, k_c=1e5)
    p0 = orc.Params.make(k_c=1e5)
    rng = np.random.default_rng(76)
    x = m.rest + rng.normal(0, 0.005, m.rest.shape)
    y = x + rng.normal(0, 0.005, m.rest.shape)
    pen, hits = 0.0, np.zeros(m.n_verts, int)
    for w in walls:
        nh = np.array(w[:3]) / np.linalg.norm(w[:3])
        d = np.where(m.pinned == 0, np.maximum(w[3] - x @ nh, 0.0), 0.0)
        assert (d > 0).sum() > 3
        pen += 0.5 * 1e5 * (d * d).sum()
        hits += d > 0
    assert model.energy_G(p, H, x, y) - model.energy_G(p0, H, x, y) == pytest.approx(pen, rel=1e-9)
    # a vertex pressed into all three walls, moved
    i = int(np.nonzero(hits == 3)[0][0])
    x2 = x.copy()
    x2[i] += rng.normal(0, 0.01, 3)
    dG = model.energy_G(p, H, x2, y) - model.energy_G(p, H, x, y)
    dGi = model.local_energy(p, H, i, x2, y) - model.local_energy(p, H, i, x, y)
    assert dGi == pytest.approx(dG, rel=1e-9)
    dG0 = model.local_energy(p0, H, i, x2, y) - model.local_energy(p0, H, i, x, y)
    assert abs(dGi - dG0) > 1e-6 * abs(dGi)  # the walls act on this vertex
