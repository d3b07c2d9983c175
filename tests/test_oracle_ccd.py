"""Pins of the oracle's vertex-triangle CCD (Sec. 3.5: collisions found
during the iterations by continuous detection along the straight paths from
x^t to the current iterate, every n_col iterations; the impact point keeps
its barycentric weights while the pair lives).  CPU only."""
import numpy as np
import pytest

from paper_2403_06321_b300 import synth

H = 1.0 / 60.0


def test_cubic_first_root_against_numpy_roots(orc):
    """The earliest real root in [t_min, 1] against numpy's companion-matrix
    roots, for random cubics with three real roots spread over [-0.5, 1.5]
    and random leading coefficients (cases with two roots closer than 1e-3
    are left out: there the answer is ill-conditioned)."""
    rng = np.random.default_rng(121)
    checked = 0
    for _ in range(3000):
        roots = np.sort(rng.uniform(-0.5, 1.5, 3))
        if np.diff(roots).min() < 1e-3:
            continue
        k = rng.choice([-1, 1]) * 10 ** rng.uniform(-3, 2)
        c = k * np.array([-roots.prod(), roots[0] * roots[1] + roots[0] * roots[2] + roots[1] * roots[2],
                          -roots.sum(), 1.0])
        t_min = float(rng.choice([0.0, rng.uniform(0, 1)]))
        want = roots[(roots >= t_min) & (roots <= 1.0)]
        got = orc.cubic_first_root(c, t_min)
        if want.size == 0:
            assert got == -1.0
        else:
            assert got == pytest.approx(want[0], abs=1e-10)
        checked += 1
    assert checked > 2500
    assert orc.cubic_first_root([0.0, 0.0, 0.0, 0.0]) == -1.0  # coplanar motion: no impact
    assert orc.cubic_first_root([0.0, 1.0, 0.0, 0.0]) == 0.0  # touching at the start
    assert orc.cubic_first_root([-0.25, 1.0, 0.0, 0.0]) == pytest.approx(0.25)  # linear
    assert orc.cubic_first_root([0.01, 0.0, -1.0, 0.0]) == pytest.approx(0.1)  # quadratic


def _tet_pair(apex0, apex1, move_lower=None):
    """Lower tet with an upward-facing top face z = 0; the upper tet's apex
    (vertex 4) moves from apex0 to apex1, the rest of it stays far above."""
    rest = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.2, 0.2, -1.0],
                     apex0, [0, 0, 3.0], [1, 0, 3.0], [0, 1, 3.0]], float)
    m = synth.MeshInput(rest=rest, tets=np.array([[0, 1, 2, 3], [4, 5, 6, 7]], np.int32),
                        young=np.full(2, 1e5, np.float32), poisson=np.full(2, 0.3, np.float32),
                        density=np.full(2, 1000.0, np.float32), pinned=np.zeros(8, np.uint8))
    x0 = rest.copy()
    x1 = rest.copy()
    x1[4] = apex1
    if move_lower is not None:
        x1[:4] = move_lower(x1[:4])
    return m, x0, x1


def _top_face(model):
    tris = model.tris()
    for T, t in enumerate(tris):
        if sorted(t.tolist()) == [0, 1, 2]:
            return T, t
    raise AssertionError("top face missing")


def test_vertex_through_a_static_face_closed_form(orc):
    """A vertex moving in a straight line through a static horizontal face
    hits it when its height reaches zero, at the point it crosses; the
    weights are that point's barycentric coordinates."""
    a0, a1 = np.array([0.2, 0.3, 0.5]), np.array([0.25, 0.2, -0.5])
    m, x0, x1 = _tet_pair(a0, a1)
    model = orc.Model.from_mesh(m)
    T, t = _top_face(model)
    got_T, toi, w = model.ccd_vertex(x0, x1, 4)
    assert got_T == T
    assert toi == pytest.approx(0.5, abs=1e-12)
    q = a0 + 0.5 * (a1 - a0)
    bary = {0: 1 - q[0] - q[1], 1: q[0], 2: q[1]}
    assert np.allclose(w, [bary[int(v)] for v in t], atol=1e-12)
    # the pair acts through the impact point, not the nearest point at x1:
    # corner k gets -k_c d w_k n with d = (q - x_a).n = 0.5
    p = orc.Params.make(self_collision=True, dcd_radius=0.05, k_c=1e5)
    assert model.ccd(x0, x1) == 1
    for v in t:
        f, _, hit = model.self_contact(p, int(v), x1)
        assert hit and np.allclose(f, [0.0, 0.0, -1e5 * 0.5 * bary[int(v)]], rtol=1e-12, atol=1e-9)
    # passing beside the face: no impact
    m2, x0, x1 = _tet_pair(np.array([0.8, 0.8, 0.5]), np.array([0.8, 0.8, -0.5]))
    assert orc.Model.from_mesh(m2).ccd_vertex(x0, x1, 4)[0] == -1
    # moving away from the face: no impact
    m3, x0, x1 = _tet_pair(np.array([0.2, 0.3, 0.5]), np.array([0.2, 0.3, 0.9]))
    assert orc.Model.from_mesh(m3).ccd_vertex(x0, x1, 4)[0] == -1


def test_moving_face_against_dense_sampling(orc):
    """The lower tet translates, rotates and deforms while the vertex moves:
    the impact time and weights agree with a dense scan of the coplanarity
    sign along the path (20,001 samples, crossing located by interpolation,
    weights from the positions at that time), for random seeded motions
    whose impact is clear of the face's edges."""
    rng = np.random.default_rng(122)
    hits = 0
    for trial in range(60):
        ang = rng.normal(0, 0.4, 3)
        shift = rng.normal(0, 0.2, 3)

        def move(p, ang=ang, shift=shift):
            c, s = np.cos(ang[2]), np.sin(ang[2])
            R = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
            out = p @ R.T + shift
            out[1] += ang[:3] * 0.1  # corner 1 deforms the face
            return out

        a0 = np.array([rng.uniform(0, 0.5), rng.uniform(0, 0.5), rng.uniform(0.2, 0.8)])
        a1 = a0 + rng.normal(0, 0.4, 3) + np.array([0, 0, -1.0])
        m, x0, x1 = _tet_pair(a0, a1, move)
        model = orc.Model.from_mesh(m)
        T, t = _top_face(model)
        got_T, toi, w = model.ccd_vertex(x0, x1, 4)
        ts = np.linspace(0, 1, 20001)
        P = [(1 - ts)[:, None] * x0[k] + ts[:, None] * x1[k] for k in (4, *t)]
        f = np.einsum("ij,ij->i", P[1] - P[0], np.cross(P[2] - P[0], P[3] - P[0]))
        sc = np.nonzero(np.sign(f[:-1]) != np.sign(f[1:]))[0]
        want = None
        for i in sc:
            tc = ts[i] - f[i] * (ts[i + 1] - ts[i]) / (f[i + 1] - f[i])
            pa, p1, p2, p3 = [(1 - tc) * x0[k] + tc * x1[k] for k in (4, *t)]
            n = np.cross(p2 - p1, p3 - p1)
            wb = np.array([np.cross(p2 - pa, p3 - pa) @ n, np.cross(p3 - pa, p1 - pa) @ n,
                           np.cross(p1 - pa, p2 - pa) @ n]) / (n @ n)
            if wb.min() >= 0:
                want = (tc, wb)
                break
        if want is None:
            assert got_T == -1, trial  # no crossing inside the face along the path
            continue
        if want[1].min() < 1e-3:  # too near an edge for the scan's resolution
            continue
        hits += 1
        assert got_T == T, trial
        assert toi == pytest.approx(want[0], abs=1e-6)
        assert np.allclose(w, want[1], atol=1e-5)
    assert hits >= 15


def test_earliest_of_two_faces_wins(orc):
    """A vertex falling through two stacked tets' top faces is caught by the
    upper face first."""
    rest = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.2, 0.2, -0.5],
                     [0, 0, -1], [1, 0, -1], [0, 1, -1], [0.2, 0.2, -1.5],
                     [0.2, 0.3, 0.5], [0, 0, 3.0], [1, 0, 3.0], [0, 1, 3.0]], float)
    m = synth.MeshInput(rest=rest, tets=np.array([[0, 1, 2, 3], [4, 5, 6, 7], [8, 9, 10, 11]], np.int32),
                        young=np.full(3, 1e5, np.float32), poisson=np.full(3, 0.3, np.float32),
                        density=np.full(3, 1000.0, np.float32), pinned=np.zeros(12, np.uint8))
    model = orc.Model.from_mesh(m)
    x1 = rest.copy()
    x1[8] = (0.2, 0.3, -1.5)
    T, toi, _ = model.ccd_vertex(rest, x1, 8)
    assert sorted(model.tris()[T].tolist()) == [0, 1, 2]
    assert toi == pytest.approx(0.25, abs=1e-12)


def test_impact_pair_force_is_the_penalty_gradient(orc):
    """A vertex driven straight down through a static face: the CCD pair's
    impact point lies right above it, so the normal's own variation drops
    out and the forces k_c d n (vertex) and -k_c d w_k n (corners) are -dE/dx
    of the energy; they sum to zero."""
    a0, a1 = np.array([0.2, 0.3, 0.5]), np.array([0.2, 0.3, -0.02])
    m, x0, x1 = _tet_pair(a0, a1)
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(self_collision=True, dcd_radius=0.05, k_c=1e5)
    assert model.ccd(x0, x1) == 1
    w, is_ccd = model.contact_weights()
    assert is_ccd[4] and not is_ccd[:4].any()
    y = x1.copy()
    el = model.elastic_grad(x1).reshape(-1, 3)
    total = np.zeros(3)
    for v in (4, 0, 1, 2):
        f, _, hit = model.self_contact(p, v, x1)
        assert hit
        g = np.zeros(3)
        for r in range(3):
            xp, xm = x1.copy(), x1.copy()
            xp[v, r] += 1e-7
            xm[v, r] -= 1e-7
            g[r] = (model.energy_G(p, H, xp, y) - model.energy_G(p, H, xm, y)) / 2e-7
        g -= el[v]
        assert np.allclose(f, -g, rtol=1e-5, atol=1e-6 * np.abs(f).max())
        total += f
    assert np.abs(total).max() <= 1e-9
    f4, _, _ = model.self_contact(p, 4, x1)
    assert f4 == pytest.approx([0, 0, 1e5 * 0.02], rel=1e-9)


def _fast_blocks(seed=131):
    lower = synth.beam(3, 3, 1, edge=0.1, E=1e5, nu=0.4, pin_face="z-", jitter_frac=0.03, seed=seed)
    upper = synth.beam(2, 2, 1, edge=0.1, E=1e5, nu=0.4, pin_face=None, jitter_frac=0.03, seed=seed + 1,
                       origin=(0.05, 0.05, 0.13))
    cat, voff, _ = synth.concat([lower, upper])
    cat.grid_ijk = None
    return cat, voff


@pytest.mark.parametrize("interval", [0, 1, 5])
def test_fast_block_is_stopped_only_with_ccd(orc, interval):
    """A block thrown down at 6 m/s at a block 3 cm below covers 10 cm per
    step: the step-start DCD alone never sees it penetrate before it has
    passed the upper face, and it tunnels into (and through) the lower
    block; CCD along each step's predicted path catches the top face and
    the block comes to rest on it."""
    cat, voff = _fast_blocks()
    model = orc.Model.from_mesh(cat)
    colors, nc = orc.color_greedy(cat.n_verts, cat.tets)
    p = orc.Params.make(gravity=(0, 0, -9.8), self_collision=True, dcd_radius=0.05, k_c=1e5,
                        ccd_interval=interval)
    v0 = np.zeros_like(cat.rest)
    v0[voff[1]:, 2] = -6.0
    x, v, _ = orc.run(model, p, colors, nc, H, 30, 20, cat.rest, v0)
    zmin_upper = x[voff[1]:, 2].min()
    top = cat.rest[:voff[1], 2].max()
    if interval:
        assert zmin_upper > top - 0.02, zmin_upper
        assert abs(v[voff[1]:, 2].mean()) < 0.2  # at rest on the lower block
    else:
        assert zmin_upper < top - 0.05, zmin_upper  # tunnelled


def test_ccd_keeps_step_start_pairs_and_replaces_its_own(orc):
    """Vertices paired by the DCD keep their pairs; a later CCD drops the
    earlier CCD pairs it no longer finds."""
    a0, a1 = np.array([0.2, 0.3, 0.5]), np.array([0.25, 0.2, -0.5])
    m, x0, x1 = _tet_pair(a0, a1)
    model = orc.Model.from_mesh(m)
    assert model.ccd(x0, x1) == 1
    assert model.contacts()[4] >= 0
    assert model.ccd(x0, x0) == 0  # no motion: no impact, the CCD pair goes
    assert model.contacts()[4] == -1
    p = orc.Params.make(self_collision=True, dcd_radius=0.6)
    xin = x0.copy()
    xin[4] = (0.2, 0.2, -0.05)  # inside the lower tet at the step start
    model.dcd(p, xin)
    T = model.contacts()[4]
    assert T >= 0
    model.ccd(xin, x0)
    assert model.contacts()[4] == T and not model.contact_weights()[1][4]


# ---- edge-edge CCD ---------------------------------------------------------

def test_edge_edge_impact_closed_form(orc):
    """A static edge along x and an edge along y falling through it: they
    cross when the falling edge reaches z = 0, at the parameters of the
    crossing point on each edge; passing beyond an end or moving in parallel
    is no impact."""
    x0 = np.array([[-1, 0.1, 0], [1, 0.1, 0], [0.3, -1, 0.5], [0.3, 1, 0.5]], float)
    x1 = x0.copy()
    x1[2:, 2] = -0.5
    t, s, u = orc.ee_impact(x0, x1, 0, 1, 2, 3)
    assert t == pytest.approx(0.5, abs=1e-12)
    assert s == pytest.approx(0.65, abs=1e-12) and u == pytest.approx(0.55, abs=1e-12)
    x0b, x1b = x0.copy(), x1.copy()
    x0b[2:, 0] = x1b[2:, 0] = 1.5  # beyond the static edge's end
    assert orc.ee_impact(x0b, x1b, 0, 1, 2, 3)[0] == -1.0
    x0c, x1c = x0.copy(), x1.copy()
    x0c[2:] = [[-1, 0.5, 0.5], [1, 0.5, 0.5]]  # parallel to the static edge
    x1c[2:] = [[-1, 0.5, -0.5], [1, 0.5, -0.5]]
    assert orc.ee_impact(x0c, x1c, 0, 1, 2, 3)[0] == -1.0


@pytest.mark.parametrize("deg, paired", [(5.0, False), (5.70, False), (5.78, True), (6.5, True), (30.0, True)])
def test_edge_edge_pairs_skip_edges_within_about_6_degrees_of_parallel(orc, deg, paired):
    """The crossing point of two nearly parallel segments is ill-conditioned,
    so edges whose directions make an angle theta with sin(theta) <= 0.1
    (theta <= 5.74 degrees) are not paired (their end points' vertex-triangle
    pairs take them).  A unit edge at angle theta to a static edge along x,
    centred above it, falls through it: above the threshold it is paired at
    t = 0.5 with the crossing at s = 0.65 on the static edge and at the
    falling edge's midpoint (u = 0.5); below it, never."""
    th = np.radians(deg)
    dv = 0.5 * np.array([np.cos(th), np.sin(th), 0.0])
    c = np.array([0.3, 0.1, 0.5])
    x0 = np.array([[-1, 0.1, 0], [1, 0.1, 0], c - dv, c + dv], float)
    x1 = x0.copy()
    x1[2:, 2] = -0.5
    t, s, u = orc.ee_impact(x0, x1, 0, 1, 2, 3)
    if paired:
        assert t == pytest.approx(0.5, abs=1e-12)
        assert s == pytest.approx(0.65, abs=1e-9) and u == pytest.approx(0.5, abs=1e-9)
    else:
        assert t == -1.0


def test_edge_edge_impact_against_dense_sampling(orc):
    """Random rotating, translating, stretching edge pairs: the first time
    the four points become coplanar with the segments crossing, from a
    20,001-sample scan of the coplanarity sign, matches the root finder
    (crossings within 1e-3 of a segment end are left out)."""
    rng = np.random.default_rng(171)
    hits = 0
    for trial in range(80):
        x0 = rng.normal(0, 1, (4, 3))
        x1 = x0 + rng.normal(0, 1, (4, 3))
        t, s, u = orc.ee_impact(x0, x1, 0, 1, 2, 3)
        ts = np.linspace(0, 1, 20001)
        P = [(1 - ts)[:, None] * x0[k] + ts[:, None] * x1[k] for k in range(4)]
        f = np.einsum("ij,ij->i", P[1] - P[0], np.cross(P[2] - P[0], P[3] - P[0]))
        sc = np.nonzero(np.sign(f[:-1]) != np.sign(f[1:]))[0]
        want = None
        for i in sc:
            tc = ts[i] - f[i] * (ts[i + 1] - ts[i]) / (f[i + 1] - f[i])
            p0, p1, q0, q1 = [(1 - tc) * x0[k] + tc * x1[k] for k in range(4)]
            e, g, w = p1 - p0, q1 - q0, q0 - p0
            n = np.cross(e, g)
            ss, uu = np.cross(w, g) @ n / (n @ n), np.cross(w, e) @ n / (n @ n)
            if 0 <= ss <= 1 and 0 <= uu <= 1:
                want = (tc, ss, uu)
                break
        if want is None:
            assert t == -1.0, trial
            continue
        if min(want[1], 1 - want[1], want[2], 1 - want[2]) < 1e-3:
            continue
        hits += 1
        assert t == pytest.approx(want[0], abs=1e-6), trial
        assert s == pytest.approx(want[1], abs=1e-4) and u == pytest.approx(want[2], abs=1e-4)
    assert hits >= 10


def _ridges(drop=1.0):
    """A lower tet whose top is a ridge along x at z = 0 and an upper tet
    whose bottom is a ridge along y at z = 0.3: the ridges are the bodies'
    extreme points, so falling onto each other they meet edge to edge."""
    rest = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, -1], [0, 1, -1],
                     [0, -1, 0.3], [0, 1, 0.3], [-1, 0, 1.3], [1, 0, 1.3]], float)
    m = synth.MeshInput(rest=rest, tets=np.array([[0, 1, 2, 3], [4, 5, 6, 7]], np.int32),
                        young=np.full(2, 1e5, np.float32), poisson=np.full(2, 0.3, np.float32),
                        density=np.full(2, 100.0, np.float32), pinned=np.array([1, 1, 1, 1, 0, 0, 0, 0], np.uint8))
    return m


def test_crossing_ridges_are_held_apart(orc):
    """Thrown down onto the lower ridge, the upper ridge tunnels through it
    with vertex-triangle CCD alone, since no vertex ever meets a face; the
    edge-edge pairs stop it."""
    m = _ridges()
    model = orc.Model.from_mesh(m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    p = orc.Params.make(gravity=(0, 0, -9.8), self_collision=True, dcd_radius=0.1, k_c=1e5, ccd_interval=1,
                        ccd_edges=True)
    v0 = np.zeros_like(m.rest)
    v0[4:, 2] = -12.0  # 0.2 m per step
    x, v, vp = m.rest.copy(), v0.copy(), v0.copy()
    n_ee = []
    for _ in range(10):
        model.step(p, colors, nc, H, 20, x, v, vp)
        n_ee.append(len(model.ee_pair_list()))
    assert max(n_ee) >= 1
    assert x[[4, 5], 2].min() > -0.05  # the upper ridge stays on the lower one
    # the ridges' crossing point: the upper ridge's vertices straddle x = 0
    x2, v2, vp2 = m.rest.copy(), v0.copy(), v0.copy()
    model2 = orc.Model.from_mesh(m)
    ridge_only = orc.Params.make(gravity=(0, 0, -9.8), self_collision=True, dcd_radius=0.1, k_c=1e5,
                                 ccd_interval=1, ccd_edges=False)
    for _ in range(10):
        model2.step(ridge_only, colors, nc, H, 20, x2, v2, vp2)
    assert x2[[4, 5], 2].min() < -0.5  # with vertex-triangle CCD alone it falls through


def test_edge_edge_force_is_the_penalty_gradient(orc):
    """With the normal frozen, the pair's depth is linear in the four
    positions, so the forces -k_c d c_v n are exactly -dE/dx of the energy
    and sum to zero; the Hessian blocks are k_c c_v^2 n n^T."""
    m = _ridges()
    model = orc.Model.from_mesh(m)
    x0 = m.rest.copy()
    x1 = m.rest.copy()
    x1[4:, 2] -= 0.4  # ridges cross
    x1[4:, 0] += 0.1
    model.ccd(x0, x1)
    pairs = model.ee_pair_list()
    assert len(pairs) == 1 and sorted(pairs[0][0]) == [0, 1, 4, 5]
    verts, su, n = [int(q) for q in pairs[0][0]], pairs[0][1], pairs[0][2]
    assert abs(np.linalg.norm(n) - 1) < 1e-12 and abs(n[2]) > 0.9  # frozen x_b - x_a direction
    p = orc.Params.make(self_collision=True, dcd_radius=0.1, k_c=1e5)
    y = x1.copy()
    el = model.elastic_grad(x1).reshape(-1, 3)
    total = np.zeros(3)
    for vert in (0, 1, 4, 5):
        f, Hc, hit = model.self_contact(p, vert, x1)
        assert hit
        g = np.zeros(3)
        for r in range(3):
            xp, xm = x1.copy(), x1.copy()
            xp[vert, r] += 1e-7
            xm[vert, r] -= 1e-7
            g[r] = (model.energy_G(p, H, xp, y) - model.energy_G(p, H, xm, y)) / 2e-7
        g -= el[vert]
        if model.free[vert]:
            assert np.allclose(f, -g, rtol=1e-6, atol=1e-6 * np.abs(f).max())
        total += f
        j = verts.index(vert)
        c = [-(1 - su[0]), -su[0], 1 - su[1], su[1]][j]
        assert np.allclose(Hc, 1e5 * c * c * np.outer(n, n), rtol=1e-12, atol=1e-6)
    assert np.abs(total).max() <= 1e-9 * max(1.0, np.abs(f).max())
    # back across: no force
    x2 = x1.copy()
    x2[4:, 2] += 0.5
    assert not model.self_contact(p, 4, x2)[2]
