"""Pins of the oracle's self-collision (Sec. 3.5: vertex-triangle penalty of
Eq. 12 with pairs from a DCD at the step start).  CPU only."""
import numpy as np
import pytest

from paper_2403_06321_b300 import synth

H = 1.0 / 60.0


def test_closest_point_on_triangle_beats_dense_sampling(orc):
    rng = np.random.default_rng(101)
    u = np.linspace(0, 1, 161)
    U, V = np.meshgrid(u, u)
    keep = U + V <= 1
    bary = np.stack([1 - U[keep] - V[keep], U[keep], V[keep]], axis=1)
    for _ in range(40):
        a, b, c = rng.normal(size=(3, 3))
        p = rng.normal(size=3) * 1.5
        q, w = orc.closest_point_tri(p, a, b, c)
        assert np.all(w >= -1e-15) and abs(w.sum() - 1) < 1e-12
        assert np.allclose(q, w[0] * a + w[1] * b + w[2] * c)
        samples = bary @ np.stack([a, b, c])
        dmin = np.linalg.norm(samples - p, axis=1).min()
        assert np.linalg.norm(q - p) <= dmin + 1e-12


def test_boundary_triangles_of_a_box(orc):
    """A Kuhn box has 2 triangles per boundary square, normals pointing out,
    total area = box surface area."""
    nx, ny, nz, e = 3, 2, 4, 0.1
    m = synth.beam(nx, ny, nz, edge=e, pin_face=None)
    model = orc.Model.from_mesh(m)
    tris = model.tris()
    assert len(tris) == 2 * 2 * (nx * ny + ny * nz + nz * nx)
    X = m.rest
    centre = X.mean(axis=0)
    area = 0.0
    for t in tris:
        n = np.cross(X[t[1]] - X[t[0]], X[t[2]] - X[t[0]])
        area += 0.5 * np.linalg.norm(n)
        assert n @ (X[t].mean(axis=0) - centre) > 0
    assert area == pytest.approx(2 * e * e * (nx * ny + ny * nz + nz * nx), rel=1e-12)


def _two_blocks(gap, seed=102):
    """A free 2x2x1 block above (or sunk into) a pinned 3x3x1 block."""
    lower = synth.beam(3, 3, 1, edge=0.1, E=1e5, nu=0.4, pin_face="z-", jitter_frac=0.05, seed=seed)
    upper = synth.beam(2, 2, 1, edge=0.1, E=1e5, nu=0.4, pin_face=None, jitter_frac=0.05, seed=seed + 1,
                       origin=(0.05, 0.05, 0.1 + gap))
    cat, voff, _ = synth.concat([lower, upper])
    cat.grid_ijk = None
    return cat, voff


def test_point_in_tet_is_barycentric_membership(orc):
    """Against sampled barycentric combinations: points with all weights >= 0
    are inside, points with one weight < 0 are outside."""
    rng = np.random.default_rng(104)
    for _ in range(20):
        x = rng.normal(size=(4, 3))
        t = np.arange(4)
        for _ in range(20):
            lam = rng.dirichlet(np.ones(4))
            assert orc.point_in_tet(x, t, lam @ x)
            lam[rng.integers(4)] -= 1.0 + rng.random()
            lam /= lam.sum() if abs(lam.sum()) > 1e-3 else 1.0
            if lam.min() < 0 and abs(lam.sum() - 1) < 1e-9:
                assert not orc.point_in_tet(x, t, lam @ x)


def test_dcd_pairs_exactly_the_vertices_inside_the_other_box(orc):
    """Two unjittered boxes, the free 2x2x1 one sunk 1 cm into the pinned
    3x3x1 one.  The paired vertices are those strictly inside the other box
    (a plain box test), each with a triangle of the face it is 1 cm behind;
    lower-box vertices next to the upper box's rim, which lie behind the
    plane of its bottom but outside it, stay unpaired."""
    lower = synth.beam(3, 3, 1, edge=0.1, pin_face="z-")
    upper = synth.beam(2, 2, 1, edge=0.1, pin_face=None, origin=(0.03, 0.04, 0.09))
    cat, voff, _ = synth.concat([lower, upper])
    model = orc.Model.from_mesh(cat)
    p = orc.Params.make(self_collision=True, dcd_radius=0.05, k_c=1e5)
    x = cat.rest
    contact = model.dcd(p, x)
    tris = model.tris()
    lo, hi = np.array([0.0, 0.0, 0.0]), np.array([0.3, 0.3, 0.1])
    ulo, uhi = np.array([0.03, 0.04, 0.09]), np.array([0.23, 0.24, 0.19])
    inside_lower = np.all((x > lo) & (x < hi), axis=1)
    inside_upper = np.all((x > ulo) & (x < uhi), axis=1)
    expect = np.zeros(cat.n_verts, bool)
    expect[voff[1]:] = inside_lower[voff[1]:]
    expect[:voff[1]] = inside_upper[:voff[1]]
    assert expect.sum() == 9 + 4
    assert np.array_equal(contact >= 0, expect)
    for a in np.nonzero(expect)[0]:
        t = tris[contact[a]]
        n = np.cross(x[t[1]] - x[t[0]], x[t[2]] - x[t[0]])
        n /= np.linalg.norm(n)
        if a >= voff[1]:  # under the lower box's top face (normal +z)
            assert np.allclose(x[t, 2], 0.1) and n[2] == pytest.approx(1.0)
        else:  # above the upper box's bottom face (normal -z)
            assert np.allclose(x[t, 2], 0.09) and n[2] == pytest.approx(-1.0)
        q, w = orc.closest_point_tri(x[a], *x[t])
        assert (q - x[a]) @ n == pytest.approx(0.01, abs=1e-12)
    rim = [a for a in range(voff[1]) if abs(x[a, 2] - 0.1) < 1e-12 and not inside_upper[a]
           and np.linalg.norm(np.maximum(np.maximum(ulo - x[a], x[a] - uhi), 0)) < p.dcd_radius]
    assert len(rim) >= 4 and np.all(contact[rim] < 0)
    # a single body at rest, and two separated bodies, have no pairs
    single = synth.beam(4, 3, 2, jitter_frac=0.1, seed=103, pin_face=None)
    assert (orc.Model.from_mesh(single).dcd(p, single.rest) < 0).all()
    cat2, _ = _two_blocks(0.02)
    assert (orc.Model.from_mesh(cat2).dcd(p, cat2.rest) < 0).all()


def test_contact_forces_are_the_gradient_and_balance(orc):
    """For a projection inside its triangle, d is the distance from the
    vertex to the triangle's plane.  Moving the vertex along n changes d by
    minus the move; moving corner k along n lifts the plane under the
    projection by w_k times the move; in-plane moves leave d alone.  So the
    forces k_c d n and -k_c d w_k n are exactly -dE/dx of the total contact
    energy sum k_c d^2 / 2, and they sum to zero."""
    lower = synth.beam(3, 3, 1, edge=0.1, E=1e5, nu=0.4, pin_face="z-", jitter_frac=0.02, seed=105)
    upper = synth.beam(2, 2, 1, edge=0.1, E=1e5, nu=0.4, pin_face=None, jitter_frac=0.02, seed=106,
                       origin=(0.03, 0.02, 0.09))
    cat, voff, _ = synth.concat([lower, upper])
    model = orc.Model.from_mesh(cat)
    p = orc.Params.make(self_collision=True, dcd_radius=0.05, k_c=1e5)
    contact = model.dcd(p, cat.rest)
    tris = model.tris()
    pairs = np.nonzero(contact >= 0)[0]
    assert pairs.size >= 4
    x = cat.rest
    for a in pairs:
        _, w = orc.closest_point_tri(x[a], *x[tris[contact[a]]])
        assert w.min() > 1e-3  # interior projections only
    involved = sorted(set(pairs.tolist()) | set(tris[contact[pairs]].ravel().tolist()))
    y = x.copy()  # no inertia gradient
    el = model.elastic_grad(x).reshape(-1, 3)
    total = np.zeros(3)
    for v in involved:
        f, _, _ = model.self_contact(p, v, x)
        e = 1e-7
        g = np.zeros(3)
        for r in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, r] += e
            xm[v, r] -= e
            g[r] = (model.energy_G(p, H, xp, y) - model.energy_G(p, H, xm, y)) / (2 * e)
        g -= el[v]  # leaves the contact energy's gradient
        if model.free[v]:
            assert np.allclose(f, -g, rtol=1e-5, atol=1e-5 * np.abs(f).max())
        total += f
    assert np.abs(total).max() <= 1e-9 * max(1.0, np.abs(total).max())

    # Gauss-Newton Hessian of k_c d^2 / 2 is k_c grad d grad d^T = f f^T / (k_c d^2)
    # for a vertex in one pair; d is recomputed here from the plane geometry.
    n_pairs = {v: 0 for v in involved}
    depth = {}
    for a in pairs:
        t = tris[contact[a]]
        nrm = np.cross(x[t[1]] - x[t[0]], x[t[2]] - x[t[0]])
        nrm /= np.linalg.norm(nrm)
        d = -(x[a] - x[t[0]]) @ nrm
        for v in [a, *t]:
            n_pairs[v] += 1
            depth[v] = d
    single = [v for v in involved if n_pairs[v] == 1 and depth[v] > 0]
    assert len(single) >= 3
    for v in single:
        f, Hc, _ = model.self_contact(p, v, x)
        assert np.allclose(Hc, np.outer(f, f) / (p.k_c * depth[v] ** 2), rtol=1e-9, atol=1e-9 * np.abs(Hc).max())


@pytest.mark.parametrize("collide", [True, False])
def test_block_dropped_on_block(orc, collide):
    cat, voff = _two_blocks(0.002)
    model = orc.Model.from_mesh(cat)
    colors, nc = orc.color_greedy(cat.n_verts, cat.tets)
    p = orc.Params.make(gravity=(0, 0, -9.8), self_collision=collide, dcd_radius=0.05, k_c=1e5)
    v0 = np.zeros_like(cat.rest)
    v0[voff[1]:, 2] = -1.0
    x, _, _ = orc.run(model, p, colors, nc, H, 40, 20, cat.rest, v0)
    zmin_upper = x[voff[1]:, 2].min()
    if collide:
        assert zmin_upper > 0.1 - 0.01  # rests on the lower block (penalty depth ~ m g / k_c)
    else:
        assert zmin_upper < 0.0  # falls through


def test_dcd_tie_on_a_shared_edge_goes_to_the_lower_index(orc):
    """A vertex sunk 1 cm under the middle of a top-face diagonal of an
    unjittered box is equally near the two triangles sharing that diagonal;
    the pair takes the lower index of the two."""
    lower = synth.beam(3, 3, 1, edge=0.1, pin_face="z-")
    upper = synth.beam(1, 1, 1, edge=0.1, pin_face=None, origin=(0.05, 0.05, 0.09))
    cat, voff, _ = synth.concat([lower, upper])
    model = orc.Model.from_mesh(cat)
    p = orc.Params.make(self_collision=True, dcd_radius=0.05, k_c=1e5)
    x = cat.rest
    contact = model.dcd(p, x)
    tris = model.tris()
    a = voff[1]  # the upper block's corner at (0.05, 0.05, 0.09)
    assert np.allclose(x[a], [0.05, 0.05, 0.09])
    tied = [T for T, t in enumerate(tris)
            if np.allclose(x[t, 2], 0.1) and any(np.allclose(x[k, :2], [0, 0]) for k in t)
            and any(np.allclose(x[k, :2], [0.1, 0.1]) for k in t)]
    assert len(tied) == 2
    assert contact[a] == min(tied)


def _f0(u, eh):
    """Antiderivative of f1 (Eq. 15) with f0(0) = 0."""
    return np.where(u < eh, u * u / eh - u ** 3 / (3 * eh * eh), u - eh / 3)


def test_self_contact_friction_is_gradient_of_lagged_potential(orc):
    """Friction of the self-contact pairs (Sec. 3.6 applied to vertex-triangle
    pairs) equals minus the gradient of sum_pairs mu_c lambda f0(|u|), with
    lambda = k_c d, the normal and the barycentric weights held at their
    current values (lagged), u the tangential part of
    (x_a - x_a^t) - sum_k w_k (x_k - x_k^t); the forces sum to zero."""
    lower = synth.beam(3, 3, 1, edge=0.1, E=1e5, nu=0.4, pin_face="z-", jitter_frac=0.02, seed=105)
    upper = synth.beam(2, 2, 1, edge=0.1, E=1e5, nu=0.4, pin_face=None, jitter_frac=0.02, seed=106,
                       origin=(0.03, 0.02, 0.09))
    cat, voff, _ = synth.concat([lower, upper])
    model = orc.Model.from_mesh(cat)
    pf = orc.Params.make(self_collision=True, dcd_radius=0.05, k_c=1e5, mu_c=0.4, eps_v=0.05)
    p0 = orc.Params.make(self_collision=True, dcd_radius=0.05, k_c=1e5)
    x = cat.rest
    contact = model.dcd(pf, x)
    tris = model.tris()
    pairs = np.nonzero(contact >= 0)[0]
    rng = np.random.default_rng(107)
    xt = x - rng.normal(0.0, 4e-4, x.shape)  # tangential motion both below and above eps_v h
    eh = pf.eps_v * H
    geo = {}
    for a in pairs:
        t = tris[contact[a]]
        q, w = orc.closest_point_tri(x[a], *x[t])
        n = np.cross(x[t[1]] - x[t[0]], x[t[2]] - x[t[0]])
        n /= np.linalg.norm(n)
        d = (q - x[a]) @ n
        if d > 0:
            geo[a] = (t, w, n, pf.k_c * d)
    mags = []

    def potential(z):
        tot = 0.0
        for a, (t, w, n, lam) in geo.items():
            dl = (z[a] - xt[a]) - sum(w[k] * (z[t[k]] - xt[t[k]]) for k in range(3))
            u = dl - (dl @ n) * n
            tot += pf.mu_c * lam * _f0(np.linalg.norm(u), eh)
        return tot

    for a, (t, w, n, lam) in geo.items():
        dl = (x[a] - xt[a]) - sum(w[k] * (x[t[k]] - xt[t[k]]) for k in range(3))
        mags.append(np.linalg.norm(dl - (dl @ n) * n))
    assert min(mags) < eh < max(mags)  # both friction regimes are exercised
    involved = sorted(set(geo) | set(np.concatenate([g[0] for g in geo.values()]).tolist()))
    total = np.zeros(3)
    fmax = 0.0
    for v in involved:
        ff = model.self_contact(pf, v, x, H, xt)[0] - model.self_contact(p0, v, x)[0]
        fmax = max(fmax, float(np.abs(ff).max()))
        e = 1e-9
        g = np.zeros(3)
        for r in range(3):
            zp, zm = x.copy(), x.copy()
            zp[v, r] += e
            zm[v, r] -= e
            g[r] = (potential(zp) - potential(zm)) / (2 * e)
        assert np.allclose(ff, -g, rtol=1e-5, atol=1e-6 * max(1e-12, np.abs(ff).max()))
        total += ff
    assert fmax > 0 and np.abs(total).max() <= 1e-12 * max(1.0, fmax)


def test_block_sliding_on_a_rigid_block_decelerates_at_mu_g(orc):
    """Coulomb regime on a self-contact: a free block sliding at 2 m/s on a
    fully pinned block carries its weight through vertex-triangle pairs, so
    its mean velocity falls by mu g per unit time."""
    mu = 0.3
    lower = synth.beam(6, 3, 1, edge=0.1, E=1e6, nu=0.3, pin_face="z-")
    lower.pinned[:] = 1
    upper = synth.beam(2, 2, 1, edge=0.1, E=1e6, nu=0.3, pin_face=None, origin=(0.03, 0.04, 0.1 - 5e-5))
    cat, voff, _ = synth.concat([lower, upper])
    model = orc.Model.from_mesh(cat)
    colors, nc = orc.color_greedy(cat.n_verts, cat.tets)
    p = orc.Params.make(gravity=(0, 0, -9.8), k_c=1e6, self_collision=True, dcd_radius=0.05, mu_c=mu, eps_v=1e-3)
    x = cat.rest.copy()
    v = np.zeros_like(x)
    v[voff[1]:, 0] = 2.0
    vp = v.copy()
    vs = []
    for _ in range(13):
        model.step(p, colors, nc, H, 500, x, v, vp)
        vs.append(v[voff[1]:, 0].mean())
    decel = (vs[3] - vs[12]) / (9 * H)
    assert decel == pytest.approx(mu * 9.8, rel=0.02)
    p_nf = orc.Params.make(gravity=(0, 0, -9.8), k_c=1e6, self_collision=True, dcd_radius=0.05)
    x = cat.rest.copy()
    v = np.zeros_like(x)
    v[voff[1]:, 0] = 2.0
    vp = v.copy()
    for _ in range(4):
        model.step(p_nf, colors, nc, H, 500, x, v, vp)
    assert abs(v[voff[1]:, 0].mean() - 2.0) < 0.02  # without friction it keeps sliding
