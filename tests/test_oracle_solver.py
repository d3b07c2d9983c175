"""Pins of the oracle's time step (Algorithm 1): inertia target (Eq. 3),
initialisation (Sec. 3.7, Eq. 17), local solve (Eqs. 7-9), Gauss-Seidel
colour passes (Sec. 3.1, 3.9), Chebyshev acceleration (Eqs. 18-19), ground
penalty (Eq. 12) and the velocity update (Eq. 6).  CPU only."""
import numpy as np
import pytest

from paper_2403_06321_b300 import synth

H = 1.0 / 60.0


def _model(orc, m):
    return orc.Model.from_mesh(m)


def test_colouring_greedy_valid_and_kuhn_closed_form(orc):
    for dims in [(10, 3, 3), (4, 4, 4), (7, 2, 5)]:
        m = synth.beam(*dims)
        c, nc = orc.color_greedy(m.n_verts, m.tets)
        assert orc.color_valid(m.n_verts, m.tets, c)
        assert nc >= 4  # every tet is a 4-clique
        kc = synth.kuhn_coloring(m.grid_ijk)
        assert orc.color_valid(m.n_verts, m.tets, kc) and kc.max() == 3
    bad = synth.kuhn_coloring(m.grid_ijk).copy()
    t0 = m.tets[0]
    bad[t0[1]] = bad[t0[0]]
    assert not orc.color_valid(m.n_verts, m.tets, bad)


def test_colouring_greedy_is_deterministic_largest_degree_first(orc):
    # a single tet: all degrees equal -> visit order by id -> colours 0,1,2,3
    c, nc = orc.color_greedy(4, np.array([[0, 1, 2, 3]], np.int32))
    assert nc == 4 and list(c) == [0, 1, 2, 3]
    # two tets sharing a face: vertices 1,2,3 (degree 4) coloured before 0 and 4
    c, nc = orc.color_greedy(5, np.array([[0, 1, 2, 3], [4, 1, 2, 3]], np.int32))
    assert list(c[[1, 2, 3]]) == [0, 1, 2] and c[0] == 3 and c[4] == 3 and nc == 4


def test_inertia_target_and_initialisation_cases(orc):
    m = synth.beam(1, 1, 1, pin_face=None)
    model = _model(orc, m)
    n = m.n_verts
    p = orc.Params.make(gravity=(0, 0, -9.8), init_mode=3)
    xt = m.rest.copy()
    v = np.tile([0.1, -0.2, 0.3], (n, 1))
    g = np.array([0, 0, -9.8])
    y = model.inertia_target(p, H, xt, v)
    assert np.allclose(y, xt + H * v + H * H * g, atol=1e-15)
    # adaptive factor: a^t.g_hat > |g| -> 1 ; < 0 -> 0 ; in between -> ratio
    for a_comp, expect in [(12.0, 1.0), (-3.0, 0.0), (4.9, 0.5), (9.8, 1.0), (0.0, 0.0)]:
        vprev = v - H * a_comp * (g / 9.8)  # a^t = (v - vprev)/h = a_comp * g_hat
        x0 = model.initial_guess(p, H, xt, v, vprev)
        assert np.allclose(x0, xt + H * v + H * H * expect * g, atol=1e-14), a_comp
    # a tangential acceleration does not count
    vprev = v - H * np.array([50.0, 0, 0])
    assert np.allclose(model.initial_guess(p, H, xt, v, vprev), xt + H * v, atol=1e-14)
    # options (a), (b), (c)
    for mode, expect in [(0, xt), (1, xt + H * v), (2, y)]:
        p2 = orc.Params.make(gravity=(0, 0, -9.8), init_mode=mode)
        assert np.allclose(model.initial_guess(p2, H, xt, v, v), expect, atol=1e-14)
    # zero gravity -> acceleration term 0
    p0 = orc.Params.make(gravity=(0, 0, 0), init_mode=3)
    assert np.allclose(model.initial_guess(p0, H, xt, v, v - 1.0), xt + H * v, atol=1e-14)


def test_single_free_vertex_solve_is_exact_minimiser(orc):
    """G restricted to one vertex is exactly quadratic (J is affine in each
    vertex), so one Newton step lands on the minimiser: G(x* + d) - G(x*)
    equals 1/2 d^T H d > 0 for every probe d, with H from finite differences."""
    m = synth.beam(2, 2, 2, pin_face=None, jitter_frac=0.1, seed=2)
    i = 13  # the interior vertex
    m.pinned[:] = 1
    m.pinned[i] = 0
    model = _model(orc, m)
    p = orc.Params.make(gravity=(0, 0, -9.8))
    rng = np.random.default_rng(0)
    x = m.rest + rng.uniform(-0.01, 0.01, m.rest.shape)
    y = x + rng.uniform(-0.01, 0.01, x.shape)
    dx, skipped, contact = model.vertex_solve(p, H, i, x, y, m.rest)
    assert skipped == 0 and contact == 0
    xs = x.copy(); xs[i] += dx
    G0 = model.energy_G(p, H, xs, y)
    e = 1e-4
    Hn = np.zeros((3, 3))
    for r in range(3):
        for s in range(3):
            def G(dr, ds):
                z = xs.copy(); z[i, r] += dr; z[i, s] += ds
                return model.energy_G(p, H, z, y)
            Hn[r, s] = (G(e, e) - G(e, -e) - G(-e, e) + G(-e, -e)) / (4 * e * e)
    for _ in range(5):
        d = rng.normal(size=3) * 1e-3
        z = xs.copy(); z[i] += d
        dG = model.energy_G(p, H, z, y) - G0
        assert dG > 0
        assert dG == pytest.approx(0.5 * d @ Hn @ d, rel=1e-5)
    # sweeping the vertex's colour again does not move it
    colors = np.zeros(m.n_verts, np.int32)
    x2 = xs.copy()
    model.sweep_color(p, H, colors, 0, x2, y, m.rest)
    assert np.allclose(x2, xs, atol=1e-14)


def test_rest_mesh_stays_fixed(orc):
    m = synth.beam(4, 2, 2, pin_face=None, jitter_frac=0.1, seed=5)
    model = _model(orc, m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    p = orc.Params.make(gravity=(0, 0, 0))
    x, v, _ = orc.run(model, p, colors, nc, H, 10, 5, m.rest, np.zeros_like(m.rest))
    assert np.abs(x - m.rest).max() <= 1e-12 * 0.4
    assert np.abs(v).max() <= 1e-10


@pytest.mark.parametrize("mode", [2, 3])
def test_free_fall_closed_form(orc, mode):
    """Undeformed body, uniform velocity, no pins or contact: x = y is the
    exact minimiser (zero elastic force), so x^{t+1} = x^t + h v^t + h^2 g and
    v^{t+1} = v^t + h g.  With adaptive init, v^{t-1} = v^t - h g gives
    a-tilde = 1, i.e. the same initial guess."""
    m = synth.beam(3, 2, 2, pin_face=None, jitter_frac=0.1, seed=6)
    model = _model(orc, m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    p = orc.Params.make(gravity=(0, 0, -9.8), init_mode=mode)
    g = np.array([0, 0, -9.8])
    v0 = np.tile([0.5, -0.25, 1.0], (m.n_verts, 1))
    steps = 6
    x, v, _ = orc.run(model, p, colors, nc, H, 3, steps, m.rest, v0, vprev0=v0 - H * g)
    T = steps * H
    assert np.allclose(v, v0 + T * g, atol=1e-10)
    # x_T = x_0 + sum_t h (v0 + t h g) + h^2 g = x0 + T v0 + h^2 g * steps(steps+1)/2
    assert np.allclose(x, m.rest + T * v0 + H * H * g * steps * (steps + 1) / 2, atol=1e-12)


def test_energy_non_increasing_per_colour_pass(orc):
    """Each vertex update is the exact minimiser of G_i and the drop of G_i
    equals the drop of G (Sec. 3.1), so G never increases (no contact, no
    acceleration, no damping)."""
    m = synth.beam(6, 2, 2, E=1e5, nu=0.45, jitter_frac=0.1, seed=7)
    model = _model(orc, m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    p = orc.Params.make(gravity=(0, 0, -9.8))
    rng = np.random.default_rng(1)
    xt = m.rest.copy()
    v = rng.normal(0, 0.5, m.rest.shape) * (1 - m.pinned[:, None])
    y = model.inertia_target(p, H, xt, v)
    x = model.initial_guess(p, H, xt, v, v)
    G = model.energy_G(p, H, x, y)
    for it in range(10):
        for c in range(nc):
            model.sweep_color(p, H, colors, c, x, y, xt)
            G1 = model.energy_G(p, H, x, y)
            assert G1 <= G + 1e-12 * abs(G)
            G = G1


def test_vbd_converges_to_dense_newton(orc):
    """Many VBD iterations reach the backward-Euler solution (Sec. 1 claim),
    computed independently by a dense global Newton solve."""
    m = synth.beam(3, 1, 1, E=1e5, nu=0.4, jitter_frac=0.1, seed=8)
    model = _model(orc, m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    p = orc.Params.make(gravity=(0, 0, -9.8))
    xt = m.rest.copy()
    v = np.zeros_like(xt)
    x_vbd, v_vbd, _ = orc.run(model, p, colors, nc, H, 3000, 1, xt, v)
    y = model.inertia_target(p, H, xt, v)
    x_nt = model.newton_solve(p, H, xt, y)
    bbox = np.linalg.norm(m.rest.max(0) - m.rest.min(0))
    assert np.abs(x_vbd - x_nt).max() <= 1e-9 * bbox
    assert np.abs(x_nt - xt).max() > 1e-4  # the solution is not trivial


def test_ground_contact_converges_to_dense_newton(orc):
    m = synth.beam(2, 1, 1, E=1e5, nu=0.4, pin_face=None, origin=(0, 0, -0.02))
    model = _model(orc, m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    p = orc.Params.make(gravity=(0, 0, -9.8), ground_on=True, k_c=1e5)
    xt = m.rest.copy()
    v = np.zeros_like(xt)
    x_vbd, _, _ = orc.run(model, p, colors, nc, H, 4000, 1, xt, v)
    y = model.inertia_target(p, H, xt, v)
    x_nt = model.newton_solve(p, H, xt, y)
    assert np.abs(x_vbd - x_nt).max() <= 1e-9
    assert (x_nt[:, 2] < 0).any()  # penalty contact leaves some penetration


def test_chebyshev_omega_recurrence():
    from oracle import oracle as orc
    rho = 0.95
    w = [orc.cheby_omega(1, rho, 0.0)]
    for n in range(2, 200):
        w.append(orc.cheby_omega(n, rho, w[-1]))
    assert w[0] == 1.0
    assert w[1] == pytest.approx(2 / (2 - rho * rho), rel=1e-15)
    assert w[2] == pytest.approx(4 / (4 - rho * rho * w[1]), rel=1e-15)
    # fixed point of w = 4/(4 - rho^2 w): 2/(1 + sqrt(1 - rho^2)) = 1.52399...
    assert w[-1] == pytest.approx(2 / (1 + np.sqrt(1 - rho * rho)), rel=1e-10)
    # from n = 2 on, omega decreases monotonically to that limit
    assert np.all(np.diff(w[1:]) <= 0) and min(w[1:]) >= 2 / (1 + np.sqrt(1 - rho * rho))


def test_chebyshev_reaches_same_fixed_point_faster(orc):
    m = synth.beam(4, 1, 1, E=1e5, nu=0.4, jitter_frac=0.1, seed=9)
    model = _model(orc, m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    xt = m.rest.copy()
    v = np.zeros_like(xt)
    p0 = orc.Params.make(gravity=(0, 0, -9.8))
    y = model.inertia_target(p0, H, xt, v)
    x_ref = model.newton_solve(p0, H, xt, y)
    errs = {}
    for rho in (0.0, 0.7):
        p = orc.Params.make(gravity=(0, 0, -9.8), cheby_rho=rho)
        x20, _, _ = orc.run(model, p, colors, nc, H, 20, 1, xt, v)
        x4k, _, _ = orc.run(model, p, colors, nc, H, 3000, 1, xt, v)
        assert np.abs(x4k - x_ref).max() <= 1e-9
        errs[rho] = np.abs(x20 - x_ref).max()
    assert errs[0.7] < errs[0.0]


def test_chebyshev_skips_colliding_vertices(orc):
    """A vertex in ground contact keeps its Gauss-Seidel position (Sec. 3.8):
    compare one accelerated step with a manual re-run of the passes."""
    m = synth.beam(2, 1, 1, pin_face=None, origin=(0, 0, -0.005))
    model = _model(orc, m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    rho = 0.9
    p = orc.Params.make(gravity=(0, 0, -9.8), ground_on=True, k_c=1e6, cheby_rho=rho)
    pg = orc.Params.make(gravity=(0, 0, -9.8), ground_on=True, k_c=1e6)
    xt = m.rest.copy()
    v = np.zeros_like(xt)
    iters = 4
    x, _, _ = orc.run(model, p, colors, nc, H, iters, 1, xt, v)
    # manual Algorithm 1 with Eq. 18 and the skip
    y = model.inertia_target(pg, H, xt, v)
    xm = model.initial_guess(pg, H, xt, v, v)
    coll = np.zeros(m.n_verts, np.uint8)
    p1, p2, w = xm.copy(), None, 1.0
    for n in range(1, iters + 1):
        for c in range(nc):
            model.sweep_color(pg, H, colors, c, xm, y, xt, coll)
        w = orc.cheby_omega(n, rho, w)
        xn = xm.copy()
        if n >= 2:
            acc = coll == 0
            xn[acc] = w * (xm[acc] - p2[acc]) + p2[acc]
        p2, p1 = p1, xn.copy()
        xm = xn
    assert coll.any() and not coll.all()
    assert np.allclose(x, xm, atol=1e-14)


def test_damped_solve_minimises_rayleigh_potential(orc):
    """With Eqs. 10-11 the local step minimises G_i + k_d/(2h) (x - x^t)^T H_el
    (x - x^t): H_el (the elastic Hessian block, constant in x_i) is measured
    here by finite differences of the energy and the gradient of that sum is
    checked to vanish at the updated position."""
    m = synth.beam(2, 2, 2, pin_face=None, jitter_frac=0.1, seed=3)
    i = 13
    m.pinned[:] = 1
    m.pinned[i] = 0
    model = orc.Model.from_mesh(m)
    kd = 0.05
    p0 = orc.Params.make(gravity=(0, 0, -9.8))
    pd = orc.Params.make(gravity=(0, 0, -9.8), k_d=kd)
    rng = np.random.default_rng(4)
    xt = m.rest + rng.uniform(-0.005, 0.005, m.rest.shape)
    x = xt + rng.uniform(-0.01, 0.01, xt.shape)
    y = x + rng.uniform(-0.01, 0.01, x.shape)
    dx, skipped, _ = model.vertex_solve(pd, H, i, x, y, xt)
    assert skipped == 0
    xs = x.copy(); xs[i] += dx
    mh = model.mass()[i] / H ** 2

    def Eel(z):  # elastic part of G_i: G minus the inertia of vertex i
        return model.energy_G(p0, H, z, y) - 0.5 * mh * np.sum((z[i] - y[i]) ** 2)

    e = 1e-4
    Hel = np.zeros((3, 3))
    for r in range(3):
        for s in range(3):
            def E2(dr, ds):
                z = xs.copy(); z[i, r] += dr; z[i, s] += ds
                return Eel(z)
            Hel[r, s] = (E2(e, e) - E2(e, -e) - E2(-e, e) + E2(-e, -e)) / (4 * e * e)

    def total(z):
        dz = z[i] - xt[i]
        return model.energy_G(p0, H, z, y) + kd / (2 * H) * dz @ Hel @ dz

    h = 1e-6
    grad = np.array([(total(xs + h * np.eye(m.n_verts * 3)[3 * i + r].reshape(-1, 3))
                      - total(xs - h * np.eye(m.n_verts * 3)[3 * i + r].reshape(-1, 3))) / (2 * h)
                     for r in range(3)])
    scale = np.abs(Hel @ dx).max() + mh * np.abs(dx).max()
    assert np.abs(grad).max() <= 1e-5 * scale
