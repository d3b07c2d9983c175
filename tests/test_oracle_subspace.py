"""Pins of the oracle's subspace constraints (Sec. 3.4, bilateral): a vertex
restricted to x^t + span(Q), Q an orthonormal 3 x L basis (L = 1 a line,
L = 2 a plane), takes the L x L Newton step Q^T H Q dz = Q^T f.  CPU only."""
import numpy as np
import pytest
from scipy.optimize import minimize, minimize_scalar

from paper_2403_06321_b300 import synth

H = 1.0 / 60.0


def _one_tet(orc, L, direction):
    """A tet with three pinned corners and a free apex restricted to a line or
    plane through its rest position."""
    m = synth.MeshInput(rest=np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0], [0.03, 0.02, 0.08]], float),
                        tets=np.array([[0, 1, 2, 3]], np.int32), young=np.array([1e4], np.float32),
                        poisson=np.array([0.4], np.float32), density=np.array([1000.0], np.float32),
                        pinned=np.array([1, 1, 1, 0], np.uint8))
    model = orc.Model.from_mesh(m)
    model.set_subspace(3, L, direction)
    return m, model


def test_line_constrained_apex_minimises_G_along_its_line(orc):
    """The converged step is the minimiser of G(x^t + t e) over t, found by a
    scalar search on the global energy (Eq. 2)."""
    e = np.array([0.3, -0.5, -0.8])
    m, model = _one_tet(orc, 1, e)
    p = orc.Params.make(gravity=(1.0, -2.0, -9.8))
    xt = m.rest.copy()
    v = np.zeros_like(xt)
    x, _, _ = orc.run(model, p, np.array([0, 1, 2, 3], np.int32), 4, H, 200, 1, xt, v)
    eh = e / np.linalg.norm(e)
    y = model.inertia_target(p, H, xt, v)

    def G(t):
        z = xt.copy()
        z[3] = xt[3] + t * eh
        return model.energy_G(p, H, z, y)

    t = minimize_scalar(G, bracket=(-0.01, 0.01), tol=1e-12).x
    d = x[3] - xt[3]
    assert np.linalg.norm(d - (d @ eh) * eh) <= 1e-15  # on the line
    assert d @ eh == pytest.approx(t, abs=1e-9)
    assert abs(t) > 1e-4


def test_plane_constrained_apex_minimises_G_in_its_plane(orc):
    n = np.array([0.2, 0.9, -0.4])
    m, model = _one_tet(orc, 2, n)
    p = orc.Params.make(gravity=(1.0, -2.0, -9.8))
    xt = m.rest.copy()
    v = np.zeros_like(xt)
    x, _, _ = orc.run(model, p, np.array([0, 1, 2, 3], np.int32), 4, H, 200, 1, xt, v)
    nh = n / np.linalg.norm(n)
    Q = np.linalg.svd(nh[None, :])[2][1:].T  # an in-plane basis of its own
    y = model.inertia_target(p, H, xt, v)

    def G(z):
        w = xt.copy()
        w[3] = xt[3] + Q @ z
        return model.energy_G(p, H, w, y)

    z = minimize(G, np.zeros(2), method="BFGS", options=dict(gtol=1e-12)).x
    d = x[3] - xt[3]
    assert abs(d @ nh) <= 1e-15
    assert np.abs(d - Q @ z).max() <= 1e-8
    assert np.linalg.norm(d) > 1e-4


def _rollers(orc, seed=81):
    """Beam pinned at x = 0 whose far face slides in its plane (a roller
    support) and whose top edge line y = 0, z = top moves along a tilted
    line, jittered so that nothing is symmetric."""
    m = synth.beam(4, 2, 2, edge=0.05, E=1e5, nu=0.4, jitter_frac=0.1, seed=seed)
    ijk = m.grid_ijk
    m.sub_dim = np.full(m.n_verts, 3, np.int32)
    m.sub_dir = np.zeros((m.n_verts, 3))
    far = ijk[:, 0] == 4
    m.sub_dim[far] = 2
    m.sub_dir[far] = (1.0, 0.1, -0.2)
    edge = (ijk[:, 1] == 0) & (ijk[:, 2] == 2) & (ijk[:, 0] > 0) & (ijk[:, 0] < 4)
    m.sub_dim[edge] = 1
    m.sub_dir[edge] = (0.6, 0.3, -0.74)
    return m


def test_rollers_converge_to_the_reduced_dense_newton(orc):
    """Many VBD iterations on a beam with plane- and line-constrained
    vertices reach the dense Newton minimiser of Eq. 2 over the admissible
    displacements (basis from an SVD, not the solver's)."""
    m = _rollers(orc)
    model = orc.Model.from_mesh(m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    p = orc.Params.make(gravity=(0, 0, -9.8))
    xt = m.rest.copy()
    v = np.zeros_like(xt)
    x_vbd, _, _ = orc.run(model, p, colors, nc, H, 3000, 1, xt, v)
    y = model.inertia_target(p, H, xt, v)
    x_nt = model.newton_solve(p, H, xt, y)
    assert np.abs(x_vbd - x_nt).max() <= 1e-9
    far = m.sub_dim == 2
    assert np.abs(x_nt[far] - xt[far]).max() > 1e-5  # the rollers do move
    m0 = synth.beam(4, 2, 2, edge=0.05, E=1e5, nu=0.4, jitter_frac=0.1, seed=81)
    x_unc = orc.Model.from_mesh(m0).newton_solve(p, H, xt, y)
    assert np.abs(x_unc - x_nt).max() > 1e-4  # and the constraints change the answer


@pytest.mark.parametrize("init_mode", [0, 1, 2, 3])
def test_constrained_vertices_stay_on_their_subspaces(orc, init_mode):
    """Over many steps with Chebyshev, the ground and every initial guess,
    each constrained vertex stays on its rest line or plane."""
    m = _rollers(orc, seed=82)
    m.rest[:, 2] += 0.01
    model = orc.Model.from_mesh(m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    p = orc.Params.make(gravity=(2.0, -1.0, -9.8), init_mode=init_mode, cheby_rho=0.7, ground_on=True,
                        k_c=1e5, ground_height=0.005)
    x = m.rest.copy()
    v = np.zeros_like(x)
    vp = v.copy()
    for _ in range(15):
        model.step(p, colors, nc, H, 12, x, v, vp)
        d = x - m.rest
        for i in np.nonzero(m.sub_dim < 3)[0]:
            e = m.sub_dir[i] / np.linalg.norm(m.sub_dir[i])
            if m.sub_dim[i] == 2:
                assert abs(d[i] @ e) <= 1e-14
            else:
                assert np.linalg.norm(d[i] - (d[i] @ e) * e) <= 1e-14
    assert np.abs(x - m.rest).max() > 1e-3


def test_direction_sign_does_not_matter(orc):
    m = _rollers(orc, seed=83)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    p = orc.Params.make(gravity=(0, 0, -9.8))
    out = []
    for sgn in (1.0, -1.0):
        mm = _rollers(orc, seed=83)
        mm.sub_dir = sgn * m.sub_dir
        x, _, _ = orc.run(orc.Model.from_mesh(mm), p, colors, nc, H, 20, 3, m.rest, np.zeros_like(m.rest))
        out.append(x)
    assert np.abs(out[0] - out[1]).max() <= 1e-14


def test_bad_subspace_arguments_are_refused(orc):
    _, model = _one_tet(orc, 1, (1, 0, 0))
    for i, L, d in ((7, 1, (1, 0, 0)), (3, 0, (1, 0, 0)), (3, 4, (1, 0, 0)), (3, 2, (0, 0, 0))):
        with pytest.raises(ValueError):
            model.set_subspace(i, L, d)
    model.set_subspace(3, 3, (0, 0, 0))  # lifting needs no direction


@pytest.mark.parametrize("L,direction", [(1, (0.3, -0.5, -0.8)), (2, (0.2, 0.9, -0.4))])
def test_one_local_step_is_the_reduced_newton_step(orc, L, direction):
    """A single iteration moves the constrained apex by -Q (Q^T H Q)^-1 Q^T g
    with g, H the gradient and Hessian of Eq. 2 at the start (dense global
    assembly) and Q an in-subspace basis of its own."""
    m, model = _one_tet(orc, L, direction)
    p = orc.Params.make(gravity=(1.0, -2.0, -9.8))
    xt = m.rest.copy()
    v = np.zeros_like(xt)
    y = model.inertia_target(p, H, xt, v)
    g, Hs = model.global_grad_hess(p, H, xt, y)
    d = np.asarray(direction, float) / np.linalg.norm(direction)
    Q = d[:, None] if L == 1 else np.linalg.svd(d[None, :])[2][1:].T
    gi, Hi = g[9:12], Hs[9:12, 9:12]
    step = -Q @ np.linalg.solve(Q.T @ Hi @ Q, Q.T @ gi)
    x, _, _ = orc.run(model, p, np.array([0, 1, 2, 3], np.int32), 4, H, 1, 1, xt, v)
    assert np.abs((x[3] - xt[3]) - step).max() <= 1e-12 * np.linalg.norm(step)
