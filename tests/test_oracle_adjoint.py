"""Pins of the oracle's dense adjoint of converged implicit-Euler steps.

The paper has no adjoint; the reverse recursion follows from the implicit
function theorem applied to dG/dx = 0 of Eq. 2 with y from Eq. 3 and the
velocity update of Eq. 6.  It is checked here against central finite
differences of a forward solved to convergence by dense Newton, and against
the closed form of a body without stiffness.  CPU only."""
import numpy as np
import pytest

from paper_2403_06321_b300 import synth

H = 1.0 / 60.0


def _converged_forward(orc, model, p, x0, v0, steps, log_young=None):
    if log_young is not None:
        model.set_log_young(log_young)
    x = np.array(x0, float)
    v = np.array(v0, float)
    xs = [x.copy()]
    for _ in range(steps):
        y = model.inertia_target(p, H, x, v)
        xn = model.newton_solve(p, H, x + H * v, y, tol=1e-14, max_iter=60)
        v = (xn - x) / H
        x = xn
        xs.append(x.copy())
    return xs


def _loss(x, tip, target):
    d = x[tip] - target
    return float((d * d).sum(axis=1).mean())


def _dloss(x, tip, target):
    g = np.zeros_like(x)
    g[tip] = 2.0 / len(tip) * (x[tip] - target)
    return g


@pytest.mark.slow
def test_dense_adjoint_matches_central_fd(orc):
    m = synth.beam(3, 1, 1, E=1e5, nu=0.4, jitter_frac=0.05, seed=21)
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(gravity=(0, 0, -9.8))
    tip = np.nonzero(m.grid_ijk[:, 0] == 3)[0]
    target = m.rest[tip] + np.array([0.03, -0.02, 0.05])
    steps = 3
    logE = np.log(m.young.astype(float))
    rng = np.random.default_rng(4)
    v0 = rng.normal(0, 0.2, m.rest.shape) * (1 - m.pinned[:, None])
    xs = _converged_forward(orc, model, p, m.rest, v0, steps, logE)
    gE, gv, _ = orc.dense_adjoint(model, p, H, xs, _dloss(xs[-1], tip, target))

    def L(le, vv):
        return _loss(_converged_forward(orc, model, p, m.rest, vv, steps, le)[-1], tip, target)

    # eps = 1e-4: smaller steps are limited by the forward's ~1e-11 residual;
    # errors are measured relative to the largest gradient entry
    eps = 1e-4
    for j in [0, 5, 11, 17]:
        e = np.zeros_like(logE); e[j] = eps
        fd = (L(logE + e, v0) - L(logE - e, v0)) / (2 * eps)
        assert abs(gE[j] - fd) <= 1e-6 * np.abs(gE).max()
    free = np.nonzero(m.pinned == 0)[0]
    for i in free[[0, 3, 7, -1]]:
        for r in range(3):
            dv = np.zeros_like(v0); dv[i, r] = eps
            fd = (L(logE, v0 + dv) - L(logE, v0 - dv)) / (2 * eps)
            assert abs(gv[i, r] - fd) <= 1e-6 * np.abs(gv).max()
    assert np.all(gv[m.pinned == 1] == 0)


def test_dense_adjoint_without_stiffness_is_free_fall(orc):
    """E -> 0: each vertex falls freely, x_T = x_0 + T h v_0 + const, so
    dL/dv_0 = T h dL/dx_T (tip vertices only, zero elsewhere)."""
    m = synth.beam(2, 1, 1, E=1e-9, nu=0.3, pin_face=None)
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(gravity=(0, 0, -9.8))
    tip = np.nonzero(m.grid_ijk[:, 0] == 2)[0]
    target = m.rest[tip] + 0.1
    steps = 4
    v0 = np.zeros_like(m.rest)
    xs = _converged_forward(orc, model, p, m.rest, v0, steps)
    dLdx = _dloss(xs[-1], tip, target)
    gE, gv, gx = orc.dense_adjoint(model, p, H, xs, dLdx)
    assert np.allclose(gv, steps * H * dLdx, rtol=1e-8, atol=1e-12)
    assert np.allclose(gx, dLdx, rtol=1e-8, atol=1e-12)
    assert np.abs(gE).max() < 1e-9


def test_sparse_and_dense_adjoint_agree(orc):
    m = synth.beam(4, 2, 1, E=1e5, nu=0.4, jitter_frac=0.05, seed=22)
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(gravity=(0, 0, -9.8), ground_on=True, ground_height=-0.001, k_c=1e5)
    tip = np.nonzero(m.grid_ijk[:, 0] == 4)[0]
    target = m.rest[tip] + 0.05
    xs = _converged_forward(orc, model, p, m.rest, np.zeros_like(m.rest), 3)
    g = _dloss(xs[-1], tip, target)
    d = orc.dense_adjoint(model, p, H, xs, g, sparse=False)
    s = orc.dense_adjoint(model, p, H, xs, g, sparse=True)
    for a, b in zip(d, s):
        assert np.allclose(a, b, rtol=1e-9, atol=1e-12 * np.abs(a).max())


@pytest.mark.slow
def test_dense_adjoint_with_subspace_constraints_matches_central_fd(orc):
    """Beam whose far face slides in a tilted plane and one of whose top
    vertices moves along a line (Sec. 3.4): gradients with respect to log E,
    v_0 and x_0 (across a constrained vertex's plane, which moves its
    subspace) against central differences of the converged forward."""
    m = synth.beam(3, 1, 1, E=1e5, nu=0.4, jitter_frac=0.05, seed=23)
    m.sub_dim = np.full(m.n_verts, 3, np.int32)
    m.sub_dir = np.zeros((m.n_verts, 3))
    far = np.nonzero(m.grid_ijk[:, 0] == 3)[0]
    m.sub_dim[far] = 2
    m.sub_dir[far] = (1.0, 0.2, -0.3)
    line = np.nonzero((m.grid_ijk[:, 0] == 2) & (m.grid_ijk[:, 2] == 1))[0]
    m.sub_dim[line] = 1
    m.sub_dir[line] = (0.3, 0.5, -0.8)
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(gravity=(1.0, 0, -9.8))
    tip = np.nonzero(m.grid_ijk[:, 0] >= 2)[0]
    target = m.rest[tip] + np.array([0.03, -0.02, 0.05])
    steps = 3
    logE = np.log(m.young.astype(float))
    rng = np.random.default_rng(5)
    Bm = model.reduced_basis()
    v0 = (Bm @ (Bm.T @ rng.normal(0, 0.2, 3 * m.n_verts))).reshape(-1, 3)  # admissible
    xs = _converged_forward(orc, model, p, m.rest, v0, steps, logE)
    gE, gv, gx = orc.dense_adjoint(model, p, H, xs, _dloss(xs[-1], tip, target))

    def L(le, vv, x0=m.rest):
        return _loss(_converged_forward(orc, model, p, x0, vv, steps, le)[-1], tip, target)

    # eps = 2e-3 with a 2e-4 tolerance: the converged forward carries noise
    # of about 2e-11 in the loss, which at smaller steps dominates the quotient
    # (the adjoint matches the quotients to 7 digits where the noise is small)
    eps = 2e-3
    for j in [0, 7, 13, 17]:
        e = np.zeros_like(logE); e[j] = eps
        fd = (L(logE + e, v0) - L(logE - e, v0)) / (2 * eps)
        assert abs(gE[j] - fd) <= 2e-4 * np.abs(gE).max()
    for i in (far[0], line[0], np.nonzero((m.sub_dim == 3) & (m.pinned == 0))[0][0]):
        Q = Bm[3 * i:3 * i + 3][:, np.abs(Bm[3 * i:3 * i + 3]).sum(0) > 0]
        for c in range(Q.shape[1]):  # admissible directions only
            dv = np.zeros_like(v0); dv[i] = eps * Q[:, c]
            fd = (L(logE, v0 + dv) - L(logE, v0 - dv)) / (2 * eps)
            assert abs(gv[i] @ Q[:, c] - fd) <= 2e-4 * np.abs(gv).max()
    n = m.sub_dir[far[0]] / np.linalg.norm(m.sub_dir[far[0]])
    dx = np.zeros_like(m.rest); dx[far[0]] = eps * n  # moves the plane the vertex is held in
    fd = (L(logE, v0, m.rest + dx) - L(logE, v0, m.rest - dx)) / (2 * eps)
    assert abs(gx[far[0]] @ n - fd) <= 2e-4 * np.abs(gx).max()
    assert abs(fd) > 1e-3 * np.abs(gx).max()  # the anchor matters
