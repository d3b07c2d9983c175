"""The stored oracle outputs under tests/golden/ (written by
tests/golden/make_golden.py from oracle/ only): the oracle must still
produce them, so that a change to its arithmetic shows up here and is made
on purpose.  Each fixture is also checked against what does not come from
the oracle: the element's rest data against numpy's inverse and determinant
of the rest edges, its gradient and Hessian blocks against central finite
differences of the stored energy, the Chebyshev ratios against Eq. 19
evaluated here and its closed-form limit, and the beam's pinned face."""
import os

import numpy as np
import pytest

from paper_2403_06321_b300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read(name):
    rows = {}
    multi = []
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            key, *vals = ln.split()
            if key in ("omega", "x"):
                multi.append([float(v) for v in vals])
            else:
                rows[key] = np.array([float(v) for v in vals])
    return rows, np.array(multi)


def test_element_fixture(orc):
    g, _ = _read("element_tet.txt")
    rest, x = g["rest"].reshape(4, 3), g["deformed"].reshape(4, 3)
    E, nu = g["E_nu"]
    mu, lam = orc.lame(E, nu)
    B, V = orc.rest_tet(rest)
    assert np.allclose([mu, lam], g["mu_lam"], rtol=1e-15, atol=0)
    assert np.allclose(B.reshape(-1), g["B"], rtol=1e-13, atol=0)
    assert abs(V - g["V"][0]) <= 1e-15 * V
    xf = x.reshape(-1)
    assert abs(orc.tet_energy(xf, B, V, mu, lam) - g["energy"][0]) <= 1e-13 * abs(g["energy"][0])
    assert np.allclose(orc.tet_grad(xf, B, V, mu, lam).reshape(-1), g["grad"], rtol=1e-12, atol=1e-12)
    assert np.allclose(orc.tet_hess_block(xf, B, V, mu, lam, 0, 0).reshape(-1), g["hess_00"], rtol=1e-12)
    assert np.allclose(orc.tet_hess_block(xf, B, V, mu, lam, 0, 1).reshape(-1), g["hess_01"], rtol=1e-12)
    # rest data by numpy: B = Dm^-1, V = |det Dm| / 6 (Dm = rest edges as columns)
    Dm = (rest[1:] - rest[0]).T
    assert np.allclose(g["B"].reshape(3, 3), np.linalg.inv(Dm), rtol=1e-12)
    assert abs(g["V"][0] - abs(np.linalg.det(Dm)) / 6) <= 1e-13 * g["V"][0]
    # the Lame pair of the stated reading: mu = E/(2(1+nu)), lam = E nu/((1+nu)(1-2nu)) + mu
    mu_r = E / (2 * (1 + nu))
    assert np.allclose(g["mu_lam"], [mu_r, E * nu / ((1 + nu) * (1 - 2 * nu)) + mu_r], rtol=1e-14)
    # stored gradient = central differences of the stored energy function;
    # stored Hessian blocks = central differences of the gradient
    step = 1e-7
    fd = np.zeros(12)
    for k in range(12):
        xp, xm = xf.copy(), xf.copy()
        xp[k] += step
        xm[k] -= step
        fd[k] = (orc.tet_energy(xp, B, V, mu, lam) - orc.tet_energy(xm, B, V, mu, lam)) / (2 * step)
    assert np.abs(fd - g["grad"]).max() <= 1e-6 * np.abs(g["grad"]).max()
    for blk, col in (("hess_00", 0), ("hess_01", 1)):
        H = np.zeros((3, 3))
        for b in range(3):
            xp, xm = xf.copy(), xf.copy()
            xp[3 * col + b] += step
            xm[3 * col + b] -= step
            H[:, b] = (orc.tet_grad(xp, B, V, mu, lam)[0] - orc.tet_grad(xm, B, V, mu, lam)[0]) / (2 * step)
        assert np.abs(H.reshape(-1) - g[blk]).max() <= 1e-5 * np.abs(g[blk]).max(), blk
    # the forces on a free tet balance: the four gradients add up to zero
    assert np.abs(g["grad"].reshape(4, 3).sum(0)).max() <= 1e-12 * np.abs(g["grad"]).max()


def test_chebyshev_fixture(orc):
    g, om = _read("chebyshev_omega.txt")
    rho = g["rho"][0]
    w = 0.0
    for n, stored in om:
        w = orc.cheby_omega(int(n), rho, w)
        assert w == stored
    # Eq. 19 evaluated here, and its limit 2 / (1 + sqrt(1 - rho^2))
    ref = [1.0, 2.0 / (2.0 - rho * rho)]
    while len(ref) < len(om):
        ref.append(4.0 / (4.0 - rho * rho * ref[-1]))
    assert np.allclose(om[:, 1], ref, rtol=1e-15, atol=0)
    assert abs(om[-1, 1] - 2.0 / (1.0 + np.sqrt(1.0 - rho * rho))) <= 1e-7


def test_cantilever_fixture(orc):
    g, rows = _read("cantilever_10_steps.txt")
    steps = int(g["steps"][0])
    m, cfg = synth.cantilever_beam()
    colors = synth.kuhn_coloring(m.grid_ijk)
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(gravity=cfg.gravity, init_mode=cfg.init_mode, det_eps=cfg.det_eps)
    x, v, _ = orc.run(model, p, colors, int(colors.max()) + 1, cfg.h, cfg.iters, steps, m.rest,
                      np.zeros_like(m.rest))
    assert rows.shape == (m.n_verts, 7)
    assert np.array_equal(rows[:, 0].astype(int), np.arange(m.n_verts))
    xs, vs = rows[:, 1:4], rows[:, 4:7]
    diag = float(np.linalg.norm(m.rest.max(0) - m.rest.min(0)))
    assert np.abs(x - xs).max() <= 1e-12 * diag
    assert np.abs(v - vs).max() <= 1e-12 * diag / cfg.h
    pinned = m.pinned == 1
    assert pinned.any() and np.array_equal(xs[pinned], m.rest[pinned]) and not vs[pinned].any()
    # the free end has fallen: the beam sags under gravity
    assert xs[~pinned, 2].min() < m.rest[:, 2].min() - 0.01


@pytest.mark.parametrize("name", ["element_tet.txt", "chebyshev_omega.txt", "cantilever_10_steps.txt"])
def test_fixture_headers_cite_and_name_the_writer(name):
    with open(os.path.join(GOLDEN, name)) as f:
        head = "".join(ln for ln in f if ln.startswith("#"))
    assert "make_golden.py" in head and "oracle/" in head
    assert "Eq." in head
