"""Pins of the oracle's ground friction (Sec. 3.6, Eqs. 13-16) with the
normal force read as a non-negative magnitude.  CPU only."""
import numpy as np
import pytest

from paper_2403_06321_b300 import synth

H = 1.0 / 60.0


def _f0(u, eh):
    """Antiderivative of f1 (Eq. 15) with f0(0) = 0: the friction potential per
    unit mu*lambda is f0(|u|), so the force is minus its gradient."""
    return np.where(u < eh, u * u / eh - u ** 3 / (3 * eh * eh), u - eh / 3)


@pytest.mark.parametrize("scale", [0.3, 3.0])  # |u| below and above eps_v h
def test_friction_force_is_gradient_of_lagged_potential(orc, scale):
    p = orc.Params.make(ground_on=True, k_c=1e5, mu_c=0.4, eps_v=0.01)
    eh = p.eps_v * H
    xt = np.array([0.3, -0.2, -0.001])
    d = np.array([0.8, -0.6, 0.25]) * scale * eh
    x = xt + d
    lam = 7.0
    f, Hf = orc.ground_friction(p, H, x, xt, lam)

    def pot(z):
        dz = z - xt
        ut = dz.copy()
        ut[2] = 0.0
        return p.mu_c * lam * _f0(np.linalg.norm(ut), eh)

    e = 1e-7 * eh
    g = np.array([(pot(x + e * np.eye(3)[r]) - pot(x - e * np.eye(3)[r])) / (2 * e) for r in range(3)])
    assert np.allclose(f, -g, rtol=1e-6, atol=1e-9 * np.abs(g).max())
    # approximate Hessian: mu lam f1(|u|)/|u| on the tangent plane, zero along n
    w = np.linalg.eigvalsh(Hf)
    assert w.min() > -1e-12 and abs(Hf[2, 2]) < 1e-12 and abs(Hf[0, 2]) < 1e-12


def test_friction_f1_is_continuous_and_regular():
    from oracle import oracle as orc
    p = orc.Params.make(ground_on=True, k_c=1e5, mu_c=0.5, eps_v=0.02)
    eh = p.eps_v * H
    xt = np.zeros(3)
    for u in (eh * (1 - 1e-9), eh * (1 + 1e-9)):
        f, _ = orc.ground_friction(p, H, np.array([u, 0.0, 0.0]), xt, 1.0)
        assert f[0] == pytest.approx(-p.mu_c, rel=1e-6)  # f1(eh) = 1 from both sides
    f, Hf = orc.ground_friction(p, H, xt, xt, 1.0)
    assert np.all(f == 0) and Hf[0, 0] == pytest.approx(p.mu_c * 2 / eh)  # f1(u)/u -> 2/(eps_v h)


def _block_on_ground(orc, mu, gravity, v0x, steps, iters=1000):
    m = synth.beam(2, 2, 1, edge=0.1, E=1e6, nu=0.3, pin_face=None)
    model = orc.Model.from_mesh(m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    p = orc.Params.make(gravity=gravity, ground_on=True, k_c=1e6, mu_c=mu, eps_v=1e-3)
    x = m.rest.copy()
    v = np.zeros_like(x)
    v[:, 0] = v0x
    vp = v.copy()
    vs = []
    for _ in range(steps):
        model.step(p, colors, nc, H, iters, x, v, vp)
        vs.append(v[:, 0].mean())
    return np.array(vs), x


def test_sliding_block_decelerates_at_mu_g(orc):
    """Coulomb regime (|u| >> eps_v h), steps solved to convergence: once the
    contact has settled the normal forces carry the weight, so the mean
    tangential velocity falls by mu g per unit time."""
    mu = 0.3
    vs, _ = _block_on_ground(orc, mu, (0, 0, -9.8), 1.0, 16)
    decel = (vs[5] - vs[15]) / (10 * H)
    assert decel == pytest.approx(mu * 9.8, rel=0.03)


def test_block_sticks_below_friction_angle_and_slides_above(orc):
    mu = 0.5
    th = np.arctan(0.5 * mu)  # tan(theta) = mu / 2 < mu: sticks
    g = 9.8 * np.array([np.sin(th), 0.0, -np.cos(th)])
    vs, _ = _block_on_ground(orc, mu, g, 0.0, 20)
    assert abs(vs[-1]) < 2e-3  # creeps at most at the eps_v scale
    th = np.arctan(2.0 * mu)  # slides: a = g (sin - mu cos)
    g = 9.8 * np.array([np.sin(th), 0.0, -np.cos(th)])
    vs, _ = _block_on_ground(orc, mu, g, 0.0, 20)
    acc = (vs[19] - vs[9]) / (10 * H)
    assert acc == pytest.approx(9.8 * (np.sin(th) - mu * np.cos(th)), rel=0.03)
