"""Pins of the oracle's element routines (stable neo-Hookean tet, Sec. 5;
gradient and Hessian blocks entering Eqs. 8-9) against finite differences,
invariances and closed forms.  CPU only."""
import numpy as np
import pytest

from paper_2403_06321_b300 import synth


def _rand_tet(seed, deform=0.15):
    rng = np.random.default_rng(seed)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.1
    X += rng.uniform(-0.02, 0.02, X.shape)
    x = X + rng.uniform(-deform, deform, X.shape) * 0.1
    return X, x


def test_rest_tet_inverse_and_volume(orc):
    X = np.array([[0, 0, 0], [2, 0, 0], [0, 3, 0], [0, 0, 4]], float)
    B, V = orc.rest_tet(X)
    Dm = (X[1:] - X[0]).T
    assert np.allclose(Dm @ B, np.eye(3), atol=1e-14)
    assert V == pytest.approx(2 * 3 * 4 / 6.0, rel=1e-14)
    # an inverted (negatively oriented) tet has the same volume
    B2, V2 = orc.rest_tet(X[[0, 2, 1, 3]])
    assert V2 == pytest.approx(V, rel=1e-14)
    with pytest.raises(ValueError):
        orc.rest_tet(np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 1, 0]], float))


def test_F_is_identity_at_rest_and_affine(orc):
    X, _ = _rand_tet(1)
    B, _ = orc.rest_tet(X)
    assert np.allclose(orc.tet_F(X, B), np.eye(3), atol=1e-13)
    A = np.array([[1.1, 0.2, -0.1], [0.05, 0.9, 0.3], [0.0, -0.2, 1.3]])
    t = np.array([0.3, -0.2, 0.5])
    assert np.allclose(orc.tet_F(X @ A.T + t, B), A, atol=1e-12)


def test_cofactor_is_derivative_of_det(orc):
    rng = np.random.default_rng(3)
    F = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
    Cf = orc.cofactor(F)
    assert np.allclose(Cf, np.linalg.det(F) * np.linalg.inv(F).T, rtol=1e-12, atol=1e-12)


def test_uniform_scaling_closed_form(orc):
    mu, lam = orc.lame(1e5, 0.4)
    alpha = 1 + mu / lam
    for s in (0.7, 1.0, 1.3):
        F = s * np.eye(3)
        psi = 0.5 * mu * (3 * s * s - 3) + 0.5 * lam * (s ** 3 - alpha) ** 2
        assert orc.psi(F, mu, lam) == pytest.approx(psi, rel=1e-13, abs=1e-12)
        P = (mu * s + lam * (s ** 3 - alpha) * s * s) * np.eye(3)
        assert np.allclose(orc.pk1(F, mu, lam), P, rtol=1e-12, atol=1e-9)
    # stress free at rest (the reading alpha = 1 + mu/lam)
    assert np.allclose(orc.pk1(np.eye(3), mu, lam), 0, atol=1e-9)
    # without the log term the rest energy is the constant lam/2 (mu/lam)^2
    assert orc.psi(np.eye(3), mu, lam) == pytest.approx(mu * mu / (2 * lam), rel=1e-13)


def test_small_strain_limit_is_linear_elasticity(orc):
    """P(I + eps G) / eps -> mu (G + G^T) + lambda_L tr(G) I with the textbook
    Lame pair of (E, nu): pins the Lame mapping and alpha together."""
    E, nu = 2.5e5, 0.35
    mu, lam = orc.lame(E, nu)
    mu_tb = E / (2 * (1 + nu))
    lam_tb = E * nu / ((1 + nu) * (1 - 2 * nu))
    G = np.array([[0.3, -0.7, 0.2], [0.4, 0.1, -0.5], [0.6, 0.2, -0.9]])
    eps = 1e-7
    lin = (orc.pk1(np.eye(3) + eps * G, mu, lam) - orc.pk1(np.eye(3) - eps * G, mu, lam)) / (2 * eps)
    ref = mu_tb * (G + G.T) + lam_tb * np.trace(G) * np.eye(3)
    assert np.allclose(lin, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())


def test_pk1_is_gradient_of_psi(orc):
    rng = np.random.default_rng(5)
    mu, lam = orc.lame(1e6, 0.45)
    F = np.eye(3) + 0.2 * rng.normal(size=(3, 3))
    P = orc.pk1(F, mu, lam)
    eps = 1e-6
    num = np.zeros((3, 3))
    for r in range(3):
        for s in range(3):
            d = np.zeros((3, 3)); d[r, s] = eps
            num[r, s] = (orc.psi(F + d, mu, lam) - orc.psi(F - d, mu, lam)) / (2 * eps)
    assert np.allclose(P, num, rtol=1e-6, atol=1e-6 * np.abs(P).max())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tet_gradient_matches_fd_of_energy(orc, seed):
    X, x = _rand_tet(seed)
    B, V = orc.rest_tet(X)
    mu, lam = orc.lame(1e5, 0.4)
    g = orc.tet_grad(x, B, V, mu, lam)
    h = 1e-6 * 0.1
    num = np.zeros((4, 3))
    for k in range(4):
        for r in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, r] += h; xm[k, r] -= h
            num[k, r] = (orc.tet_energy(xp, B, V, mu, lam) - orc.tet_energy(xm, B, V, mu, lam)) / (2 * h)
    assert np.allclose(g, num, rtol=1e-6, atol=1e-6 * np.abs(g).max())
    # translation invariance: the four vertex forces sum to zero
    assert np.allclose(g.sum(axis=0), 0, atol=1e-10 * np.abs(g).max())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tet_hessian_blocks_match_fd_of_gradient(orc, seed):
    """All 16 blocks, including the (J - alpha) [F(g_l x g_k)]_x skew term of
    the off-diagonal ones; diagonal blocks have no such term."""
    X, x = _rand_tet(seed + 10, deform=0.3)
    B, V = orc.rest_tet(X)
    mu, lam = orc.lame(1e5, 0.4)
    H = orc.tet_hess(x, B, V, mu, lam)
    h = 1e-6 * 0.1
    num = np.zeros((12, 12))
    for l in range(4):
        for s in range(3):
            xp, xm = x.copy(), x.copy()
            xp[l, s] += h; xm[l, s] -= h
            dg = orc.tet_grad(xp, B, V, mu, lam) - orc.tet_grad(xm, B, V, mu, lam)
            num[:, 3 * l + s] = (dg / (2 * h)).reshape(-1)
    assert np.allclose(H, num, rtol=1e-6, atol=1e-6 * np.abs(H).max())
    assert np.allclose(H, H.T, atol=1e-9 * np.abs(H).max())
    for k in range(4):
        for l in range(4):
            assert np.allclose(orc.tet_hess_block(x, B, V, mu, lam, k, l), H[3 * k:3 * k + 3, 3 * l:3 * l + 3])
    # the diagonal block is mu|g|^2 I + lam c c^T: symmetric PSD
    for k in range(4):
        w = np.linalg.eigvalsh(H[3 * k:3 * k + 3, 3 * k:3 * k + 3])
        assert w.min() > 0


def test_rigid_motion_invariance(orc):
    rng = np.random.default_rng(7)
    mu, lam = orc.lame(1e6, 0.45)
    for seed in range(5):
        R = synth.random_rotation(seed)
        F = np.eye(3) + 0.25 * rng.normal(size=(3, 3))
        assert orc.psi(R @ F, mu, lam) == pytest.approx(orc.psi(F, mu, lam), rel=1e-12)
        assert np.allclose(orc.pk1(R @ F, mu, lam), R @ orc.pk1(F, mu, lam), rtol=1e-11, atol=1e-6)
    # element energy is invariant under rotating + translating the vertices
    X, x = _rand_tet(4)
    B, V = orc.rest_tet(X)
    R = synth.random_rotation(11)
    e0 = orc.tet_energy(x, B, V, mu, lam)
    e1 = orc.tet_energy(x @ R.T + np.array([1.0, -2.0, 0.5]), B, V, mu, lam)
    assert e1 == pytest.approx(e0, rel=1e-11)


def test_lumped_mass_sums_to_total_mass(orc):
    # the 6-tet split tiles the box exactly: volumes add up to the box
    m = synth.beam(3, 2, 2, edge=0.1, rho=1000.0)
    B, V, mu, lam = orc.Model.from_mesh(m).tet_data()
    assert V.sum() == pytest.approx(0.3 * 0.2 * 0.2, rel=1e-12)
    m = synth.beam(3, 2, 2, edge=0.1, rho=1000.0, jitter_frac=0.1, seed=3)
    model = orc.Model.from_mesh(m)
    B, V, mu, lam = model.tet_data()
    assert model.mass().sum() == pytest.approx(1000.0 * V.sum(), rel=1e-12)
