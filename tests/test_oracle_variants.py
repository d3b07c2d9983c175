"""Pins of the oracle's optional solver variants: the local backtracking line
search (Sec. 3.2, Algorithm 1) and block-Jacobi iterations (all vertices
against the previous iterate).  CPU only."""
import numpy as np
import pytest

from paper_2403_06321_b300 import synth

H = 1.0 / 60.0


def test_line_search_keeps_full_steps_without_contact(orc):
    """Without contact G_i is an exact quadratic with an SPD Hessian, so the
    Newton step is its minimiser and the search accepts alpha = 1."""
    m = synth.beam(5, 2, 2, E=1e5, nu=0.4, jitter_frac=0.1, seed=71)
    model = orc.Model.from_mesh(m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    v0 = np.random.default_rng(72).normal(0, 0.3, m.rest.shape)
    xa, _, _ = orc.run(model, orc.Params.make(), colors, nc, H, 6, 4, m.rest, v0)
    xb, _, _ = orc.run(model, orc.Params.make(line_search=True), colors, nc, H, 6, 4, m.rest, v0)
    assert np.abs(xa - xb).max() <= 1e-12


def test_line_search_never_raises_local_or_global_energy_with_contact(orc):
    """With a stiff ground penalty a full Newton step from the free side can
    overshoot; with the search every vertex update lowers G_i, hence G, and
    every colour pass is monotone (the guarantee the search exists for)."""
    m = synth.beam(4, 3, 2, edge=0.05, E=1e4, nu=0.4, pin_face=None, jitter_frac=0.1, seed=73,
                   origin=(0, 0, 0.004))
    model = orc.Model.from_mesh(m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    v = np.zeros_like(m.rest)
    v[:, 2] = -5.0  # hits the ground within the step
    xt = m.rest.copy()
    rises = {}
    for ls in (False, True):
        p = orc.Params.make(ground_on=True, k_c=1e8, line_search=ls)
        y = model.inertia_target(p, H, xt, v)
        x = model.initial_guess(p, H, xt, v, v)
        G = model.energy_G(p, H, x, y)
        rises[ls] = 0
        for it in range(6):
            for c in range(nc):
                model.sweep_color(p, H, colors, c, x, y, xt)
                G1 = model.energy_G(p, H, x, y)
                rises[ls] += int(G1 > G + 1e-12 * abs(G))
                G = G1
    assert rises[True] == 0
    assert rises[False] > 0  # the case does exercise the search


def test_local_energy_matches_global_energy_difference(orc):
    """Moving one vertex changes G exactly as much as G_i (Sec. 3.1)."""
    m = synth.beam(3, 2, 2, jitter_frac=0.1, seed=74)
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(ground_on=True, ground_height=0.05, k_c=1e5)
    rng = np.random.default_rng(75)
    x = m.rest + rng.normal(0, 0.005, m.rest.shape)
    y = x + rng.normal(0, 0.005, m.rest.shape)
    i = int(np.nonzero(m.pinned == 0)[0][7])
    x2 = x.copy()
    x2[i] += rng.normal(0, 0.01, 3)
    dG = model.energy_G(p, H, x2, y) - model.energy_G(p, H, x, y)
    dGi = model.local_energy(p, H, i, x2, y) - model.local_energy(p, H, i, x, y)
    assert dGi == pytest.approx(dG, rel=1e-9)


def test_block_jacobi_converges_to_dense_newton(orc):
    """Jacobi needs the inertia term to dominate the coupling (it diverges on
    stiffer settings where Gauss-Seidel still converges); on a soft beam it
    reaches the same fixed point as Gauss-Seidel and dense Newton."""
    m = synth.beam(3, 1, 1, E=2e3, nu=0.4, jitter_frac=0.1, seed=76)
    model = orc.Model.from_mesh(m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    p = orc.Params.make(jacobi=True)
    xt = m.rest.copy()
    v = np.zeros_like(xt)
    xj, _, _ = orc.run(model, p, colors, nc, H, 4000, 1, xt, v)
    y = model.inertia_target(p, H, xt, v)
    x_nt = model.newton_solve(orc.Params.make(), H, xt, y)
    assert np.abs(xj - x_nt).max() <= 1e-9


def test_block_jacobi_ignores_the_colouring(orc):
    """Every vertex reads only the previous iterate, so the colouring and the
    visiting order cannot change one Jacobi iteration, while they do change
    a Gauss-Seidel one."""
    m = synth.beam(4, 2, 2, E=1e5, nu=0.4, jitter_frac=0.1, seed=77)
    model = orc.Model.from_mesh(m)
    c1, n1 = orc.color_greedy(m.n_verts, m.tets)
    c2 = synth.kuhn_coloring(m.grid_ijk)
    v0 = np.random.default_rng(78).normal(0, 0.3, m.rest.shape)
    pj = orc.Params.make(jacobi=True)
    a, _, _ = orc.run(model, pj, c1, n1, H, 3, 2, m.rest, v0)
    b, _, _ = orc.run(model, pj, c2, 4, H, 3, 2, m.rest, v0)
    assert np.array_equal(a, b)
    pg = orc.Params.make()
    a, _, _ = orc.run(model, pg, c1, n1, H, 3, 2, m.rest, v0)
    b, _, _ = orc.run(model, pg, c2, 4, H, 3, 2, m.rest, v0)
    assert not np.array_equal(a, b)
