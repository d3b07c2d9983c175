"""Writes the stored expected values under tests/golden/ from the FP64 oracle
(oracle/) and the seeded input generators (paper_2403_06321_b300.synth),
nothing else.  The paper prints no worked numeric example, so every stored
value here is an oracle output: the fixtures pin the oracle against later
changes to its own arithmetic (tests/test_oracle_golden.py recomputes them),
and their independent checks (finite differences, closed forms) live in the
test beside them.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_2403_06321_b300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

# one rest tet and one deformed placement of it (metres), written out so that
# the fixture states its own input
ELEMENT_REST = np.array([[0.00, 0.00, 0.00],
                         [0.10, 0.01, 0.00],
                         [0.02, 0.11, 0.01],
                         [0.01, 0.02, 0.09]])
ELEMENT_X = np.array([[0.001, -0.002, 0.000],
                      [0.115, 0.012, -0.004],
                      [0.018, 0.098, 0.016],
                      [0.006, 0.025, 0.104]])
ELEMENT_E, ELEMENT_NU = 1e5, 0.4
CHEBY_RHO, CHEBY_N = 0.95, 30
BEAM_STEPS = 10


def _fmt(a) -> str:
    return " ".join("%.17g" % v for v in np.asarray(a, np.float64).reshape(-1))


def element_lines() -> list[str]:
    mu, lam = oracle.lame(ELEMENT_E, ELEMENT_NU)
    B, V = oracle.rest_tet(ELEMENT_REST)
    x = ELEMENT_X.reshape(-1)
    e = oracle.tet_energy(x, B, V, mu, lam)
    g = oracle.tet_grad(x, B, V, mu, lam)
    h00 = oracle.tet_hess_block(x, B, V, mu, lam, 0, 0)
    h01 = oracle.tet_hess_block(x, B, V, mu, lam, 0, 1)
    return ["# One stable neo-Hookean tet (Sec. 5 names the material and prints no formula; read as",
            "# Psi = mu/2 (tr F^T F - 3) + lam/2 (J - alpha)^2, alpha = 1 + mu/lam, with",
            "# mu = E/(2(1+nu)) and lam = E nu/((1+nu)(1-2nu)) + mu): its element energy V Psi, the",
            "# gradient dE/dx_k of Eq. 8 and Hessian blocks of Eq. 9.  Written by",
            "# tests/golden/make_golden.py from oracle/ (FP64).",
            "rest " + _fmt(ELEMENT_REST),
            "deformed " + _fmt(ELEMENT_X),
            "E_nu %.17g %.17g" % (ELEMENT_E, ELEMENT_NU),
            "mu_lam %.17g %.17g" % (mu, lam),
            "V %.17g" % V,
            "B " + _fmt(B),
            "energy %.17g" % e,
            "grad " + _fmt(g),
            "hess_00 " + _fmt(h00),
            "hess_01 " + _fmt(h01)]


def omega_lines() -> list[str]:
    out = ["# Chebyshev acceleration ratios omega_n of Eq. 19 (omega_1 = 1, omega_2 = 2/(2 - rho^2),",
           "# omega_n = 4/(4 - rho^2 omega_{n-1})) for rho = %g, n = 1..%d.  Written by" % (CHEBY_RHO, CHEBY_N),
           "# tests/golden/make_golden.py from oracle/ (FP64).",
           "rho %.17g" % CHEBY_RHO]
    w = 0.0
    for n in range(1, CHEBY_N + 1):
        w = oracle.cheby_omega(n, CHEBY_RHO, w)
        out.append("omega %d %.17g" % (n, w))
    return out


def beam_lines() -> list[str]:
    m, cfg = synth.cantilever_beam()
    colors = synth.kuhn_coloring(m.grid_ijk)
    model = oracle.Model.from_mesh(m)
    p = oracle.Params.make(gravity=cfg.gravity, init_mode=cfg.init_mode, det_eps=cfg.det_eps)
    x, v, _ = oracle.run(model, p, colors, int(colors.max()) + 1, cfg.h, cfg.iters, BEAM_STEPS,
                         m.rest, np.zeros_like(m.rest))
    out = ["# The cantilever workload (synth.cantilever_beam: 10x3x3 cubes of 0.1 m, 176 vertices,",
           "# 540 tets, E = 1e5, nu = 0.4, x = 0 face pinned, g = -9.8 z, h = 1/60, 20 iterations per",
           "# step, Kuhn 4-colouring) after %d steps of Algorithm 1 from rest (Eq. 3 inertia," % BEAM_STEPS,
           "# adaptive initial guess of Sec. 3.7, vertex solves of Eqs. 7-9, Eq. 6 velocities):",
           "# final positions and velocities, one vertex per line in caller order.  Written by",
           "# tests/golden/make_golden.py from oracle/ (FP64).",
           "steps %d" % BEAM_STEPS]
    for i in range(m.n_verts):
        out.append("x %d %s %s" % (i, _fmt(x[i]), _fmt(v[i])))
    return out


def main() -> None:
    oracle.build()
    for name, lines in (("element_tet.txt", element_lines()), ("chebyshev_omega.txt", omega_lines()),
                        ("cantilever_10_steps.txt", beam_lines())):
        with open(os.path.join(HERE, name), "w") as f:
            f.write("\n".join(lines) + "\n")
        print("wrote", name)


if __name__ == "__main__":
    main()
