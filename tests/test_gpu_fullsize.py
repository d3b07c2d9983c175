"""Parity at the full size of the benchmark workload (100^3 cubes, 1,030,301
vertices, 6,000,000 tets, ground penalty 1e7) in the launch configuration
bench.py times.  The oracle cannot run whole steps at this size in seconds,
so it checks (a) sampled vertices of the first colour pass one by one, each
an exact function of the seeded input state, and (b) a property that holds
at any size: without contact, no colour pass raises the FP64 energy G."""
import numpy as np
import pytest
import torch

from paper_2403_06321_b300 import synth, vbd
from gpu_util import bbox_diag, params_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    from paper_2403_06321_b300.build import build
    build()
    m, cfg = synth.large_cube(100)
    x0, v0 = synth.perturbed_state(m.rest, 0.0005, 0.5, seed=31)
    # float32-representable so both sides read the same numbers
    x0 = x0.astype(np.float32).astype(np.float64)
    v0 = v0.astype(np.float32).astype(np.float64)
    return m, cfg, x0, v0


def test_first_colour_pass_sampled(orc, big):
    m, cfg, x0, v0 = big
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(cfg)
    sim = vbd.Sim(m, vbd.make_params(**pd), colors=colors)
    try:
        sim.set_state(x0, v0)
        vbd.vbd_begin_step(sim.ctx, cfg.h)
        vbd.vbd_sweep_color(sim.ctx, 0)
        xg, _ = sim.get_state()
        xg = xg.cpu().numpy().astype(np.float64)
        vbd.vbd_end_step(sim.ctx)
        sim.sync_status()
    finally:
        sim.close()
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(**pd)
    y = model.inertia_target(p, cfg.h, x0, v0)
    xi = model.initial_guess(p, cfg.h, x0, v0, v0)
    rng = np.random.default_rng(32)
    c0 = np.nonzero(colors == 0)[0]
    others = np.nonzero(colors != 0)[0]
    diag = bbox_diag(m.rest)
    worst = 0.0
    for i in rng.choice(c0, 400, replace=False):
        dx, skipped, _ = model.vertex_solve(p, cfg.h, i, xi, y, x0)
        assert skipped == 0
        worst = max(worst, float(np.abs(xg[i] - (xi[i] + dx)).max()))
    for i in rng.choice(others, 200, replace=False):
        worst = max(worst, float(np.abs(xg[i] - xi[i]).max()))
    print("large cube first pass: worst |x_gpu - x_oracle| / bbox = %.3e" % (worst / diag))
    assert worst <= 1e-6 * diag


def test_energy_never_rises_per_pass(big):
    m, cfg, x0, v0 = big
    pd = params_of(cfg)  # the cube starts 0.5 m above the ground: no contact
    sim = vbd.Sim(m, vbd.make_params(**pd), colors=synth.kuhn_coloring(m.grid_ijk))
    try:
        sim.set_state(x0, v0)
        vbd.vbd_begin_step(sim.ctx, cfg.h)
        G = [sim.energy()]
        for it in range(2):
            for c in range(4):
                vbd.vbd_sweep_color(sim.ctx, c)
                G.append(sim.energy())
        vbd.vbd_end_step(sim.ctx)
        sim.sync_status()
    finally:
        sim.close()
    G = np.array(G)
    print("large cube G per pass:", G)
    assert np.all(np.diff(G) <= 1e-9 * np.abs(G[:-1]))
    assert G[-1] < G[0]


def test_sweep_variants_agree_at_full_size(big):
    """One full iteration (all colours) of the benchmark cube with each sweep
    kernel: the persistent grid and the warp-row stream equal the plain grid
    bit for bit at equal lanes, the TMA-staged kernel equals the plain 8-lane sweep bit for bit,
    the two-phase scatter agrees to FP32 rounding, the compact slots (shape
    gradients from the rest positions) to 1e-6 of the bbox, as do the packed
    two-slot compact pass and the compact pass, and the fused cluster
    loop refuses a mesh this large."""
    m, cfg, x0, v0 = big
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(cfg)
    out = {}
    sim = vbd.Sim(m, vbd.make_params(scatter_sweep=True, warp_rows=True, **pd), colors=colors)
    try:
        for key, (lanes, block, variant) in {"plain4": (4, 256, 0), "persist4": (4, 256, 2),
                                             "plain8": (8, 256, 0), "tma8": (8, 256, 1),
                                             "scatter4": (4, 256, 3), "rest4": (4, 256, 5),
                                             "pair4": (4, 256, 6), "rows4": (4, 256, 7)}.items():
            vbd.vbd_set_launch(sim.ctx, lanes, block if variant != 1 else 256, variant)
            sim.set_state(x0, v0)
            vbd.vbd_begin_step(sim.ctx, cfg.h)
            vbd.vbd_iterate(sim.ctx, 1)
            vbd.vbd_end_step(sim.ctx)
            sim.sync_status()
            out[key] = sim.get_state()[0].cpu().numpy()
        with pytest.raises(vbd.VbdError) as e:
            vbd.vbd_set_launch(sim.ctx, 4, 0, 4)
        assert e.value.status == "VBD_ERR_INVALID_ARG"
    finally:
        sim.close()
    assert np.array_equal(out["persist4"], out["plain4"])
    assert np.array_equal(out["rows4"], out["plain4"])
    assert np.array_equal(out["tma8"], out["plain8"])
    diag = bbox_diag(m.rest)
    assert float(np.abs(out["scatter4"] - out["plain4"]).max()) <= 1e-7 * diag
    assert float(np.abs(out["plain8"] - out["plain4"]).max()) <= 1e-7 * diag
    # gradients from the FP32 rest positions instead of the FP64-derived ones
    rest_err = float(np.abs(out["rest4"] - out["plain4"]).max()) / diag
    pair_err = float(np.abs(out["pair4"] - out["rest4"]).max()) / diag
    print("compact rest slots vs stored gradients: %.2e of the bbox; packed pairs vs compact: %.2e" % (
        rest_err, pair_err))
    assert rest_err <= 1e-6
    assert pair_err <= 1e-6


_ORACLE_TWO_STEPS = r'''
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from oracle import oracle
from paper_2403_06321_b300 import synth
m, cfg = synth.large_cube(100)
x0, v0 = synth.perturbed_state(m.rest, 0.0005, 0.5, seed=31)
x = x0.astype(np.float32).astype(np.float64)
v = v0.astype(np.float32).astype(np.float64)
vp = v.copy()
model = oracle.Model.from_mesh(m)
p = oracle.Params.make(gravity=cfg.gravity, ground_on=cfg.ground_on, ground_height=cfg.ground_height,
                       ground_normal=cfg.ground_normal, k_c=cfg.k_c, init_mode=cfg.init_mode, det_eps=cfg.det_eps)
colors = synth.kuhn_coloring(m.grid_ijk)
for _ in range(int(sys.argv[3])):
    model.step(p, colors, 4, cfg.h, cfg.iters, x, v, vp)
np.save(sys.argv[2], x)
'''


def test_two_full_steps_every_vertex(big, tmp_path):
    """The benchmark workload at full size (1.03M vertices, 100 iterations per
    step) from a deformed state with 0.5 m/s random velocities: two whole
    steps on the GPU against two whole steps of the FP64 oracle, every
    vertex compared.  The oracle runs its OpenMP build (bit-identical to the
    serial one) in a child process on all host cores."""
    import os
    import subprocess
    import sys
    from oracle import oracle
    m, cfg, x0, v0 = big
    steps = 2
    colors = synth.kuhn_coloring(m.grid_ijk)
    sim = vbd.Sim(m, vbd.make_params(**params_of(cfg)), colors=colors)
    try:
        sim.set_state(x0, v0)
        for _ in range(steps):
            sim.step(cfg.h, cfg.iters)
        sim.sync_status()
        xg = sim.get_state()[0].cpu().numpy().astype(np.float64)
    finally:
        sim.close()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "x.npy")
    env = dict(os.environ, VBD_ORACLE_LIB=oracle.build(openmp=True))
    subprocess.run([sys.executable, "-c", _ORACLE_TWO_STEPS, root, out, str(steps)], check=True, env=env,
                   timeout=1800)
    xo = np.load(out)
    diag = bbox_diag(m.rest)
    err = float(np.abs(xg - xo).max()) / diag
    print("large cube, two full steps from a deformed state: max err / bbox = %.3e (moved %.3e)" % (
        err, float(np.abs(xo - x0).max())))
    assert float(np.abs(xo - x0).max()) > 1e-3
    assert err <= 1e-5


def test_adjoint_one_sweep_sampled(orc, big):
    """The adjoint's first block Gauss-Seidel sweep at full size, where each
    colour pass takes several turns of the persistent grid.  With one recorded
    step, lam = 0 before the sweep and dL/dv0 = M/h lam after it, and for the
    first two colours lam after one sweep is an exact function of the recorded
    state: colour 0: lam_i = H_ii^-1 r_i; colour 1: lam_i = H_ii^-1 (r_i -
    sum_k H_ik lam_k) over its colour-0 neighbours k (the others are still 0),
    with r = dL/dx_T and H = M/h^2 + d2E/dx2 (+ ground) at the recorded
    positions.  Sampled vertices across each colour's whole range are
    recomputed in FP64 from the oracle's element Hessian blocks."""
    m, cfg, x0, v0 = big
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(cfg)
    sim = vbd.Sim(m, vbd.make_params(tape_steps=1, **pd), colors=colors)
    rng = np.random.default_rng(41)
    g = rng.normal(0.0, 1.0, size=m.rest.shape)
    try:
        dev = sim.workspace.device
        sim.set_state(x0, v0)
        sim.step(cfg.h, cfg.iters)
        x1 = sim.get_state()[0].cpu().numpy().astype(np.float64)
        gx = torch.tensor(g.reshape(-1), dtype=torch.float32, device=dev)
        gE = torch.empty(m.n_tets, dtype=torch.float32, device=dev)
        gv = torch.empty(3 * m.n_verts, dtype=torch.float32, device=dev)
        vbd.vbd_backward(sim.ctx, gx, gE, gv, 1)
        sim.sync_status()
        gv = gv.cpu().numpy().astype(np.float64).reshape(-1, 3)
    finally:
        sim.close()
    r = g.astype(np.float32).astype(np.float64)  # the seed as the GPU read it
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(**pd)
    h = cfg.h
    mass = model.mass()
    B, V, mu, lam = model.tet_data()
    tets = m.tets
    order = np.argsort(tets.reshape(-1), kind="stable")
    start = np.searchsorted(tets.reshape(-1)[order], np.arange(m.n_verts + 1))
    planes = model._plane_terms(p, x1)

    def incident(i):
        e = order[start[i]:start[i + 1]]
        return e // 4, e % 4

    def block(j, a, b):
        return orc.tet_hess_block(x1[tets[j]].reshape(-1), B[j], V[j], mu[j], lam[j], int(a), int(b))

    def h_ii(i):
        H = mass[i] / h ** 2 * np.eye(3)
        for j, a in zip(*incident(i)):
            H += block(j, a, a)
        for nrm, _, act in planes:
            if act[i]:
                H += p.k_c * np.outer(nrm, nrm)
        return H

    lam0 = {}

    def lam_colour0(k):
        if k not in lam0:
            lam0[k] = np.linalg.solve(h_ii(k), r[k])
        return lam0[k]

    turn = torch.cuda.get_device_properties(0).multi_processor_count * 8 * 128 // 4
    for c in (0, 1):
        ids = np.nonzero(colors == c)[0]
        sample = ids[np.unique(np.linspace(0, len(ids) - 1, 120).astype(np.int64))]
        want = np.zeros((len(sample), 3))
        for s, i in enumerate(sample):
            b = r[i].copy()
            if c == 1:
                for j, a in zip(*incident(i)):
                    for bl in range(4):
                        k = tets[j][bl]
                        if bl != a and colors[k] == 0:
                            b -= block(j, a, bl) @ lam_colour0(k)
            want[s] = np.linalg.solve(h_ii(i), b)
        got = gv[sample] * h / mass[sample][:, None]
        err = float(np.abs(got - want).max() / np.abs(want).max())
        print("adjoint one sweep, colour %d (%d vertices, about %.1f turns of the grid): max err / max |lam| = %.2e"
              % (c, len(ids), len(ids) / turn, err))
        assert err <= 1e-4
