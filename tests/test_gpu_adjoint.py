"""GPU adjoint (vbd_backward, via the torch.autograd wrapper) against the
oracle's FP64 adjoint of the same steps, and on a converged beam straight
against central finite differences of the FP64 forward.  The oracle adjoint
is itself pinned to central finite differences (tests/test_oracle_adjoint.py).
Gate, element by element: every entry of dL/dlog E within 1e-3 of the
largest |entry| of the oracle's, likewise each component of dL/dv0 against
that component's largest entry, and the same sign wherever the oracle's
entry exceeds 1 % of that largest one (a norm could hide a few hundred
wrong entries among the many small ones).  The relative 2-norm is printed
as a diagnostic only."""
import numpy as np
import pytest
import torch

from paper_2403_06321_b300 import synth, vbd
from paper_2403_06321_b300.autograd import simulate
from gpu_util import params_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_06321_b300.build import build
    build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _elementwise(g, o):
    """Worst |g - o| / max|o| over the columns (one column for dL/dlog E,
    x, y, z for dL/dv0), and the number of sign disagreements among entries
    above 1 % of their column's largest |entry|."""
    g = g.reshape(len(g), -1)
    o = o.reshape(len(o), -1)
    worst, flips = 0.0, 0
    for c in range(o.shape[1]):
        scale = float(np.abs(o[:, c]).max())
        if scale == 0.0:
            assert np.all(g[:, c] == 0.0)
            continue
        worst = max(worst, float(np.abs(g[:, c] - o[:, c]).max()) / scale)
        big = np.abs(o[:, c]) > 0.01 * scale
        flips += int((np.sign(g[big, c]) != np.sign(o[big, c])).sum())
    return worst, flips


def _check(label, gE, oE, gv, ov):
    wE, fE = _elementwise(gE, oE)
    wv, fv = _elementwise(gv, ov)
    print("%s: dlogE worst %.2e (2-norm %.2e, sign flips %d)  dv0 worst %.2e (2-norm %.2e, sign flips %d)" % (
        label, wE, _rel(gE, oE), fE, wv, _rel(gv, ov), fv))
    assert wE <= 1e-3 and wv <= 1e-3
    assert fE == 0 and fv == 0


def _gpu_grads(m, pd, colors, h, iters, steps, v0, tip, target, adj_iters, logE=None, graph=True):
    sim = vbd.Sim(m, vbd.make_params(tape_steps=steps, **pd), colors=colors)
    try:
        vbd.vbd_set_graph(sim.ctx, graph)
        dev = sim.workspace.device
        le = torch.tensor(np.log(m.young.astype(np.float64)) if logE is None else logE,
                          dtype=torch.float32, device=dev, requires_grad=True)
        vv = torch.tensor(v0, dtype=torch.float32, device=dev, requires_grad=True)
        x0 = torch.tensor(m.rest, dtype=torch.float32, device=dev)
        xT = simulate(le, vv, sim, x0, h, iters, steps, adj_iters)
        tip_t = torch.tensor(tip, device=dev)
        tgt = torch.tensor(target, dtype=torch.float32, device=dev)
        loss = ((xT[tip_t] - tgt) ** 2).sum(dim=1).mean()
        gE, gv = torch.autograd.grad(loss, [le, vv])
        sim.sync_status()
        return (gE.cpu().numpy().astype(np.float64), gv.cpu().numpy().astype(np.float64),
                xT.detach().cpu().numpy().astype(np.float64))
    finally:
        sim.close()


def _oracle_grads(orc, m, pd, colors, h, iters, steps, v0, tip, target, newton=False):
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(**pd)
    x, v = m.rest.copy(), np.array(v0, np.float64)
    vp = v.copy()
    xs = [x.copy()]
    for _ in range(steps):
        if newton:
            y = model.inertia_target(p, h, x, v)
            xn = model.newton_solve(p, h, x + h * v, y, tol=1e-13)
            vp, v, x = v, (xn - x) / h, xn
        else:
            model.step(p, colors, int(colors.max()) + 1, h, iters, x, v, vp)
        xs.append(x.copy())
    g = np.zeros_like(x)
    g[tip] = 2.0 / len(tip) * (x[tip] - target)
    gE, gv, _ = orc.dense_adjoint(model, p, h, xs, g)
    return gE, gv, x


def test_adjoint_converged_small_beam(orc):
    """6x2x2 beam, 4 steps solved to convergence on both sides."""
    m = synth.beam(6, 2, 2, E=1e5, nu=0.4, jitter_frac=0.05, seed=51)
    colors, _ = orc.color_greedy(m.n_verts, m.tets)
    pd = params_of(synth.SimConfig())
    rng = np.random.default_rng(52)
    v0 = rng.normal(0, 0.3, m.rest.shape) * (1 - m.pinned[:, None])
    tip = np.nonzero(m.grid_ijk[:, 0] == 6)[0]
    target = m.rest[tip] + np.array([0.05, -0.03, 0.08])
    h, steps = 1 / 60, 4
    gE, gv, xg = _gpu_grads(m, pd, colors, h, 400, steps, v0, tip, target, adj_iters=300)
    oE, ov, xo = _oracle_grads(orc, m, pd, colors, h, 0, steps, v0, tip, target, newton=True)
    print("small beam: |x|err %.2e" % np.abs(xg - xo).max())
    assert np.abs(xg - xo).max() < 1e-5
    _check("small beam", gE, oE, gv, ov)
    assert np.all(gv[m.pinned == 1] == 0)


def test_adjoint_against_central_fd(orc):
    """The GPU adjoint straight against central finite differences of the
    loss (no oracle adjoint in between): the 6x2x2 beam of the test above, 4
    steps, the GPU forward and adjoint run to convergence; the differences
    are taken on the FP64 forward solved by dense Newton for sampled tets'
    log E and sampled components of v0.  Gate: every sampled entry within
    1e-3 of its column's largest |entry|.  Steps: 3e-2 in log E and 1e-2
    m/s in v0.  The converged forward leaves about 1e-11 of noise in the
    loss and the dL/dlog E entries here are only ~1e-5, so smaller steps
    measure the noise (at 1e-4 the quotient is off by 1e-2 of the largest
    entry); at these steps the central differences agree with the oracle's
    dense adjoint to 1e-4 (log E) and 1e-5 (v0) of the largest entry."""
    m = synth.beam(6, 2, 2, E=1e5, nu=0.4, jitter_frac=0.05, seed=51)
    colors, _ = orc.color_greedy(m.n_verts, m.tets)
    pd = params_of(synth.SimConfig())
    rng = np.random.default_rng(52)
    v0 = rng.normal(0, 0.3, m.rest.shape) * (1 - m.pinned[:, None])
    tip = np.nonzero(m.grid_ijk[:, 0] == 6)[0]
    target = m.rest[tip] + np.array([0.05, -0.03, 0.08])
    h, steps = 1 / 60, 4
    gE, gv, _ = _gpu_grads(m, pd, colors, h, 400, steps, v0, tip, target, adj_iters=300)
    model = orc.Model.from_mesh(m)
    p = orc.Params.make(**pd)
    logE = np.log(m.young.astype(np.float64))

    def loss(le, vv):
        model.set_log_young(le)
        x, v = m.rest.copy(), np.array(vv, np.float64)
        for _ in range(steps):
            y = model.inertia_target(p, h, x, v)
            xn = model.newton_solve(p, h, x + h * v, y, tol=1e-14, max_iter=60)
            v, x = (xn - x) / h, xn
        d = x[tip] - target
        return float((d * d).sum(axis=1).mean())

    eps_E, eps_v = 3e-2, 1e-2
    worst_E = worst_v = 0.0
    for j in rng.choice(m.n_tets, 6, replace=False):
        e = np.zeros_like(logE)
        e[j] = eps_E
        fd = (loss(logE + e, v0) - loss(logE - e, v0)) / (2 * eps_E)
        worst_E = max(worst_E, abs(gE[j] - fd) / np.abs(gE).max())
    free = np.nonzero(m.pinned == 0)[0]
    for i in rng.choice(free, 4, replace=False):
        for r in range(3):
            dv = np.zeros_like(v0)
            dv[i, r] = eps_v
            fd = (loss(logE, v0 + dv) - loss(logE, v0 - dv)) / (2 * eps_v)
            worst_v = max(worst_v, abs(gv[i, r] - fd) / np.abs(gv[:, r]).max())
    print("GPU adjoint vs central FD: dlogE worst %.2e, dv0 worst %.2e (of the column's largest entry)" % (
        worst_E, worst_v))
    assert worst_E <= 1e-3 and worst_v <= 1e-3


def test_backward_graph_equals_eager():
    """The backward's step loop replayed as one CUDA graph gives the same
    gradients, bit for bit, as its launches issued one by one; a second
    backward through the same context (the cached graph) repeats them."""
    m, cfg, tip, target = synth.differentiable_beam()
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(cfg)
    v0 = np.zeros_like(m.rest)
    steps = 6
    out = {}
    for graph in (True, False):
        out[graph] = _gpu_grads(m, pd, colors, cfg.h, cfg.iters, steps, v0, tip, target, adj_iters=40,
                                graph=graph)
    for a, b in zip(out[True], out[False]):
        assert np.array_equal(a, b)
    sim = vbd.Sim(m, vbd.make_params(tape_steps=steps, **pd), colors=colors)
    try:
        dev = sim.workspace.device
        sim.set_state(m.rest, v0)
        for _ in range(steps):
            sim.step(cfg.h, cfg.iters)
        gx = torch.zeros(3 * m.n_verts, dtype=torch.float32, device=dev)
        gx[2::3] = 1.0
        res = []
        for _ in range(2):
            gE = torch.empty(m.n_tets, dtype=torch.float32, device=dev)
            gv = torch.empty(3 * m.n_verts, dtype=torch.float32, device=dev)
            vbd.vbd_backward(sim.ctx, gx, gE, gv, 40)
            torch.cuda.synchronize()  # the backward runs on the context's stream
            res.append((gE.cpu().numpy(), gv.cpu().numpy()))
        sim.sync_status()
    finally:
        sim.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert np.abs(res[0][1]).max() > 0
    # a new recording with another step size in a context that holds a captured
    # backward: the cached graph does not match it, a new one is captured, and
    # the gradients equal those of eager launches
    h2 = 0.5 * cfg.h
    out2 = {}
    for graph in (True, False):
        sim = vbd.Sim(m, vbd.make_params(tape_steps=steps, **pd), colors=colors)
        try:
            vbd.vbd_set_graph(sim.ctx, graph)
            dev = sim.workspace.device
            for h in ((cfg.h, h2) if graph else (h2,)):
                sim.set_state(m.rest, v0)
                for _ in range(steps):
                    sim.step(h, cfg.iters)
                gE = torch.empty(m.n_tets, dtype=torch.float32, device=dev)
                gv = torch.empty(3 * m.n_verts, dtype=torch.float32, device=dev)
                vbd.vbd_backward(sim.ctx, gx, gE, gv, 40)
                torch.cuda.synchronize()
            out2[graph] = (gE.cpu().numpy(), gv.cpu().numpy())
            sim.sync_status()
        finally:
            sim.close()
    assert np.array_equal(out2[True][0], out2[False][0]) and np.array_equal(out2[True][1], out2[False][1])
    assert not np.array_equal(out2[True][1], res[0][1])


def test_adjoint_differentiable_beam_full_size(orc):
    """40x8x8 beam (3,321 verts, 15,360 tets), 30 steps of 50 iterations; both
    sides run the same fixed-iteration forward and apply the converged-step
    adjoint at their own recorded positions."""
    m, cfg, tip, target = synth.differentiable_beam()
    colors = synth.kuhn_coloring(m.grid_ijk)
    pd = params_of(cfg)
    v0 = np.zeros_like(m.rest)
    gE, gv, xg = _gpu_grads(m, pd, colors, cfg.h, cfg.iters, cfg.steps, v0, tip, target, adj_iters=150)
    oE, ov, xo = _oracle_grads(orc, m, pd, colors, cfg.h, cfg.iters, cfg.steps, v0, tip, target)
    diag = float(np.linalg.norm(m.rest.max(0) - m.rest.min(0)))
    print("differentiable beam: x err/bbox %.2e" % (np.abs(xg - xo).max() / diag))
    assert np.abs(xg - xo).max() <= 1e-5 * diag
    _check("differentiable beam", gE, oE, gv, ov)


def test_adjoint_with_ground_contact(orc):
    """A free block falling onto the ground (k_c = 1e5), 6 steps solved to
    convergence on both sides; the adjoint then includes the contact
    Hessian k_c n n^T of every penetrating vertex."""
    m = synth.beam(4, 3, 2, edge=0.05, E=1e5, nu=0.4, pin_face=None, jitter_frac=0.05, seed=53)
    m.rest[:, 2] -= m.rest[:, 2].min()  # lowest vertex on the plane
    colors, _ = orc.color_greedy(m.n_verts, m.tets)
    pd = params_of(synth.SimConfig(), ground_on=True, k_c=1e5)
    rng = np.random.default_rng(54)
    v0 = rng.normal(0, 0.05, m.rest.shape)
    v0[:, 2] = -0.3
    top = np.nonzero(m.grid_ijk[:, 2] == 2)[0]
    target = m.rest[top] + np.array([0.01, -0.02, -0.01])
    h, steps = 1 / 60, 6
    gE, gv, xg = _gpu_grads(m, pd, colors, h, 600, steps, v0, top, target, adj_iters=400)
    oE, ov, xo = _oracle_grads(orc, m, pd, colors, h, 0, steps, v0, top, target, newton=True)
    assert (xo[:, 2] < 0).sum() >= 4  # vertices in contact at the last step
    print("ground contact: |x|err %.2e" % np.abs(xg - xo).max())
    assert np.abs(xg - xo).max() < 1e-5
    _check("ground contact", gE, oE, gv, ov)
