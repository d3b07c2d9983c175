"""Seeded random combinations of the options the sweep composes, each run on
the GPU (through the C ABI) and by the FP64 oracle with the same colouring:
mesh shape and jitter, per-tet materials, pins, init mode, ground contact
with friction, world-box walls, subspace constraints, Chebyshev, damping,
line search, colouring and sweep variant.  Tolerance 1e-5 of the bounding-box diagonal."""
import numpy as np
import pytest
import torch

from paper_2403_06321_b300 import synth
from gpu_util import bbox_diag, gpu_run, oracle_run, params_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_06321_b300.build import build
    build()
    assert torch.cuda.is_available()


def _case(seed: int):
    rng = np.random.default_rng(1000 + seed)
    dims = tuple(int(v) for v in rng.integers(1, 10, 3))
    edge = float(rng.choice([0.02, 0.05, 0.1]))
    pin = [None, "x-", "y+", "z-"][int(rng.integers(4))]
    m = synth.beam(*dims, edge=edge, pin_face=pin, jitter_frac=float(rng.uniform(0, 0.12)),
                   seed=int(rng.integers(1 << 30)), origin=(0.0, 0.0, float(rng.uniform(0.0, 0.3)) * edge))
    if rng.random() < 0.5:  # per-tet materials
        m.young = np.exp(rng.uniform(np.log(1e4), np.log(1e6), m.n_tets)).astype(np.float32)
        m.poisson = rng.uniform(0.2, 0.45, m.n_tets).astype(np.float32)
    else:
        m.young[:] = float(np.exp(rng.uniform(np.log(1e4), np.log(1e6))))
    ground = bool(rng.random() < 0.6)
    pd = params_of(synth.SimConfig(),
                   init_mode=int(rng.integers(4)),
                   ground_on=ground, k_c=float(rng.choice([1e4, 1e5, 1e6])),
                   mu_c=float(rng.choice([0.0, 0.2, 0.5])) if ground else 0.0,
                   eps_v=float(rng.choice([1e-3, 1e-2])),
                   cheby_rho=float(rng.choice([0.0, 0.0, 0.6, 0.9])),
                   k_d=float(rng.choice([0.0, 1e-6, 1e-5])),
                   line_search=bool(rng.random() < 0.25))
    v0 = rng.normal(0.0, 0.3, m.rest.shape)
    v0[m.pinned == 1] = 0.0
    v0[:, 2] -= float(rng.uniform(0.0, 1.0))
    greedy = bool(rng.random() < 0.5)
    variant = int(rng.choice([0, 1, 2, 4, 5, 6, 7]))
    lanes = int(rng.choice([4, 8, 16]))
    h = float(rng.choice([1 / 60, 1 / 120, 1 / 300]))
    iters, steps = int(rng.integers(3, 15)), int(rng.integers(2, 8))
    if rng.random() < 0.4:  # world-box walls just outside the rest mesh, slightly tilted
        walls = []
        for w in synth.world_box(m.rest.min(0), m.rest.max(0))[:int(rng.integers(1, 7))]:
            n = np.array(w[:3]) + rng.normal(0.0, 0.1, 3)
            n /= np.linalg.norm(n)
            walls.append(tuple(n) + (float((m.rest @ n).min() - rng.uniform(0.0, 0.5) * edge),))
        pd["walls"] = walls
    if rng.random() < 0.3:  # a few free vertices restricted to random lines or planes
        free = np.nonzero(m.pinned == 0)[0]
        k = rng.choice(free, size=min(len(free), int(rng.integers(1, 12))), replace=False)
        m.sub_dim = np.full(m.n_verts, 3, np.int32)
        m.sub_dir = np.zeros((m.n_verts, 3))
        m.sub_dim[k] = rng.integers(1, 3, len(k))
        m.sub_dir[k] = rng.normal(0, 1, (len(k), 3))
        v0[k] = 0.0  # start on the subspaces with no motion across them
    return m, pd, v0, greedy, variant, lanes, h, iters, steps


@pytest.mark.parametrize("seed", range(24))
def test_random_option_mix_matches_oracle(orc, seed):
    m, pd, v0, greedy, variant, lanes, h, iters, steps = _case(seed)
    colors = orc.color_greedy(m.n_verts, m.tets)[0] if greedy else synth.kuhn_coloring(m.grid_ijk)
    v0 = np.asarray(v0, np.float32).astype(np.float64)
    xg, _ = gpu_run(m, pd, colors, h, iters, steps, v0=v0, variant=variant,
                    lanes=None if variant == 1 else lanes)
    xo, _ = oracle_run(orc, m, pd, colors, h, iters, steps, v0=v0)
    err = float(np.abs(xg - xo).max() / bbox_diag(m.rest))
    print("seed %d: %d verts, variant %d, %s: err %.2e" % (seed, m.n_verts, variant,
                                                          {k: pd[k] for k in ("ground_on", "mu_c", "cheby_rho", "k_d",
                                                                             "line_search", "init_mode")}, err))
    assert np.isfinite(xg).all()
    assert err <= 1e-5
