"""The batched workload at full size: 4096 independent beams (cube counts
U{4..40} x U{2..8} x U{2..8}, E log-uniform [1e4, 1e6], nu U[0.3, 0.48], a
random face pinned), h = 1/60, 30 iterations per step, 50 steps, swept as one
union in one launch per colour under a CUDA graph.  Beams never interact, so
a seeded sample of them is recomputed one by one by the oracle with the same
colouring; tolerance 1e-5 of each beam's bbox diagonal."""
import numpy as np
import pytest

from paper_2403_06321_b300 import synth, vbd
from gpu_util import bbox_diag, oracle_run, params_of

pytestmark = pytest.mark.gpu


def test_batch_of_4096_beams_sampled(orc):
    from paper_2403_06321_b300.build import build
    build()
    meshes, cfg = synth.beam_batch(4096)
    cat, voff, toff = synth.concat(meshes)
    colors = np.concatenate([synth.kuhn_coloring(m.grid_ijk) for m in meshes])
    pd = params_of(cfg)
    # the library's default launch, and the compact slots at 4 lanes x 128
    # threads that the autotuner picks for this batch (the launch the bench times)
    runs = {}
    for name, launch in (("default", None), ("compact slots, 4 x 128", (4, 128, 5))):
        sim = vbd.Sim(cat, vbd.make_params(**pd), colors=colors, vert_offset=voff, tet_offset=toff)
        try:
            assert vbd.vbd_get_info(sim.ctx).n_meshes == 4096
            if launch:
                vbd.vbd_set_launch(sim.ctx, *launch)
            sim.set_state(cat.rest, np.zeros_like(cat.rest))
            for _ in range(cfg.steps):
                sim.step(cfg.h, cfg.iters)
            sim.sync_status()
            runs[name] = sim.get_state()[0].cpu().numpy().astype(np.float64)
        finally:
            sim.close()
    rng = np.random.default_rng(91)
    worst = dict.fromkeys(runs, 0.0)
    for b in rng.choice(len(meshes), 6, replace=False):
        m = meshes[b]
        xo, _ = oracle_run(orc, m, pd, synth.kuhn_coloring(m.grid_ijk), cfg.h, cfg.iters, cfg.steps)
        assert np.abs(xo - m.rest).max() > 1e-5  # the beam moved
        for name, xg in runs.items():
            err = float(np.abs(xg[voff[b]:voff[b + 1]] - xo).max()) / bbox_diag(m.rest)
            worst[name] = max(worst[name], err)
    for name, w in worst.items():
        print("4096-beam batch, %s: worst sampled err / bbox = %.3e" % (name, w))
        assert w <= 1e-5, name
