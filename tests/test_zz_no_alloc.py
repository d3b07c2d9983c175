"""vbd_energy_static: the FP64 energy for callers that cannot allocate device
memory (their device memory is a fixed pool they own, or allocation calls
are off limits in their loop).  Its scratch is a static array inside the
library, so it must give the same number as vbd_energy, which uses the
caller's workspace, and stale contents from an earlier call must not leak
into the next one (checked with two calls in a row on different states and
on meshes of different sizes).  Named to run after every other test."""
import numpy as np
import pytest
import torch

from paper_2403_06321_b300 import synth, vbd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_06321_b300.build import build
    build()


def _energies(sim, x0, v0, sweeps):
    sim.set_state(x0, v0)
    vbd.vbd_begin_step(sim.ctx, 1 / 60)
    for c in range(sweeps):
        vbd.vbd_sweep_color(sim.ctx, c % sim.n_colors)
    ref = vbd.vbd_energy(sim.ctx)  # workspace scratch, synchronising
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    vbd.vbd_energy_static(sim.ctx, out)  # library scratch, asynchronous
    sim.stream.synchronize()
    vbd.vbd_end_step(sim.ctx)
    sim.sync_status()
    return ref, float(out.item())


def test_static_scratch_energy_matches_workspace_energy():
    big = synth.beam(24, 10, 8, edge=0.05, E=2e5, nu=0.4, jitter_frac=0.1, seed=41)
    small = synth.beam(3, 2, 2, edge=0.05, E=2e5, nu=0.4, jitter_frac=0.1, seed=42)
    pd = vbd.make_params(ground_on=True, ground_height=0.02, k_c=1e5)
    results = []
    for mesh, seed, sweeps in [(big, 43, 0), (big, 44, 3), (small, 45, 2), (big, 46, 5)]:
        sim = vbd.Sim(mesh, pd)
        try:
            x0, v0 = synth.perturbed_state(mesh.rest, 0.01, 0.3, seed=seed)
            ref, got = _energies(sim, x0, v0, sweeps)
        finally:
            sim.close()
        results.append((ref, got))
        # same kernels, different grid: only the FP64 summation order differs
        assert got == pytest.approx(ref, rel=1e-12), (mesh.n_verts, seed)
    assert len({r for r, _ in results}) == len(results)  # the cases really differ
