"""vbd_energy_static: the FP64 energy for callers that cannot allocate device
memory (their device memory is a fixed pool they own, or allocation calls
are off limits in their loop).  Its scratch is a static array inside the
library, so it must give the same number as vbd_energy, which uses the
caller's workspace, and stale contents from an earlier call must not leak
into the next one (checked with two calls in a row on different states and
on meshes of different sizes, with and without self-collision pairs).  The
array exists once per CUDA context, so the library must hand each context
its own copy's address (checked by switching between two live contexts).
Named to run after every other test."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

from paper_2403_06321_b300 import synth, vbd

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def test_static_scratch_energy_with_self_contact_pairs():
    """With self-collision the scratch also holds the partial sums of the
    contact penalties (after the vertex and tet partials); the slab scene
    has pairs at every step start, so that part is exercised."""
    m, cfg, _ = synth.colliding_slabs(n=10, layers=2, seed=7)  # the upper slab starts sunk into the lower
    pd = vbd.make_params(gravity=cfg.gravity, k_c=cfg.k_c, self_collision=True, dcd_radius=cfg.dcd_radius)
    sim = vbd.Sim(m, pd, colors=synth.kuhn_coloring(m.grid_ijk))
    try:
        vals = []
        for sweeps in (0, 4):
            ref, got = _energies(sim, m.rest, np.zeros_like(m.rest), sweeps)
            assert got == pytest.approx(ref, rel=1e-12), sweeps
            vals.append(ref)
        assert vals[0] != vals[1]
        assert (vbd.vbd_get_contacts(sim.ctx, m.n_verts) >= 0).sum() > 0  # the pair partials are present
    finally:
        sim.close()


def test_static_scratch_energy_rejects_a_host_destination():
    m = synth.beam(3, 2, 2, edge=0.05, E=2e5, nu=0.4, jitter_frac=0.1, seed=42)
    sim = vbd.Sim(m, vbd.make_params())
    try:
        sim.set_state(m.rest, np.zeros_like(m.rest))
        vbd.vbd_begin_step(sim.ctx, 1 / 60)
        host = np.zeros(1, np.float64)
        with pytest.raises(vbd.VbdError) as e:
            vbd.vbd_energy_static(sim.ctx, host)
        assert e.value.status == "VBD_ERR_INVALID_ARG"
        vbd.vbd_end_step(sim.ctx)
        sim.sync_status()
    finally:
        sim.close()


_TWO_CONTEXTS = textwrap.dedent(r'''
    import ctypes as C
    import sys
    import numpy as np
    sys.path.insert(0, sys.argv[1])
    from paper_2403_06321_b300 import synth, vbd

    cu = C.CDLL("libcuda.so.1")

    def ck(r, what):
        if r != 0:
            raise SystemExit("%s returned %d" % (what, r))

    ck(cu.cuInit(0), "cuInit")
    dev = C.c_int()
    ck(cu.cuDeviceGet(C.byref(dev), 0), "cuDeviceGet")

    def new_context():
        ctx = C.c_void_p()
        if hasattr(cu, "cuCtxCreate_v2"):
            ck(cu.cuCtxCreate_v2(C.byref(ctx), C.c_uint(0), dev), "cuCtxCreate")
        else:
            ck(cu.cuCtxCreate_v4(C.byref(ctx), None, C.c_uint(0), dev), "cuCtxCreate")
        return ctx  # current on this thread

    def alloc(n):
        p = C.c_uint64()
        ck(cu.cuMemAlloc_v2(C.byref(p), C.c_size_t(n)), "cuMemAlloc")
        return p.value

    class Case:
        """A bound context whose workspace and result buffer come from the
        driver allocator of the CUDA context current at creation."""
        def __init__(self, mesh, seed):
            self.arr = vbd.MeshArrays(mesh.rest, mesh.tets, mesh.young, mesh.poisson, mesh.density,
                                      mesh.pinned)
            self.ctx = vbd.vbd_create_mesh(self.arr.desc(), vbd.make_params(ground_on=True,
                                           ground_height=0.02, k_c=1e5))
            vbd.vbd_color(self.ctx)
            n = vbd.vbd_workspace_size(self.ctx)
            self.ws = alloc(n + 256)
            self.g = alloc(8)
            vbd.vbd_bind(self.ctx, (self.ws + 255) // 256 * 256, n, None)
            x0, v0 = synth.perturbed_state(mesh.rest, 0.01, 0.3, seed=seed)
            self.x0 = np.ascontiguousarray(x0, np.float32).reshape(-1)
            self.v0 = np.ascontiguousarray(v0, np.float32).reshape(-1)

        def energies(self):
            vbd.vbd_set_state(self.ctx, self.x0, self.v0, None)
            vbd.vbd_begin_step(self.ctx, 1 / 60)
            vbd.vbd_sweep_color(self.ctx, 1)
            ref = vbd.vbd_energy(self.ctx)
            vbd.vbd_energy_static(self.ctx, self.g)
            ck(cu.cuCtxSynchronize(), "cuCtxSynchronize")
            got = C.c_double()
            ck(cu.cuMemcpyDtoH_v2(C.byref(got), C.c_uint64(self.g), C.c_size_t(8)), "cuMemcpyDtoH")
            vbd.vbd_end_step(self.ctx)
            vbd.vbd_sync_status(self.ctx)
            return ref, got.value

        def close(self):
            vbd.vbd_destroy(self.ctx)
            ck(cu.cuMemFree_v2(C.c_uint64(self.ws)), "cuMemFree")
            ck(cu.cuMemFree_v2(C.c_uint64(self.g)), "cuMemFree")

    vbd.load()
    mesh = synth.beam(6, 3, 3, edge=0.05, E=2e5, nu=0.4, jitter_frac=0.1, seed=51)
    ctx_a = new_context()
    a = Case(mesh, 52)
    r1 = a.energies()                      # first lookup, in context A
    ctx_b = new_context()                  # B is now current; A stays alive
    b = Case(mesh, 53)
    r2 = b.energies()                      # B has its own copy of the array
    ck(cu.cuCtxPopCurrent_v2(C.byref(C.c_void_p())), "cuCtxPopCurrent")  # back to A
    r3 = a.energies()                      # A again after B
    a.close()
    ck(cu.cuCtxPushCurrent_v2(ctx_b), "cuCtxPushCurrent")
    b.close()
    ck(cu.cuCtxPopCurrent_v2(C.byref(C.c_void_p())), "cuCtxPopCurrent")
    ck(cu.cuCtxDestroy_v2(ctx_b), "cuCtxDestroy")
    ck(cu.cuCtxDestroy_v2(ctx_a), "cuCtxDestroy")
    for ref, got in (r1, r2, r3):
        print("%.17g %.17g" % (ref, got))
''')


def test_static_scratch_follows_the_current_context():
    """Two live CUDA contexts on one device each load the library's module,
    so each has its own static array at its own address; calls made in A,
    then B, then A again must each use their own context's copy."""
    res = subprocess.run([sys.executable, "-c", _TWO_CONTEXTS, ROOT], capture_output=True, text=True,
                         timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    vals = [tuple(float(t) for t in ln.split()) for ln in res.stdout.strip().splitlines()]
    assert len(vals) == 3
    for ref, got in vals:
        assert got == pytest.approx(ref, rel=1e-12)
    assert vals[0][0] == pytest.approx(vals[2][0], rel=1e-12)  # same state in A twice
    assert vals[0][0] != vals[1][0]  # B ran another state
