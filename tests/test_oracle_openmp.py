"""The OpenMP build of the oracle (liboracle_omp.so, used only to time the
multi-core CPU baseline) solves the vertices of one colour on several
threads.  Sec. 3.9 makes that order-free (same-colour vertices share no
force element; with self-contacts the pass reads a pass-start copy), so
its results must equal the serial build's bit for bit.  CPU only."""
import os
import subprocess
import sys
import tempfile
import textwrap

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RUN = textwrap.dedent(r'''
    import sys
    import numpy as np
    sys.path.insert(0, sys.argv[1])
    from oracle import oracle as orc
    from paper_2403_06321_b300 import synth
    out = {}
    # ground contact (k_c 1e5), Chebyshev, adaptive init, Kuhn colouring
    m, _ = synth.large_cube(8, drop_height=0.002)
    p = orc.Params.make(ground_on=True, k_c=1e5, cheby_rho=0.9)
    model = orc.Model.from_mesh(m)
    x, v = m.rest.copy(), np.zeros_like(m.rest)
    v[:, 2] = -0.4
    vp = v.copy()
    for _ in range(4):
        model.step(p, synth.kuhn_coloring(m.grid_ijk), 4, 1 / 60, 15, x, v, vp)
    out["cube_x"], out["cube_v"] = x, v
    # self-collision pairs (x^new + copy-back passes), greedy colouring
    m, cfg, _ = synth.colliding_slabs(n=6, layers=2, seed=5)
    p = orc.Params.make(gravity=cfg.gravity, k_c=cfg.k_c, self_collision=True, dcd_radius=cfg.dcd_radius)
    model = orc.Model.from_mesh(m)
    colors, nc = orc.color_greedy(m.n_verts, m.tets)
    x, v = m.rest.copy(), np.zeros_like(m.rest)
    vp = v.copy()
    for _ in range(2):
        model.step(p, colors, nc, cfg.h, 8, x, v, vp)
    out["slab_x"] = x
    # block Jacobi
    m = synth.beam(5, 2, 2, jitter_frac=0.05, seed=3)
    p = orc.Params.make(jacobi=True)
    model = orc.Model.from_mesh(m)
    x, v = m.rest.copy(), np.zeros_like(m.rest)
    vp = v.copy()
    for _ in range(3):
        model.step(p, synth.kuhn_coloring(m.grid_ijk), 4, 1 / 60, 10, x, v, vp)
    out["jacobi_x"] = x
    np.savez(sys.argv[2], **out)
''')


def _run(lib, threads, path):
    env = dict(os.environ, VBD_ORACLE_LIB=lib, OMP_NUM_THREADS=str(threads))
    subprocess.run([sys.executable, "-c", _RUN, ROOT, path], check=True, env=env, timeout=600)
    return np.load(path)


def test_openmp_build_equals_serial_build_bit_for_bit():
    from oracle import oracle
    serial = oracle.build()
    omp = oracle.build(openmp=True)
    with tempfile.TemporaryDirectory() as d:
        a = _run(serial, 1, os.path.join(d, "serial.npz"))
        b = _run(omp, 4, os.path.join(d, "omp.npz"))
        for k in a.files:
            assert np.array_equal(a[k], b[k]), k
        assert np.abs(a["cube_v"]).max() > 0.1  # the runs did something
