"""Host-side checks of the C-ABI library that need no GPU: it loads, it
exports every entry point include/vbd.h declares, and its host logic
(mesh validation, colouring, workspace sizing) behaves as documented."""
import os
import re

import numpy as np
import pytest

from paper_2403_06321_b300 import synth, vbd
from paper_2403_06321_b300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return vbd.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "vbd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vbd_[a-z_]+)\s*\(", src)))


def test_every_declared_entry_point_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(vbd.ENTRY_POINTS) == names


def _create(m, **kw):
    arr = vbd.MeshArrays(m.rest, m.tets, m.young, m.poisson, m.density, m.pinned)
    return vbd.vbd_create_mesh(arr.desc(), vbd.make_params(**kw))


def test_create_rejects_bad_meshes(lib):
    m = synth.beam(2, 1, 1)
    bad = synth.beam(2, 1, 1)
    bad.tets = bad.tets.copy()
    bad.tets[3, 2] = m.n_verts  # out of range
    with pytest.raises(vbd.VbdError) as e:
        _create(bad)
    assert e.value.status == "VBD_ERR_BAD_MESH"
    deg = synth.beam(2, 1, 1)
    deg.rest = deg.rest.copy()
    t = deg.tets[0]
    deg.rest[t[3]] = deg.rest[t[0]] + 0.5 * (deg.rest[t[1]] - deg.rest[t[0]])  # collinear -> flat tet
    with pytest.raises(vbd.VbdError) as e:
        _create(deg)
    assert e.value.status == "VBD_ERR_BAD_MESH"
    mat = synth.beam(2, 1, 1, nu=0.5)
    with pytest.raises(vbd.VbdError) as e:
        _create(mat)
    assert e.value.status == "VBD_ERR_BAD_MESH"
    with pytest.raises(vbd.VbdError) as e:
        _create(m, cheby_rho=1.5)
    assert e.value.status == "VBD_ERR_INVALID_ARG"


def test_colouring_matches_oracle_greedy_and_validates(lib, orc):
    for dims in [(10, 3, 3), (5, 4, 3)]:
        m = synth.beam(*dims)
        ctx = _create(m)
        try:
            nc = vbd.vbd_color(ctx, None)
            ours = vbd.vbd_get_colors(ctx, m.n_verts)
            ref, nref = orc.color_greedy(m.n_verts, m.tets)
            assert nc == nref
            assert np.array_equal(ours, ref)
            assert orc.color_valid(m.n_verts, m.tets, ours)
            # the Kuhn closed-form colouring is accepted as given
            kc = synth.kuhn_coloring(m.grid_ijk)
            assert vbd.vbd_color(ctx, kc) == 4
            assert np.array_equal(vbd.vbd_get_colors(ctx, m.n_verts), kc)
            bad = kc.copy()
            bad[m.tets[7, 0]] = bad[m.tets[7, 1]]
            with pytest.raises(vbd.VbdError) as e:
                vbd.vbd_color(ctx, bad)
            assert e.value.status == "VBD_ERR_BAD_COLORING"
        finally:
            vbd.vbd_destroy(ctx)


def test_info_workspace_and_call_order(lib):
    m = synth.cantilever_beam()[0]
    ctx = _create(m)
    try:
        with pytest.raises(vbd.VbdError) as e:
            vbd.vbd_workspace_size(ctx)
        assert e.value.status == "VBD_ERR_NOT_COLORED"
        vbd.vbd_color(ctx, synth.kuhn_coloring(m.grid_ijk))
        info = vbd.vbd_get_info(ctx)
        assert (info.n_verts, info.n_tets, info.n_colors) == (176, 540, 4)
        assert info.n_free == 176 - 16
        # every (free vertex, tet) incidence is one slot
        assert info.n_slots == int(sum((m.tets == i).sum() for i in np.nonzero(m.pinned == 0)[0]))
        size = vbd.vbd_workspace_size(ctx)
        assert size % 256 == 0 and size > 56 * info.n_slots
        # a host pointer is not a workspace; stepping before binding is refused
        buf = np.zeros(size // 4 + 64, np.float32)
        with pytest.raises(vbd.VbdError) as e:
            vbd.vbd_bind(ctx, buf.ctypes.data, size, 0)
        assert e.value.status == "VBD_ERR_WORKSPACE"
        with pytest.raises(vbd.VbdError) as e:
            vbd.vbd_step(ctx, 1 / 60, 5)
        assert e.value.status == "VBD_ERR_WORKSPACE"
        with pytest.raises(vbd.VbdError) as e:
            vbd.vbd_set_launch(ctx, 3, 0, 0)
        assert e.value.status == "VBD_ERR_INVALID_ARG"
    finally:
        vbd.vbd_destroy(ctx)


def test_batched_union_rejects_cross_mesh_tets(lib):
    ms = [synth.beam(2, 1, 1), synth.beam(3, 1, 1)]
    cat, voff, toff = synth.concat(ms)
    arr = vbd.MeshArrays(cat.rest, cat.tets, cat.young, cat.poisson, cat.density, cat.pinned, voff, toff)
    ctx = vbd.vbd_create_mesh(arr.desc(), vbd.make_params())
    assert vbd.vbd_get_info(ctx).n_meshes == 2
    vbd.vbd_destroy(ctx)
    tets = cat.tets.copy()
    tets[0, 0] = voff[1]  # a tet of mesh 0 that reaches into mesh 1
    arr = vbd.MeshArrays(cat.rest, tets, cat.young, cat.poisson, cat.density, cat.pinned, voff, toff)
    with pytest.raises(vbd.VbdError) as e:
        vbd.vbd_create_mesh(arr.desc(), vbd.make_params())
    assert e.value.status in ("VBD_ERR_BAD_MESH",)


def test_surface_matches_oracle_and_self_collision_params(lib, orc):
    """The library's boundary triangles (host preprocessing) equal the
    oracle's, orientation and order included; the self-collision options are
    validated and enlarge the workspace."""
    lower = synth.beam(3, 3, 1, edge=0.1, pin_face="z-", jitter_frac=0.05, seed=102)
    upper = synth.beam(2, 2, 1, edge=0.1, pin_face=None, jitter_frac=0.05, seed=103, origin=(0.05, 0.05, 0.09))
    cat, voff, toff = synth.concat([lower, upper])
    arr = vbd.MeshArrays(cat.rest, cat.tets, cat.young, cat.poisson, cat.density, cat.pinned, voff, toff)
    ctx = vbd.vbd_create_mesh(arr.desc(), vbd.make_params())
    try:
        vbd.vbd_color(ctx, None)
        size0 = vbd.vbd_workspace_size(ctx)
        tris = vbd.vbd_get_surface(ctx)
        assert np.array_equal(tris, orc.Model.from_mesh(cat).tris())
        info = vbd.vbd_get_info(ctx)
        assert info.n_surface_tris == len(tris)
        assert info.n_surface_verts == len(np.unique(tris))
        for bad in (dict(self_collision=True, dcd_radius=0.0), dict(self_collision=True, line_search=True)):
            with pytest.raises(vbd.VbdError) as e:
                vbd.vbd_set_params(ctx, vbd.make_params(**bad))
            assert e.value.status == "VBD_ERR_INVALID_ARG"
        vbd.vbd_set_params(ctx, vbd.make_params(self_collision=True, dcd_radius=0.02))
        assert vbd.vbd_workspace_size(ctx) > size0
    finally:
        vbd.vbd_destroy(ctx)


def test_wall_params_are_validated(lib):
    """World-box walls: at most six, each with a non-zero finite normal and a
    finite offset; the Python helper refuses malformed tuples."""
    m = synth.beam(2, 1, 1, edge=0.1)
    arr = vbd.MeshArrays(m.rest, m.tets, m.young, m.poisson, m.density, m.pinned)
    ctx = vbd.vbd_create_mesh(arr.desc(), vbd.make_params(walls=synth.world_box((-1, -1, 0), (1, 1, 2))))
    try:
        box = vbd.make_params(walls=synth.world_box((-1, -1, 0), (1, 1, 2)))
        assert box.n_walls == 6 and list(box.walls[1]) == [-1.0, 0.0, 0.0, -1.0]
        for k in (0, 3, 5):
            bad = vbd.make_params(walls=synth.world_box((-1, -1, 0), (1, 1, 2)))
            bad.walls[k][0] = bad.walls[k][1] = bad.walls[k][2] = 0.0
            with pytest.raises(vbd.VbdError) as e:
                vbd.vbd_set_params(ctx, bad)
            assert e.value.status == "VBD_ERR_INVALID_ARG"
        bad = vbd.make_params(walls=[(0, 0, 1, float("nan"))])
        with pytest.raises(vbd.VbdError):
            vbd.vbd_set_params(ctx, bad)
        bad = vbd.make_params()
        bad.n_walls = 7
        with pytest.raises(vbd.VbdError):
            vbd.vbd_set_params(ctx, bad)
        with pytest.raises(ValueError):
            vbd.make_params(walls=[(0, 0, 1)])
        with pytest.raises(ValueError):
            vbd.make_params(walls=[(0, 0, 1, 0)] * 7)
        vbd.vbd_set_params(ctx, vbd.make_params(walls=[(0, 0, 1, 0)], ground_on=True))
    finally:
        vbd.vbd_destroy(ctx)


def test_subspace_constraints_are_validated(lib):
    """Subspace constraints (Sec. 3.4): caller ids in range, not pinned, once
    each, dimension 1 or 2, a non-zero finite direction; they enlarge the
    workspace."""
    m = synth.beam(3, 2, 2, edge=0.1)
    arr = vbd.MeshArrays(m.rest, m.tets, m.young, m.poisson, m.density, m.pinned)
    ctx = vbd.vbd_create_mesh(arr.desc(), vbd.make_params())
    try:
        pinned = int(np.nonzero(m.pinned)[0][0])
        free = np.nonzero(m.pinned == 0)[0][:3]
        for vertex, dim, d in (([-1], [1], [(1, 0, 0)]), ([pinned], [2], [(1, 0, 0)]),
                               ([free[0], free[0]], [1, 1], [(1, 0, 0)] * 2), ([free[0]], [0], [(1, 0, 0)]),
                               ([free[0]], [1], [(0, 0, 0)]), ([free[0]], [2], [(np.inf, 1, 0)])):
            with pytest.raises(vbd.VbdError) as e:
                vbd.vbd_set_subspaces(ctx, vertex, dim, d)
            assert e.value.status == "VBD_ERR_INVALID_ARG"
        with pytest.raises(ValueError):
            vbd.vbd_set_subspaces(ctx, [free[0]], [1, 2], [(1, 0, 0)])
        vbd.vbd_color(ctx, None)
        size0 = vbd.vbd_workspace_size(ctx)
        vbd.vbd_set_subspaces(ctx, free, [1, 2, 1], [(1, 0, 0), (0, 0, 2), (0.3, 0.4, 0)])
        assert vbd.vbd_workspace_size(ctx) > size0
        vbd.vbd_set_subspaces(ctx, [], [], np.zeros((0, 3)))
        assert vbd.vbd_workspace_size(ctx) == size0
    finally:
        vbd.vbd_destroy(ctx)


def test_unknown_parameter_keywords_are_rejected(lib):
    """A misspelt option must fail on both sides instead of running the
    default on both (which would let a parity test pass without testing it)."""
    from oracle import oracle
    with pytest.raises(TypeError):
        vbd.make_params(cheby_roh=0.9)
    with pytest.raises(TypeError):
        oracle.Params.make(cheby_roh=0.9)
    assert vbd.make_params(cheby_rho=0.9).cheby_rho == pytest.approx(0.9)
    assert oracle.Params.make(cheby_rho=0.9).cheby_rho == pytest.approx(0.9)
