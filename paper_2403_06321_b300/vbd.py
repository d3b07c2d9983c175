"""Thin Python binding of the C ABI in include/vbd.h (argument marshalling only).

Every function here has the name of the C entry point it wraps and raises
VbdError when that entry point returns a status other than VBD_OK.  All
arithmetic runs in libvbd.so; there is no fallback: if the library is
missing, loading fails loudly.  PyTorch supplies device memory and streams
(see ``Sim``); pointers may be torch tensors, numpy arrays or ints.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvbd.so")

STATUS = {0: "VBD_OK", 1: "VBD_ERR_INVALID_ARG", 2: "VBD_ERR_BAD_MESH", 3: "VBD_ERR_BAD_COLORING",
          4: "VBD_ERR_NOT_COLORED", 5: "VBD_ERR_WORKSPACE", 6: "VBD_ERR_CUDA", 7: "VBD_ERR_NONFINITE",
          8: "VBD_ERR_NO_TAPE", 9: "VBD_ERR_STATE", 10: "VBD_ERR_TIMEOUT", 11: "VBD_ERR_RANGE"}
STATUS_CODE = {v: k for k, v in STATUS.items()}

# every entry point declared in include/vbd.h
ENTRY_POINTS = [
    "vbd_default_params", "vbd_create_mesh", "vbd_color", "vbd_get_colors", "vbd_get_info",
    "vbd_get_surface", "vbd_workspace_size", "vbd_bind", "vbd_set_params", "vbd_set_subspaces", "vbd_set_state",
    "vbd_get_state",
    "vbd_set_log_young", "vbd_step", "vbd_begin_step", "vbd_iterate", "vbd_sweep_color",
    "vbd_accelerate", "vbd_end_step", "vbd_energy", "vbd_energy_static", "vbd_get_contacts", "vbd_get_edge_pairs",
    "vbd_sync_status",
    "vbd_backward", "vbd_adjoint_residuals", "vbd_gradient_norm",
    "vbd_set_launch", "vbd_debug_stall_pipeline", "vbd_set_graph", "vbd_autotune", "vbd_autotune_ex",
    "vbd_last_error",
    "vbd_destroy",
]


class VbdError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__("%s failed: %s (%s)" % (fn, STATUS.get(code, code), msg))
        self.fn, self.code, self.msg = fn, code, msg

    @property
    def status(self) -> str:
        return STATUS.get(self.code, str(self.code))


class vbd_mesh_desc(C.Structure):
    _fields_ = [("n_meshes", C.c_int32), ("vert_offset", C.c_void_p), ("tet_offset", C.c_void_p),
                ("n_verts", C.c_int32), ("n_tets", C.c_int32), ("rest_pos", C.c_void_p),
                ("tets", C.c_void_p), ("young", C.c_void_p), ("poisson", C.c_void_p),
                ("density", C.c_void_p), ("pinned", C.c_void_p)]


class vbd_params(C.Structure):
    _fields_ = [("gravity", C.c_float * 3), ("ground_on", C.c_int32), ("ground_height", C.c_float),
                ("ground_normal", C.c_float * 3), ("k_c", C.c_float), ("cheby_rho", C.c_float),
                ("init_mode", C.c_int32), ("det_eps", C.c_float), ("k_d", C.c_float),
                ("tape_steps", C.c_int32), ("mu_c", C.c_float), ("eps_v", C.c_float),
                ("line_search", C.c_int32), ("jacobi", C.c_int32), ("self_collision", C.c_int32),
                ("dcd_radius", C.c_float), ("scatter_sweep", C.c_int32), ("xnew_copy_back", C.c_int32),
                ("n_walls", C.c_int32), ("walls", (C.c_float * 4) * 6), ("ccd_interval", C.c_int32),
                ("ccd_edges", C.c_int32), ("warp_rows", C.c_int32)]


class vbd_info(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tets", C.c_int32), ("n_meshes", C.c_int32),
                ("n_free", C.c_int32), ("n_colors", C.c_int32), ("n_slots", C.c_int64),
                ("lanes_per_vertex", C.c_int32), ("block_threads", C.c_int32), ("pipeline", C.c_int32),
                ("pipe_stage_slots", C.c_int32), ("pipe_ctas_per_sm", C.c_int32), ("use_graph", C.c_int32),
                ("n_surface_tris", C.c_int32), ("n_surface_verts", C.c_int32)]


_lib = None


def load() -> C.CDLL:
    """Loads the in-tree libvbd.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libvbd.so is missing: the CUDA extension has not been built "
                           "(python -m paper_2403_06321_b300.build)")
    L = C.CDLL(LIB_PATH)
    P, I32, F, D = C.c_void_p, C.c_int32, C.c_float, C.c_double
    sig = {
        "vbd_default_params": (None, [C.POINTER(vbd_params)]),
        "vbd_set_subspaces": (C.c_int, [P, I32, P, P, P]),
        "vbd_get_edge_pairs": (C.c_int, [P, C.POINTER(I32), P, P]),
        "vbd_create_mesh": (C.c_int, [C.POINTER(vbd_mesh_desc), C.POINTER(vbd_params), C.POINTER(P)]),
        "vbd_color": (C.c_int, [P, P, C.POINTER(I32)]),
        "vbd_get_colors": (C.c_int, [P, P]),
        "vbd_get_info": (C.c_int, [P, C.POINTER(vbd_info)]),
        "vbd_get_surface": (C.c_int, [P, C.POINTER(I32), P]),
        "vbd_workspace_size": (C.c_int, [P, C.POINTER(C.c_size_t)]),
        "vbd_bind": (C.c_int, [P, P, C.c_size_t, P]),
        "vbd_set_params": (C.c_int, [P, C.POINTER(vbd_params)]),
        "vbd_set_state": (C.c_int, [P, P, P, P]),
        "vbd_get_state": (C.c_int, [P, P, P]),
        "vbd_set_log_young": (C.c_int, [P, P]),
        "vbd_step": (C.c_int, [P, F, I32]),
        "vbd_begin_step": (C.c_int, [P, F]),
        "vbd_iterate": (C.c_int, [P, I32]),
        "vbd_sweep_color": (C.c_int, [P, I32]),
        "vbd_accelerate": (C.c_int, [P, I32]),
        "vbd_end_step": (C.c_int, [P]),
        "vbd_energy": (C.c_int, [P, C.POINTER(D)]),
        "vbd_energy_static": (C.c_int, [P, P]),
        "vbd_get_contacts": (C.c_int, [P, P]),
        "vbd_sync_status": (C.c_int, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "vbd_backward": (C.c_int, [P, P, P, P, I32]),
        "vbd_adjoint_residuals": (C.c_int, [P, P, I32]),
        "vbd_gradient_norm": (C.c_int, [P, C.POINTER(D), C.POINTER(D)]),
        "vbd_set_launch": (C.c_int, [P, I32, I32, I32]),
        "vbd_debug_stall_pipeline": (C.c_int, [P, I32]),
        "vbd_set_graph": (C.c_int, [P, I32]),
        "vbd_autotune": (C.c_int, [P, F, I32, C.POINTER(F)]),
        "vbd_autotune_ex": (C.c_int, [P, F, I32, I32, C.POINTER(F)]),
        "vbd_last_error": (C.c_char_p, [P]),
        "vbd_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(a) -> Optional[int]:
    """Address of a torch tensor, numpy array, int or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    raise TypeError("cannot take the address of %r" % type(a))


def _check(fn: str, ctx, code: int) -> None:
    if code != 0:
        msg = load().vbd_last_error(ctx).decode() if ctx else ""
        raise VbdError(fn, code, msg)


# ---------------------------------------------------------------- entry points

def vbd_default_params() -> vbd_params:
    p = vbd_params()
    load().vbd_default_params(C.byref(p))
    return p


def vbd_create_mesh(desc: vbd_mesh_desc, params: vbd_params) -> int:
    out = C.c_void_p()
    _check("vbd_create_mesh", None, load().vbd_create_mesh(C.byref(desc), C.byref(params), C.byref(out)))
    return out.value


def vbd_color(ctx: int, colors=None) -> int:
    nc = C.c_int32()
    c = None if colors is None else np.ascontiguousarray(colors, dtype=np.int32)
    _check("vbd_color", ctx, load().vbd_color(ctx, _ptr(c), C.byref(nc)))
    return nc.value


def vbd_get_colors(ctx: int, n_verts: int) -> np.ndarray:
    out = np.zeros(n_verts, np.int32)
    _check("vbd_get_colors", ctx, load().vbd_get_colors(ctx, _ptr(out)))
    return out


def vbd_get_info(ctx: int) -> vbd_info:
    info = vbd_info()
    _check("vbd_get_info", ctx, load().vbd_get_info(ctx, C.byref(info)))
    return info


def vbd_get_surface(ctx: int) -> np.ndarray:
    """Boundary triangles (n, 3) in caller vertex ids."""
    n = C.c_int32()
    _check("vbd_get_surface", ctx, load().vbd_get_surface(ctx, C.byref(n), None))
    out = np.zeros((n.value, 3), np.int32)
    _check("vbd_get_surface", ctx, load().vbd_get_surface(ctx, C.byref(n), _ptr(out)))
    return out


def vbd_workspace_size(ctx: int) -> int:
    n = C.c_size_t()
    _check("vbd_workspace_size", ctx, load().vbd_workspace_size(ctx, C.byref(n)))
    return n.value


def vbd_bind(ctx: int, workspace, nbytes: int, stream: int) -> None:
    _check("vbd_bind", ctx, load().vbd_bind(ctx, _ptr(workspace), nbytes, stream))


def vbd_set_params(ctx: int, params: vbd_params) -> None:
    _check("vbd_set_params", ctx, load().vbd_set_params(ctx, C.byref(params)))


def vbd_set_subspaces(ctx: int, vertex, dim, direction) -> None:
    """Subspace constraints (Sec. 3.4): vertex ids (caller order), dim 1 (line)
    or 2 (plane), direction (n, 3): line direction or plane normal."""
    vertex = np.ascontiguousarray(vertex, dtype=np.int32).reshape(-1)
    dim = np.ascontiguousarray(dim, dtype=np.int32).reshape(-1)
    direction = np.ascontiguousarray(direction, dtype=np.float32).reshape(-1)
    if not (len(dim) == len(vertex) and len(direction) == 3 * len(vertex)):
        raise ValueError("vertex, dim and direction must describe the same constraints")
    _check("vbd_set_subspaces", ctx, load().vbd_set_subspaces(
        ctx, len(vertex), vertex.ctypes.data if len(vertex) else None, dim.ctypes.data if len(vertex) else None,
        direction.ctypes.data if len(vertex) else None))


def vbd_get_edge_pairs(ctx: int, with_partners: bool = True):
    """(edges (E, 2) caller ids, partner per edge or None) of the edge-edge CCD pairs."""
    n = C.c_int32(0)
    _check("vbd_get_edge_pairs", ctx, load().vbd_get_edge_pairs(ctx, C.byref(n), None, None))
    edges = np.zeros(2 * n.value, np.int32)
    partner = np.zeros(n.value, np.int32) if with_partners else None
    _check("vbd_get_edge_pairs", ctx, load().vbd_get_edge_pairs(
        ctx, C.byref(n), edges.ctypes.data if n.value else None,
        partner.ctypes.data if (with_partners and n.value) else None))
    return edges.reshape(-1, 2), partner


def vbd_set_state(ctx: int, x, v, v_prev=None) -> None:
    _check("vbd_set_state", ctx, load().vbd_set_state(ctx, _ptr(x), _ptr(v), _ptr(v_prev)))


def vbd_get_state(ctx: int, x=None, v=None) -> None:
    _check("vbd_get_state", ctx, load().vbd_get_state(ctx, _ptr(x), _ptr(v)))


def vbd_set_log_young(ctx: int, log_young) -> None:
    _check("vbd_set_log_young", ctx, load().vbd_set_log_young(ctx, _ptr(log_young)))


def vbd_step(ctx: int, h: float, iters: int) -> None:
    _check("vbd_step", ctx, load().vbd_step(ctx, h, iters))


def vbd_begin_step(ctx: int, h: float) -> None:
    _check("vbd_begin_step", ctx, load().vbd_begin_step(ctx, h))


def vbd_iterate(ctx: int, iters: int) -> None:
    _check("vbd_iterate", ctx, load().vbd_iterate(ctx, iters))


def vbd_sweep_color(ctx: int, color: int) -> None:
    _check("vbd_sweep_color", ctx, load().vbd_sweep_color(ctx, color))


def vbd_accelerate(ctx: int, n: int) -> None:
    _check("vbd_accelerate", ctx, load().vbd_accelerate(ctx, n))


def vbd_end_step(ctx: int) -> None:
    _check("vbd_end_step", ctx, load().vbd_end_step(ctx))


def vbd_energy(ctx: int) -> float:
    g = C.c_double()
    _check("vbd_energy", ctx, load().vbd_energy(ctx, C.byref(g)))
    return g.value


def vbd_energy_static(ctx: int, G_out) -> None:
    """G_out: device buffer of one float64 (e.g. a torch tensor); asynchronous."""
    _check("vbd_energy_static", ctx, load().vbd_energy_static(ctx, _ptr(G_out)))


def vbd_get_contacts(ctx: int, n_verts: int) -> np.ndarray:
    out = np.zeros(n_verts, np.int32)
    _check("vbd_get_contacts", ctx, load().vbd_get_contacts(ctx, _ptr(out)))
    return out


def vbd_sync_status(ctx: int, with_contacts: bool = False):
    """Singular-Hessian skips since the last call; with_contacts=True also
    returns the self-collision pairs detected since the last call."""
    skips, contacts = C.c_int64(), C.c_int64()
    _check("vbd_sync_status", ctx, load().vbd_sync_status(ctx, C.byref(skips), C.byref(contacts)))
    return (skips.value, contacts.value) if with_contacts else skips.value


def vbd_backward(ctx: int, dL_dxT, dL_dlogE, dL_dv0, adj_iters: int) -> None:
    _check("vbd_backward", ctx, load().vbd_backward(ctx, _ptr(dL_dxT), _ptr(dL_dlogE), _ptr(dL_dv0), adj_iters))


def vbd_adjoint_residuals(ctx: int, n_steps: int) -> np.ndarray:
    """max |r - H lam| / max |r| of each recorded step after the last vbd_backward."""
    out = np.zeros(max(n_steps, 1), np.float64)
    _check("vbd_adjoint_residuals", ctx, load().vbd_adjoint_residuals(ctx, out.ctypes.data, len(out)))
    return out[:n_steps]


def vbd_gradient_norm(ctx: int):
    """(max_i |dG/dx_i| at the current iterate, max_i m_i |a_ext|) in newtons."""
    g, w = C.c_double(), C.c_double()
    _check("vbd_gradient_norm", ctx, load().vbd_gradient_norm(ctx, C.byref(g), C.byref(w)))
    return g.value, w.value


def vbd_set_launch(ctx: int, lanes_per_vertex: int = 0, block_threads: int = 0, variant: int = -1) -> None:
    """variant: 0 plain, 1 TMA-staged, 2 persistent, 3 two-phase scatter, 4 fused loop,
    5 compact slots, 6 compact slots in packed pairs, 7 warp rows (< 0 keeps it)."""
    _check("vbd_set_launch", ctx, load().vbd_set_launch(ctx, lanes_per_vertex, block_threads, variant))


def vbd_debug_stall_pipeline(ctx: int, enable: bool) -> None:
    _check("vbd_debug_stall_pipeline", ctx, load().vbd_debug_stall_pipeline(ctx, 1 if enable else 0))


def vbd_set_graph(ctx: int, enable: bool) -> None:
    _check("vbd_set_graph", ctx, load().vbd_set_graph(ctx, 1 if enable else 0))


def vbd_autotune(ctx: int, h: float, iters: int) -> float:
    ms = C.c_float()
    _check("vbd_autotune", ctx, load().vbd_autotune(ctx, h, iters, C.byref(ms)))
    return ms.value


VBD_TUNE_SAME_ARITHMETIC = 1


def vbd_autotune_ex(ctx: int, h: float, iters: int, flags: int = 0) -> float:
    ms = C.c_float()
    _check("vbd_autotune_ex", ctx, load().vbd_autotune_ex(ctx, h, iters, flags, C.byref(ms)))
    return ms.value


def vbd_last_error(ctx: int) -> str:
    return load().vbd_last_error(ctx).decode()


def vbd_destroy(ctx: int) -> None:
    if ctx:
        load().vbd_destroy(ctx)


# ------------------------------------------------------------------ helpers

def make_params(gravity=(0.0, 0.0, -9.8), ground_on=False, ground_height=0.0, ground_normal=(0.0, 0.0, 1.0),
                k_c=1e7, cheby_rho=0.0, init_mode=3, det_eps=1e-12, k_d=0.0, tape_steps=0, mu_c=0.0,
                eps_v=1e-3, line_search=False, jacobi=False, self_collision=False, dcd_radius=0.01,
                scatter_sweep=False, xnew_copy_back=False, walls=(), ccd_interval=0,
                ccd_edges=False, warp_rows=False) -> vbd_params:
    """vbd_params from keywords (an unknown keyword raises TypeError, so a
    misspelt option cannot silently run the default).  walls: up to 6
    world-box half-spaces (nx, ny, nz, offset), the allowed side being
    x.n/|n| >= offset."""
    p = vbd_default_params()
    p.gravity[:] = [float(g) for g in gravity]
    p.ground_on = int(bool(ground_on))
    p.ground_height = float(ground_height)
    p.ground_normal[:] = [float(g) for g in ground_normal]
    p.k_c = float(k_c)
    p.cheby_rho = float(cheby_rho)
    p.init_mode = int(init_mode)
    p.det_eps = float(det_eps)
    p.k_d = float(k_d)
    p.tape_steps = int(tape_steps)
    p.mu_c = float(mu_c)
    p.eps_v = float(eps_v)
    p.line_search = int(bool(line_search))
    p.jacobi = int(bool(jacobi))
    p.self_collision = int(bool(self_collision))
    p.dcd_radius = float(dcd_radius)
    p.scatter_sweep = int(bool(scatter_sweep))
    p.xnew_copy_back = int(bool(xnew_copy_back))
    p.ccd_interval = int(ccd_interval)
    p.ccd_edges = int(bool(ccd_edges))
    p.warp_rows = int(bool(warp_rows))
    walls = [tuple(float(v) for v in w) for w in walls]
    if len(walls) > 6 or any(len(w) != 4 for w in walls):
        raise ValueError("walls: at most 6 tuples (nx, ny, nz, offset)")
    p.n_walls = len(walls)
    for k, w in enumerate(walls):
        p.walls[k][:] = list(w)
    return p


class MeshArrays:
    """Host arrays of a mesh in the dtypes of vbd_mesh_desc, kept alive for the call."""

    def __init__(self, rest, tets, young, poisson, density, pinned=None, vert_offset=None, tet_offset=None):
        self.rest = np.ascontiguousarray(rest, dtype=np.float64).reshape(-1, 3)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
        self.young = np.ascontiguousarray(young, dtype=np.float32)
        self.poisson = np.ascontiguousarray(poisson, dtype=np.float32)
        self.density = np.ascontiguousarray(density, dtype=np.float32)
        self.pinned = None if pinned is None else np.ascontiguousarray(pinned, dtype=np.uint8)
        self.vert_offset = None if vert_offset is None else np.ascontiguousarray(vert_offset, dtype=np.int32)
        self.tet_offset = None if tet_offset is None else np.ascontiguousarray(tet_offset, dtype=np.int32)

    def desc(self) -> vbd_mesh_desc:
        d = vbd_mesh_desc()
        d.n_meshes = 1 if self.vert_offset is None else len(self.vert_offset) - 1
        d.vert_offset = _ptr(self.vert_offset)
        d.tet_offset = _ptr(self.tet_offset)
        d.n_verts = self.rest.shape[0]
        d.n_tets = self.tets.shape[0]
        d.rest_pos = _ptr(self.rest)
        d.tets = _ptr(self.tets)
        d.young = _ptr(self.young)
        d.poisson = _ptr(self.poisson)
        d.density = _ptr(self.density)
        d.pinned = _ptr(self.pinned)
        return d


class Sim:
    """A bound context: torch supplies the workspace and the stream."""

    def __init__(self, mesh, params: vbd_params, colors=None, stream=None, device="cuda",
                 vert_offset=None, tet_offset=None):
        import torch
        self.torch = torch
        arrs = MeshArrays(mesh.rest, mesh.tets, mesh.young, mesh.poisson, mesh.density, mesh.pinned,
                          vert_offset, tet_offset)
        self.n_verts = arrs.rest.shape[0]
        self.n_tets = arrs.tets.shape[0]
        self.tape_steps = int(params.tape_steps)
        self.ctx = vbd_create_mesh(arrs.desc(), params)
        try:
            sub_dim = getattr(mesh, "sub_dim", None)
            if sub_dim is not None:
                k = np.nonzero(np.asarray(sub_dim) < 3)[0]
                vbd_set_subspaces(self.ctx, k, np.asarray(sub_dim)[k], np.asarray(mesh.sub_dir)[k])
            self.n_colors = vbd_color(self.ctx, colors)
            self.ws_bytes = vbd_workspace_size(self.ctx)
            self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
            self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
            vbd_bind(self.ctx, self.workspace, self.ws_bytes, self.stream.cuda_stream)
        except Exception:
            vbd_destroy(self.ctx)
            self.ctx = None
            raise
        self.info = vbd_get_info(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            vbd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    def set_state(self, x, v, v_prev=None) -> None:
        keep = [self._as_f32(a) for a in (x, v, v_prev)]
        vbd_set_state(self.ctx, *keep)
        self.stream.synchronize()  # host sources must outlive the async copies

    def _as_f32(self, a):
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            return np.ascontiguousarray(a, dtype=np.float32).reshape(-1)
        return a.to(dtype=self.torch.float32).contiguous().reshape(-1)

    def get_state(self):
        torch = self.torch
        x = torch.empty(3 * self.n_verts, dtype=torch.float32, device=self.workspace.device)
        v = torch.empty_like(x)
        vbd_get_state(self.ctx, x, v)
        self.stream.synchronize()
        return x.view(-1, 3), v.view(-1, 3)

    def step(self, h: float, iters: int) -> None:
        vbd_step(self.ctx, h, iters)

    def energy(self) -> float:
        return vbd_energy(self.ctx)

    def sync_status(self) -> int:
        return vbd_sync_status(self.ctx)
