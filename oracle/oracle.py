"""Python face of the serial FP64 CPU oracle (vbd_oracle.c) for Vertex Block Descent.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product package.  It shares no
code with the CUDA path; both are fed the same seeded inputs.

Besides marshalling, this file holds the two dense FP64 references that need
a linear-algebra library primitive:
  * ``newton_solve``: the global implicit-Euler minimiser of Eqs. 1-2 by a dense
    Newton method with backtracking (VBD iterations converge to the
    implicit-Euler solution, Sec. 1 and Sec. 3.1);
  * ``dense_adjoint``: reverse-mode derivative of converged implicit-Euler
    steps (implicit function theorem on dG/dx = 0 of Eq. 2; the paper has
    no adjoint, this is derived from Eqs. 2, 3 and 6).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vbd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, no fast-math).  openmp=True
    builds liboracle_omp.so from the same source with -fopenmp: the vertices
    of one colour are then solved on several threads (the timed multi-core
    baseline; same results bit for bit).  Load it by naming it in
    VBD_ORACLE_LIB before the first call of lib()."""
    out = _LIB_OMP if openmp else _LIB
    hdr = os.path.join(_HERE, "vbd_oracle.h")
    stale = (not os.path.exists(out) or
             os.path.getmtime(out) < max(os.path.getmtime(_SRC), os.path.getmtime(hdr)))
    if force or stale:
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off"] + (["-fopenmp"] if openmp else []) +
                              ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class Params(C.Structure):
    _fields_ = [("gravity", C.c_double * 3), ("ground_on", C.c_int), ("ground_height", C.c_double),
                ("ground_normal", C.c_double * 3), ("k_c", C.c_double), ("cheby_rho", C.c_double),
                ("init_mode", C.c_int), ("det_eps", C.c_double), ("k_d", C.c_double),
                ("mu_c", C.c_double), ("eps_v", C.c_double), ("line_search", C.c_int), ("jacobi", C.c_int),
                ("self_collision", C.c_int), ("dcd_radius", C.c_double), ("ccd_interval", C.c_int),
                ("ccd_edges", C.c_int),
                ("n_walls", C.c_int), ("walls", C.c_double * 24)]

    @classmethod
    def make(cls, gravity=(0.0, 0.0, -9.8), ground_on=False, ground_height=0.0,
             ground_normal=(0.0, 0.0, 1.0), k_c=0.0, cheby_rho=0.0, init_mode=3,
             det_eps=1e-12, k_d=0.0, mu_c=0.0, eps_v=1e-3, line_search=False, jacobi=False,
             self_collision=False, dcd_radius=0.0, walls=(), ccd_interval=0,
             ccd_edges=False) -> "Params":
        """Parameters from keywords; an unknown keyword raises TypeError.
        walls: up to 6 world-box half-spaces (nx, ny, nz, offset), the allowed
        side being x.n/|n| >= offset (Sec. 3.4)."""
        p = cls()
        p.gravity[:] = [float(g) for g in gravity]
        p.ground_on = int(bool(ground_on))
        p.ground_height = float(ground_height)
        p.ground_normal[:] = [float(g) for g in ground_normal]
        p.k_c = float(k_c)
        p.cheby_rho = float(cheby_rho)
        p.init_mode = int(init_mode)
        p.det_eps = float(det_eps)
        p.k_d = float(k_d)
        p.mu_c = float(mu_c)
        p.eps_v = float(eps_v)
        p.line_search = int(bool(line_search))
        p.jacobi = int(bool(jacobi))
        p.self_collision = int(bool(self_collision))
        p.dcd_radius = float(dcd_radius)
        p.ccd_interval = int(ccd_interval)
        p.ccd_edges = int(bool(ccd_edges))
        walls = [tuple(float(v) for v in w) for w in walls]
        if len(walls) > 6 or any(len(w) != 4 for w in walls):
            raise ValueError("walls: at most 6 tuples (nx, ny, nz, offset)")
        p.n_walls = len(walls)
        for k, w in enumerate(walls):
            p.walls[4 * k:4 * k + 4] = list(w)
        return p


class Stats(C.Structure):
    _fields_ = [("vertex_solves", C.c_longlong), ("det_skips", C.c_longlong), ("contacts", C.c_longlong)]


def lib():
    """The oracle library; VBD_ORACLE_LIB names another build of vbd_oracle.c
    (used only by the planted-mistake tests, which compile mutated copies)."""
    global _lib
    if _lib is None:
        L = C.CDLL(os.environ.get("VBD_ORACLE_LIB") or build())
        vp = C.c_void_p
        sig = {
            "orc_lame": (None, [C.c_double, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "orc_rest_tet": (C.c_int, [_dp, _dp, C.POINTER(C.c_double)]),
            "orc_tet_F": (None, [_dp, _dp, _dp]),
            "orc_nh_psi": (C.c_double, [_dp, C.c_double, C.c_double]),
            "orc_nh_pk1": (None, [_dp, C.c_double, C.c_double, _dp]),
            "orc_cofactor": (None, [_dp, _dp]),
            "orc_tet_energy": (C.c_double, [_dp, _dp, C.c_double, C.c_double, C.c_double]),
            "orc_tet_grad": (None, [_dp, _dp, C.c_double, C.c_double, C.c_double, _dp]),
            "orc_tet_hess_block": (None, [_dp, _dp, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, _dp]),
            "orc_tet_hess": (None, [_dp, _dp, C.c_double, C.c_double, C.c_double, _dp]),
            "orc_color_greedy": (C.c_int, [C.c_int, C.c_int, _ip, _ip]),
            "orc_color_valid": (C.c_int, [C.c_int, C.c_int, _ip, _ip]),
            "orc_model_new": (vp, [C.c_int, C.c_int, _dp, _ip, _dp, _dp, _dp, _up, C.POINTER(C.c_int)]),
            "orc_model_free": (None, [vp]),
            "orc_model_mass": (None, [vp, _dp]),
            "orc_model_tet_data": (None, [vp, _dp, _dp, _dp, _dp]),
            "orc_model_set_log_young": (None, [vp, _dp]),
            "orc_model_set_subspace": (C.c_int, [vp, C.c_int, C.c_int, _dp]),
            "orc_inertia_target": (None, [vp, C.POINTER(Params), C.c_double, _dp, _dp, _dp]),
            "orc_initial_guess": (None, [vp, C.POINTER(Params), C.c_double, _dp, _dp, _dp, _dp]),
            "orc_ground_friction": (None, [C.POINTER(Params), C.c_double, _dp, _dp, C.c_double, _dp, _dp]),
            "orc_vertex_solve": (C.c_int, [vp, C.POINTER(Params), C.c_double, C.c_int, _dp, _dp, _dp, _dp,
                                           C.POINTER(C.c_int)]),
            "orc_sweep_color": (None, [vp, C.POINTER(Params), C.c_double, _ip, C.c_int, _dp, _dp, _dp, _up,
                                       C.POINTER(Stats)]),
            "orc_cheby_omega": (C.c_double, [C.c_int, C.c_double, C.c_double]),
            "orc_local_energy": (C.c_double, [vp, C.POINTER(Params), C.c_double, C.c_int, _dp, _dp]),
            "orc_model_n_tris": (C.c_int, [vp]),
            "orc_model_tris": (None, [vp, _ip]),
            "orc_closest_point_tri": (None, [_dp, _dp, _dp, _dp, _dp, _dp]),
            "orc_point_in_tet": (C.c_int, [_dp, _ip, _dp]),
            "orc_ccd_vertex": (C.c_int, [vp, _dp, _dp, C.c_int, C.POINTER(C.c_double), _dp]),
            "orc_ccd": (C.c_int, [vp, _dp, _dp]),
            "orc_ccd_edges": (None, [vp, _dp, _dp]),
            "orc_ee_first_hit": (C.c_int, [vp, _dp, _dp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "orc_cubic_first_root": (C.c_double, [_dp, C.c_double]),
            "orc_model_contact_weights": (None, [vp, _dp, _up]),
            "orc_ee_impact": (C.c_double, [_dp, _dp, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                           C.POINTER(C.c_double)]),
            "orc_model_n_edges": (C.c_int, [vp]),
            "orc_model_edges": (None, [vp, _ip]),
            "orc_model_ee_pairs": (C.c_int, [vp, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
            "orc_dcd_vertex": (C.c_int, [vp, C.POINTER(Params), _dp, C.c_int]),
            "orc_dcd": (None, [vp, C.POINTER(Params), _dp]),
            "orc_model_contacts": (None, [vp, _ip]),
            "orc_self_contact": (C.c_int, [vp, C.POINTER(Params), C.c_double, C.c_int, _dp, C.c_void_p, _dp,
                                            _dp]),
            "orc_step": (C.c_int, [vp, C.POINTER(Params), _ip, C.c_int, C.c_double, C.c_int, _dp, _dp, _dp,
                                   C.POINTER(Stats)]),
            "orc_energy_G": (C.c_double, [vp, C.POINTER(Params), C.c_double, _dp, _dp]),
            "orc_elastic_grad": (None, [vp, _dp, _dp]),
            "orc_elastic_hess_triplets": (None, [vp, _dp, _ip, _ip, _dp]),
            "orc_tet_grads": (None, [vp, _dp, _dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _d(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


# ---------------------------------------------------------------- element --

def lame(E: float, nu: float) -> tuple[float, float]:
    mu, lam = C.c_double(), C.c_double()
    lib().orc_lame(E, nu, C.byref(mu), C.byref(lam))
    return mu.value, lam.value


def rest_tet(X: np.ndarray) -> tuple[np.ndarray, float]:
    B = np.zeros(9)
    V = C.c_double()
    if lib().orc_rest_tet(_d(X, 12), B, C.byref(V)):
        raise ValueError("degenerate rest tet")
    return B.reshape(3, 3), V.value


def tet_F(x, B) -> np.ndarray:
    F = np.zeros(9)
    lib().orc_tet_F(_d(x, 12), _d(B, 9), F)
    return F.reshape(3, 3)


def psi(F, mu, lam) -> float:
    return lib().orc_nh_psi(_d(F, 9), mu, lam)


def pk1(F, mu, lam) -> np.ndarray:
    P = np.zeros(9)
    lib().orc_nh_pk1(_d(F, 9), mu, lam, P)
    return P.reshape(3, 3)


def cofactor(F) -> np.ndarray:
    Cm = np.zeros(9)
    lib().orc_cofactor(_d(F, 9), Cm)
    return Cm.reshape(3, 3)


def tet_energy(x, B, V, mu, lam) -> float:
    return lib().orc_tet_energy(_d(x, 12), _d(B, 9), V, mu, lam)


def tet_grad(x, B, V, mu, lam) -> np.ndarray:
    g = np.zeros(12)
    lib().orc_tet_grad(_d(x, 12), _d(B, 9), V, mu, lam, g)
    return g.reshape(4, 3)


def tet_hess(x, B, V, mu, lam) -> np.ndarray:
    H = np.zeros(144)
    lib().orc_tet_hess(_d(x, 12), _d(B, 9), V, mu, lam, H)
    return H.reshape(12, 12)


def tet_hess_block(x, B, V, mu, lam, k, l) -> np.ndarray:
    H = np.zeros(9)
    lib().orc_tet_hess_block(_d(x, 12), _d(B, 9), V, mu, lam, k, l, H)
    return H.reshape(3, 3)


def ee_impact(x0, x1, p0, p1, q0, q1):
    """(time of impact or -1, s, u) of edges (p0, p1), (q0, q1) moving linearly."""
    s, u = C.c_double(-1.0), C.c_double(-1.0)
    t = lib().orc_ee_impact(_d(x0).reshape(-1), _d(x1).reshape(-1), int(p0), int(p1), int(q0), int(q1),
                            C.byref(s), C.byref(u))
    return float(t), float(s.value), float(u.value)


def cubic_first_root(c, t_min=0.0) -> float:
    """Earliest root in [t_min, 1] of c0 + c1 t + c2 t^2 + c3 t^3, or -1."""
    return float(lib().orc_cubic_first_root(_d(c, 4), float(t_min)))


def ground_friction(p: "Params", h: float, xi, xti, lambda_n: float):
    """(force, approximate Hessian) of the ground friction term for one vertex."""
    f, H = np.zeros(3), np.zeros(9)
    lib().orc_ground_friction(C.byref(p), h, _d(xi, 3), _d(xti, 3), lambda_n, f, H)
    return f, H.reshape(3, 3)


def closest_point_tri(p, a, b, c):
    """(closest point, barycentric weights) of triangle abc to point p."""
    q, w = np.zeros(3), np.zeros(3)
    lib().orc_closest_point_tri(_d(p, 3), _d(a, 3), _d(b, 3), _d(c, 3), q, w)
    return q, w


def point_in_tet(x, tet, q) -> bool:
    """Whether q lies in the closed tet x[tet] (barycentric coordinates >= 0)."""
    return bool(lib().orc_point_in_tet(_d(x).reshape(-1), np.ascontiguousarray(tet, np.int32), _d(q, 3)))


def cheby_omega(n: int, rho: float, omega_prev: float) -> float:
    return lib().orc_cheby_omega(n, rho, omega_prev)


# --------------------------------------------------------------- colouring --

def color_greedy(n_verts: int, tets: np.ndarray) -> tuple[np.ndarray, int]:
    t = np.ascontiguousarray(tets, dtype=np.int32)
    colors = np.zeros(n_verts, np.int32)
    nc = lib().orc_color_greedy(n_verts, t.shape[0], t.reshape(-1), colors)
    if nc < 0:
        raise ValueError("bad tet index")
    return colors, nc


def color_valid(n_verts: int, tets: np.ndarray, colors: np.ndarray) -> bool:
    t = np.ascontiguousarray(tets, dtype=np.int32)
    return bool(lib().orc_color_valid(n_verts, t.shape[0], t.reshape(-1),
                                      np.ascontiguousarray(colors, dtype=np.int32)))


# ------------------------------------------------------------------- model --

class Model:
    """One (or a union of independent) tet mesh(es) with FP64 rest data."""

    def __init__(self, rest, tets, young, poisson, density, pinned):
        self.n = int(np.asarray(rest).shape[0])
        self.t = int(np.asarray(tets).shape[0])
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)
        self.pinned = np.ascontiguousarray(pinned, dtype=np.uint8)
        status = C.c_int()
        self._h = lib().orc_model_new(self.n, self.t, _d(rest).reshape(-1), self.tets.reshape(-1),
                                      _d(young), _d(poisson), _d(density), self.pinned, C.byref(status))
        if not self._h:
            raise ValueError("oracle model rejected mesh (status %d)" % status.value)
        self.poisson = _d(poisson).copy()
        self.sub_dim = np.full(self.n, 3, np.int32)
        self.sub_dir = np.zeros((self.n, 3))

    @classmethod
    def from_mesh(cls, m) -> "Model":
        model = cls(m.rest, m.tets, m.young, m.poisson, m.density, m.pinned)
        sub_dim = getattr(m, "sub_dim", None)
        if sub_dim is not None:
            for i in np.nonzero(np.asarray(sub_dim) < 3)[0]:
                model.set_subspace(int(i), int(sub_dim[i]), m.sub_dir[i])
        return model

    def set_subspace(self, i: int, L: int, direction) -> None:
        """Sec. 3.4 subspace constraint: L = 1 line (direction), 2 plane (normal), 3 none."""
        if lib().orc_model_set_subspace(self._h, int(i), int(L), _d(direction, 3)) != 0:
            raise ValueError("bad subspace constraint for vertex %d" % i)
        self.sub_dim[i] = int(L)
        self.sub_dir[i] = np.asarray(direction, np.float64)

    def reduced_basis(self) -> np.ndarray:
        """(3N, k) orthonormal basis of the admissible displacements: the
        three axes of every free vertex, the line direction or two in-plane
        axes of a subspace-constrained one (from an SVD, independently of the
        basis the local solve uses), nothing for a pinned vertex."""
        cols = []
        for i in range(self.n):
            if self.pinned[i]:
                continue
            L = int(self.sub_dim[i])
            if L == 3:
                Q = np.eye(3)
            else:
                d = self.sub_dir[i] / np.linalg.norm(self.sub_dir[i])
                Q = d[:, None] if L == 1 else np.linalg.svd(d[None, :])[2][1:].T
            for c in range(Q.shape[1]):
                col = np.zeros(3 * self.n)
                col[3 * i:3 * i + 3] = Q[:, c]
                cols.append(col)
        return np.array(cols).T

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_model_free(h)
            self._h = None

    @property
    def free(self) -> np.ndarray:
        return self.pinned == 0

    def mass(self) -> np.ndarray:
        m = np.zeros(self.n)
        lib().orc_model_mass(self._h, m)
        return m

    def tet_data(self):
        B, V, mu, lam = np.zeros(9 * self.t), np.zeros(self.t), np.zeros(self.t), np.zeros(self.t)
        lib().orc_model_tet_data(self._h, B, V, mu, lam)
        return B.reshape(-1, 3, 3), V, mu, lam

    def set_log_young(self, log_young) -> None:
        lib().orc_model_set_log_young(self._h, _d(log_young))

    # -- Algorithm 1 pieces
    def inertia_target(self, p: Params, h, xt, vt) -> np.ndarray:
        y = np.zeros(3 * self.n)
        lib().orc_inertia_target(self._h, C.byref(p), h, _d(xt).reshape(-1), _d(vt).reshape(-1), y)
        return y.reshape(-1, 3)

    def initial_guess(self, p: Params, h, xt, vt, vprev) -> np.ndarray:
        x = np.zeros(3 * self.n)
        lib().orc_initial_guess(self._h, C.byref(p), h, _d(xt).reshape(-1), _d(vt).reshape(-1),
                                _d(vprev).reshape(-1), x)
        return x.reshape(-1, 3)

    def vertex_solve(self, p: Params, h, i, x, y, xt) -> tuple[np.ndarray, int, int]:
        dx = np.zeros(3)
        contact = C.c_int()
        skipped = lib().orc_vertex_solve(self._h, C.byref(p), h, int(i), _d(x).reshape(-1), _d(y).reshape(-1),
                                         _d(xt).reshape(-1), dx, C.byref(contact))
        return dx, skipped, contact.value

    def sweep_color(self, p: Params, h, colors, color, x, y, xt, colliding=None) -> Stats:
        st = Stats()
        if colliding is None:
            colliding = np.zeros(self.n, np.uint8)
        xx = _d(x).reshape(-1)
        lib().orc_sweep_color(self._h, C.byref(p), h, np.ascontiguousarray(colors, np.int32), int(color),
                              xx, _d(y).reshape(-1), _d(xt).reshape(-1), colliding, C.byref(st))
        x[...] = xx.reshape(x.shape)
        return st

    def step(self, p: Params, colors, n_colors, h, iters, x, v, vprev) -> Stats:
        """In place: (x, v, vprev) = (x^t, v^t, v^{t-1}) -> (x^{t+1}, v^{t+1}, v^t)."""
        st = Stats()
        for a in (x, v, vprev):
            assert a.dtype == np.float64 and a.flags.c_contiguous
        lib().orc_step(self._h, C.byref(p), np.ascontiguousarray(colors, np.int32), int(n_colors), h,
                       int(iters), x.reshape(-1), v.reshape(-1), vprev.reshape(-1), C.byref(st))
        return st

    def tris(self) -> np.ndarray:
        """Boundary triangles (outward at rest), (F, 3)."""
        t = np.zeros(3 * lib().orc_model_n_tris(self._h), np.int32)
        lib().orc_model_tris(self._h, t)
        return t.reshape(-1, 3)

    def dcd(self, p: Params, x) -> np.ndarray:
        """Runs the DCD at positions x and returns the per-vertex contact triangle (-1 = none)."""
        lib().orc_dcd(self._h, C.byref(p), _d(x).reshape(-1))
        return self.contacts()

    def dcd_vertex(self, p: Params, x, a) -> int:
        """The DCD pair of vertex a alone at positions x (triangle index or -1)."""
        return int(lib().orc_dcd_vertex(self._h, C.byref(p), _d(x).reshape(-1), int(a)))

    def self_contact(self, p: Params, i, x, h=1.0 / 60.0, xt=None):
        """(force, Hessian, hit) of the self-contact terms acting on vertex i;
        with xt (positions at the step start) and mu_c > 0, friction too."""
        f, H = np.zeros(3), np.zeros(9)
        xt_arr = None if xt is None else _d(xt).reshape(-1)
        hit = lib().orc_self_contact(self._h, C.byref(p), float(h), int(i), _d(x).reshape(-1),
                                     None if xt_arr is None else xt_arr.ctypes.data, f, H)
        return f, H.reshape(3, 3), bool(hit)

    def contacts(self) -> np.ndarray:
        c = np.zeros(self.n, np.int32)
        lib().orc_model_contacts(self._h, c)
        return c

    def contact_weights(self):
        """(impact weights (N, 3), CCD flag (N,)) of the current pairs."""
        w = np.zeros(3 * self.n)
        f = np.zeros(self.n, np.uint8)
        lib().orc_model_contact_weights(self._h, w, f)
        return w.reshape(-1, 3), f.astype(bool)

    def ccd_vertex(self, x0, x1, a):
        """(triangle or -1, time of impact, weights) of vertex a's CCD (Sec. 3.5)."""
        toi = C.c_double(-1.0)
        w = np.zeros(3)
        T = lib().orc_ccd_vertex(self._h, _d(x0).reshape(-1), _d(x1).reshape(-1), int(a), C.byref(toi), w)
        return int(T), float(toi.value), w

    def ee_first_hit(self, x0, x1, e):
        """(partner edge or -1, s, u): the edge-edge CCD's search for edge e
        alone (Sec. 3.5), before the pairing rules."""
        s, u = C.c_double(-1.0), C.c_double(-1.0)
        f = lib().orc_ee_first_hit(self._h, _d(x0).reshape(-1), _d(x1).reshape(-1), int(e), C.byref(s),
                                   C.byref(u))
        return int(f), float(s.value), float(u.value)

    def edges(self) -> np.ndarray:
        e = np.zeros(2 * lib().orc_model_n_edges(self._h), np.int32)
        lib().orc_model_edges(self._h, e)
        return e.reshape(-1, 2)

    def ee_pairs(self):
        """Edge-edge pairs, by holding edge: (partner per edge (-1 = none),
        carried flag, (s, u) per edge, normal per edge)."""
        ne = lib().orc_model_n_edges(self._h)
        partner = np.zeros(ne, np.int32)
        carried = np.zeros(ne, np.uint8)
        su = np.zeros(2 * ne)
        n = np.zeros(3 * ne)
        lib().orc_model_ee_pairs(self._h, partner.ctypes.data, carried.ctypes.data, su.ctypes.data, n.ctypes.data)
        return partner, carried.astype(bool), su.reshape(-1, 2), n.reshape(-1, 3)

    def ee_pair_list(self):
        """[(v0, v1, v2, v3), (s, u), normal] for each current edge-edge pair."""
        partner, _, su, n = self.ee_pairs()
        e = self.edges()
        return [((*e[k], *e[partner[k]]), su[k], n[k]) for k in np.nonzero(partner >= 0)[0]]

    def ccd(self, x0, x1, edges=True) -> int:
        """CCD of every vertex without a step-start pair (and, with edges, of
        the boundary edges); returns the vertex-triangle pair count."""
        n = int(lib().orc_ccd(self._h, _d(x0).reshape(-1), _d(x1).reshape(-1)))
        if edges:
            lib().orc_ccd_edges(self._h, _d(x0).reshape(-1), _d(x1).reshape(-1))
        return n

    def local_energy(self, p: Params, h, i, x, y) -> float:
        return lib().orc_local_energy(self._h, C.byref(p), h, int(i), _d(x).reshape(-1), _d(y).reshape(-1))

    def energy_G(self, p: Params, h, x, y) -> float:
        return lib().orc_energy_G(self._h, C.byref(p), h, _d(x).reshape(-1), _d(y).reshape(-1))

    def elastic_grad(self, x) -> np.ndarray:
        g = np.zeros(3 * self.n)
        lib().orc_elastic_grad(self._h, _d(x).reshape(-1), g)
        return g

    def elastic_hess(self, x, sparse: bool = False):
        """3N x 3N elastic Hessian: dense (small meshes) or scipy CSR."""
        nt = 144 * self.t
        r, c, v = np.zeros(nt, np.int32), np.zeros(nt, np.int32), np.zeros(nt)
        lib().orc_elastic_hess_triplets(self._h, _d(x).reshape(-1), r, c, v)
        if sparse:
            import scipy.sparse as sp
            return sp.csr_matrix((v, (r, c)), shape=(3 * self.n, 3 * self.n))
        H = np.zeros((3 * self.n, 3 * self.n))
        np.add.at(H, (r, c), v)
        return H

    def tet_grads(self, x) -> np.ndarray:
        g = np.zeros(12 * self.t)
        lib().orc_tet_grads(self._h, _d(x).reshape(-1), g)
        return g.reshape(self.t, 4, 3)

    # -- dense global references (small meshes only)
    def _plane_terms(self, p: Params, x):
        """[(unit normal n, depths d, active mask)] of every static half-space
        (the ground, then the walls; Sec. 3.4, Eq. 12)."""
        planes = []
        if p.ground_on:
            planes.append((np.array(p.ground_normal[:], dtype=np.float64), p.ground_height))
        for k in range(p.n_walls):
            planes.append((np.array(p.walls[4 * k:4 * k + 3], dtype=np.float64), p.walls[4 * k + 3]))
        out = []
        for n, c in planes:
            n = n / np.linalg.norm(n)
            d = c - x @ n
            out.append((n, d, (d > 0) & self.free))
        return out

    def global_grad_hess(self, p: Params, h, x, y):
        """dG/dx and d2G/dx2 of Eq. 2 (+ ground penalty), dense, all DoFs."""
        m = self.mass()
        M = np.repeat(np.where(self.free, m, 0.0), 3)
        g = M / h ** 2 * (x - y).reshape(-1) + self.elastic_grad(x)
        H = self.elastic_hess(x) + np.diag(M / h ** 2)
        for n, d, act in self._plane_terms(p, x):
            for i in np.nonzero(act)[0]:
                g[3 * i:3 * i + 3] -= p.k_c * d[i] * n
                H[3 * i:3 * i + 3, 3 * i:3 * i + 3] += p.k_c * np.outer(n, n)
        return g, H

    def newton_solve(self, p: Params, h, x0, y, tol=1e-11, max_iter=200) -> np.ndarray:
        """Global minimiser of G (Eqs. 1-2) over the admissible displacements
        from x0 (free DoFs, restricted to their subspaces where constrained,
        Sec. 3.4): dense Newton in the coordinates of reduced_basis() with
        backtracking on G.  Used as the backward-Euler reference."""
        x = np.array(x0, dtype=np.float64).reshape(-1, 3)
        Bm = self.reduced_basis()
        if Bm.size == 0:
            return x
        scale = None
        for _ in range(max_iter):
            g, H = self.global_grad_hess(p, h, x, y)
            gz = Bm.T @ g
            if scale is None:
                scale = max(np.abs(gz).max(), 1e-300)
            if np.abs(gz).max() <= tol * scale:
                break
            Hz = Bm.T @ H @ Bm
            try:
                dz = -np.linalg.solve(Hz, gz)
            except np.linalg.LinAlgError:
                dz = -gz
            if dz @ gz > 0:
                dz = -gz
            dx = Bm @ dz
            G0 = self.energy_G(p, h, x, y)
            a = 1.0
            while a > 1e-12:
                xn = x + a * dx.reshape(-1, 3)
                if self.energy_G(p, h, xn, y) <= G0 + 1e-4 * a * (g @ dx):
                    break
                a *= 0.5
            x = xn
        return x


def dense_adjoint(model: Model, p: Params, h: float, xs: list, dL_dxT: np.ndarray, sparse=None):
    """Reverse-mode gradients of L(x_T) through T converged implicit-Euler steps.

    xs = [x_0, ..., x_T] (positions after each step).  At a converged step
    dG/dx(x_{t+1}; x_t, v_t, theta) = 0 on free DoFs, so with
    H = M/h^2 + d2E/dx2 (+ contact):
        r = xbar_{t+1} + vbar_{t+1}/h,   H lam = r,
        xbar_t += M/h^2 lam - vbar_{t+1}/h,   vbar_t = M/h lam,
        thetabar_j -= sum_{i in tet j} lam_i . dE_j/dx_i   (theta_j = log E_j).
    Returns (dL/dlogE per tet, dL/dv_0 (N,3), dL/dx_0 (N,3)).  The linear
    solve is dense LU for small meshes and a sparse direct solve (scipy) for
    larger ones (sparse=None picks by size).

    With subspace constraints (Sec. 3.4) a step solves for x_{t+1} = x_t + B z
    (B = reduced_basis()) with B^T dG/dx = 0, so lam = B (B^T H B)^-1 B^T r,
    and since x_{t+1} follows x_t across the constrained directions,
    xbar_t gains r - H lam (zero on the unconstrained free DoFs).
    """
    n = model.n
    fd = np.repeat(model.free, 3)
    m = np.repeat(model.mass(), 3)
    xbar = np.asarray(dL_dxT, np.float64).reshape(-1).copy()
    xbar[~fd] = 0.0
    vbar = np.zeros(3 * n)
    theta_bar = np.zeros(model.t)
    T = len(xs) - 1
    if sparse is None:
        sparse = n > 400
    Bm = model.reduced_basis() if (model.sub_dim < 3).any() else None
    for t in range(T - 1, -1, -1):
        x1 = np.asarray(xs[t + 1], np.float64).reshape(-1, 3)
        planes = model._plane_terms(p, x1)
        diag = m / h ** 2
        r = xbar + vbar / h
        lam = np.zeros(3 * n)
        resid = np.zeros(3 * n)
        if Bm is not None:
            Hd = model.elastic_hess(x1) + np.diag(diag)
            for nrm, d, act in planes:
                for i in np.nonzero(act)[0]:
                    Hd[3 * i:3 * i + 3, 3 * i:3 * i + 3] += p.k_c * np.outer(nrm, nrm)
            lam = Bm @ np.linalg.solve(Bm.T @ Hd @ Bm, Bm.T @ r)
            resid = r - Hd @ lam
        elif sparse:
            import scipy.sparse as sp
            import scipy.sparse.linalg as spla
            H = model.elastic_hess(x1, sparse=True) + sp.diags(diag)
            rows, cols, vals = [], [], []
            for nrm, d, act in planes:
                for i in np.nonzero(act)[0]:
                    for a_ in range(3):
                        for b_ in range(3):
                            rows.append(3 * i + a_); cols.append(3 * i + b_)
                            vals.append(p.k_c * nrm[a_] * nrm[b_])
            if rows:
                H = H + sp.csr_matrix((vals, (rows, cols)), shape=H.shape)
            idx = np.nonzero(fd)[0]
            lam[fd] = spla.spsolve(H[idx][:, idx].tocsc(), r[fd])
        else:
            H = model.elastic_hess(x1) + np.diag(diag)
            for nrm, d, act in planes:
                for i in np.nonzero(act)[0]:
                    H[3 * i:3 * i + 3, 3 * i:3 * i + 3] += p.k_c * np.outer(nrm, nrm)
            lam[fd] = np.linalg.solve(H[np.ix_(fd, fd)], r[fd])
        tg = model.tet_grads(x1)  # (T, 4, 3)
        lam3 = lam.reshape(-1, 3)
        theta_bar -= np.einsum("tkr,tkr->t", tg, lam3[model.tets])
        xbar_new = m / h ** 2 * lam - vbar / h + resid
        vbar = m / h * lam
        xbar = xbar_new
        xbar[~fd] = 0.0
        vbar[~fd] = 0.0
    return theta_bar, vbar.reshape(-1, 3), xbar.reshape(-1, 3)


def run(model: Model, p: Params, colors, n_colors, h, iters, steps, x0, v0,
        vprev0: Optional[np.ndarray] = None, record: bool = False):
    """Run `steps` VBD steps from (x0, v0); v^{-1} defaults to v0."""
    x = np.array(x0, np.float64).reshape(-1, 3).copy()
    v = np.array(v0, np.float64).reshape(-1, 3).copy()
    vp = (v.copy() if vprev0 is None else np.array(vprev0, np.float64).reshape(-1, 3).copy())
    traj = [x.copy()] if record else None
    for _ in range(steps):
        model.step(p, colors, n_colors, h, iters, x, v, vp)
        if record:
            traj.append(x.copy())
    return (x, v, vp, traj) if record else (x, v, vp)
