"""ctypes front end of the FP64 C oracle (test infrastructure only).

Each wrapper names the C function it calls; the C source cites the passage of
the paper (arXiv 1210.1491) that each function restates.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


class OrGeom(C.Structure):
    _fields_ = [("kind", C.c_int), ("center", C.c_double * 3), ("radius", C.c_double),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("n_boxes", C.c_int),
                ("boxes", C.POINTER(C.c_double)), ("truncation", C.c_double)]


class OrData(C.Structure):
    _fields_ = [("kind", C.c_int), ("x0", C.c_double * 3), ("strength", C.c_double),
                ("lmax", C.c_int), ("clm", C.POINTER(C.c_double)), ("center", C.c_double * 3),
                ("scale", C.c_double), ("constant", C.c_double)]


class OrWosOpts(C.Structure):
    _fields_ = [("eps", C.c_double), ("seed", C.c_uint64), ("max_steps", C.c_uint64),
                ("stream", C.c_int), ("score", C.c_int)]


class OrPiece(C.Structure):
    _fields_ = [("ax", C.c_int), ("side", C.c_int), ("ua", C.c_int), ("va", C.c_int), ("fv", C.c_double),
                ("rlo", C.c_double * 2), ("rhi", C.c_double * 2), ("cf", C.c_double * 2), ("rf", C.c_double),
                ("P", C.c_double * 2), ("onlo", C.c_int * 2), ("onhi", C.c_int * 2), ("nsub", C.c_int),
                ("sub", C.c_double * 17), ("area", C.c_double)]


class OrPatch(C.Structure):
    _fields_ = [("kind", C.c_int), ("c", C.c_double * 3), ("n", C.c_double * 3),
                ("t1", C.c_double * 3), ("t2", C.c_double * 3), ("a", C.c_double),
                ("R", C.c_double), ("sc", C.c_double * 3), ("theta_max", C.c_double),
                ("umax", C.c_double), ("blo", C.c_double * 3), ("bhi", C.c_double * 3),
                ("npiece", C.c_int), ("piece", OrPiece * 6)]

    def pieces(self):
        """Wrapped patch: (face axis, side, area, sub-range cuts) of each piece."""
        return [(self.piece[k].ax, self.piece[k].side, self.piece[k].area,
                 list(self.piece[k].sub[: self.piece[k].nsub + 1])) for k in range(self.npiece)]


STREAM_F64 = 0   # one Philox call per jump, 53-bit uniforms
STREAM_F32 = 1   # one Philox call per three jumps, 21-bit uniforms


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.or_u01_21.argtypes = [C.c_uint32]
        L.or_u01_21.restype = C.c_double
        L.or_fields21.argtypes = [_u32p, _u32p]
        L.or_u01_53.argtypes = [C.c_uint32, C.c_uint32]
        L.or_u01_53.restype = C.c_double
        L.or_direction.argtypes = [C.c_double, C.c_double, C.c_int, _f64p]
        L.or_set_num_threads.argtypes = [C.c_int]
        L.or_set_sk_self_order.argtypes = [C.c_int]
        L.or_set_sk_self_order.restype = C.c_int
        L.or_gauss_legendre.argtypes = [C.c_int, _f64p, _f64p]
        L.or_distance.argtypes = [C.POINTER(OrGeom), _f64p, _f64p]
        L.or_distance.restype = C.c_double
        L.or_real_sh.argtypes = [C.c_int, _f64p, _f64p]
        L.or_dirichlet.argtypes = [C.POINTER(OrData), _f64p]
        L.or_dirichlet.restype = C.c_double
        L.or_neumann_exact.argtypes = [C.POINTER(OrData), _f64p, _f64p]
        L.or_neumann_exact.restype = C.c_double
        L.or_walk.argtypes = [C.POINTER(OrGeom), C.POINTER(OrData), _f64p, C.c_uint32,
                              C.c_uint32, C.c_uint32, C.POINTER(OrWosOpts),
                              C.POINTER(C.c_double), C.POINTER(C.c_uint64)]
        L.or_walk.restype = C.c_int
        L.or_wos_points.argtypes = [C.POINTER(OrGeom), C.POINTER(OrData), C.c_int64, _f64p,
                                    _u32p, _u32p, _i64p, C.POINTER(OrWosOpts), _f64p, _f64p,
                                    _u64p, _u64p]
        L.or_patch_frame.argtypes = [C.POINTER(OrGeom), _f64p, C.c_double, C.POINTER(OrPatch)]
        L.or_patch_frame.restype = C.c_int
        L.or_gamma_nodes.argtypes = [C.POINTER(OrPatch), C.c_int, C.c_int, _f64p, _f64p, _f64p]
        L.or_panels.argtypes = [C.POINTER(OrPatch), C.c_int, C.c_int, _f64p, _f64p, _f64p,
                                _f64p, _f64p]
        L.or_green.argtypes = [C.c_double, _f64p, _f64p]
        L.or_green.restype = C.c_double
        L.or_green_grad_y.argtypes = [C.c_double, _f64p, _f64p, _f64p]
        L.or_poisson.argtypes = [C.c_double, _f64p, _f64p]
        L.or_poisson.restype = C.c_double
        L.or_panel_integral.argtypes = [C.POINTER(OrPatch), C.POINTER(OrData), C.c_int, _f64p,
                                        _f64p, C.c_void_p, C.c_double]
        L.or_panel_integral.restype = C.c_double
        L.or_assemble.argtypes = [C.POINTER(OrPatch), C.POINTER(OrData), C.c_int, C.c_int,
                                  C.c_int, C.c_int, _f64p, C.c_double, _f64p, _f64p]
        L.or_lu_solve.argtypes = [C.c_int, _f64p, _f64p, _f64p]
        L.or_lu_solve.restype = C.c_int
        L.or_solve_patch.argtypes = [C.POINTER(OrGeom), C.POINTER(OrData), _f64p, C.c_double,
                                     C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_uint32,
                                     C.POINTER(OrWosOpts), C.c_void_p, C.c_double, _f64p, _f64p,
                                     _u64p, _f64p]
        L.or_solve_patch.restype = C.c_int
        L.or_potential.argtypes = [C.c_int64, _f64p, _f64p, _f64p, _f64p, _f64p, C.c_int64,
                                   _f64p, _f64p]
        L.or_potential_majorants.argtypes = [C.c_int64, _f64p, _f64p, _f64p, _f64p, C.c_int64, _f64p,
                                             _f64p, _f64p]
        L.or_owned.argtypes = [C.c_int64, _f64p, _i64p, C.c_int64, _f64p, _u8p]
        L.or_single_point.argtypes = [C.POINTER(OrGeom), C.POINTER(OrData), _f64p, C.c_double, C.c_int,
                                      C.c_int, C.c_double, C.c_int64, C.c_uint32, C.POINTER(OrWosOpts),
                                      C.c_void_p, _f64p, C.c_void_p]
        L.or_single_point.restype = C.c_int
        L.or_green_dnn.argtypes = [C.c_double, _f64p, _f64p, _f64p, _f64p]
        L.or_green_dnn.restype = C.c_double
        L.or_second_kind_flat.argtypes = [C.POINTER(OrPatch), C.POINTER(OrData), C.c_int, C.c_int, C.c_int,
                                          C.c_int, _f64p, C.c_int, _f64p]
        L.or_second_kind_flat.restype = C.c_int
        L.or_second_kind.argtypes = [C.POINTER(OrPatch), C.POINTER(OrData), C.c_int, C.c_int, C.c_int, C.c_int,
                                     _f64p, C.c_double, C.c_void_p, C.c_void_p, _f64p]
        L.or_second_kind.restype = C.c_int
        L.or_num_threads.restype = C.c_int
        _lib = L
    return _lib


# ------------------------------------------------------------------ helpers

class _Keep:
    """Holds numpy buffers referenced by ctypes structs."""

    def __init__(self):
        self.refs = []


def make_geom(g) -> tuple:
    """workloads.Geometry -> (OrGeom, keepalive)."""
    k = _Keep()
    og = OrGeom()
    og.kind = int(g.kind)
    og.center[:] = list(map(float, g.center))
    og.radius = float(g.radius)
    og.lo[:] = list(map(float, g.lo))
    og.hi[:] = list(map(float, g.hi))
    og.truncation = float(getattr(g, "truncation", 0.0))
    if g.boxes is not None and len(g.boxes):
        b = np.ascontiguousarray(g.boxes, dtype=np.float64)
        k.refs.append(b)
        og.n_boxes = int(b.shape[0])
        og.boxes = b.ctypes.data_as(C.POINTER(C.c_double))
    else:
        og.n_boxes = 0
        og.boxes = None
    return og, k


def make_data(d) -> tuple:
    k = _Keep()
    od = OrData()
    od.kind = int(d.kind)
    od.x0[:] = list(map(float, d.x0))
    od.strength = float(d.strength)
    od.lmax = int(d.lmax)
    if d.clm is not None:
        c = np.ascontiguousarray(d.clm, dtype=np.float64)
        k.refs.append(c)
        od.clm = c.ctypes.data_as(C.POINTER(C.c_double))
    else:
        od.clm = None
    od.center[:] = list(map(float, d.center))
    od.scale = float(d.scale)
    od.constant = float(d.constant)
    return od, k


def wos_opts(eps=1e-4, seed=0, max_steps=1_000_000, stream=STREAM_F64, score=0) -> OrWosOpts:
    o = OrWosOpts()
    o.eps, o.seed, o.max_steps, o.stream, o.score = eps, seed, max_steps, stream, score
    return o


def philox(ctr, key) -> np.ndarray:
    """or_philox4x32_10: 4 output words for counter ctr (4 x u32) and key (2 x u32)."""
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(np.asarray(ctr, dtype=np.uint32), np.asarray(key, dtype=np.uint32), out)
    return out


def u01_21(f: int) -> float:
    return lib().or_u01_21(int(f) & 0xFFFFFFFF)


def fields21(w) -> np.ndarray:
    """or_fields21: the six 21-bit fields of one Philox block."""
    ww = np.ascontiguousarray(w, dtype=np.uint32)
    f = np.zeros(6, dtype=np.uint32)
    lib().or_fields21(ww, f)
    return f


def u01_53(hi: int, lo: int) -> float:
    return lib().or_u01_53(int(hi) & 0xFFFFFFFF, int(lo) & 0xFFFFFFFF)


def direction(u1: float, u2: float, stream: int) -> np.ndarray:
    """or_direction: the unit jump direction of a walk from two uniforms."""
    om = np.zeros(3)
    lib().or_direction(float(u1), float(u2), int(stream), om)
    return om


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().or_gauss_legendre(n, x, w)
    return x, w


def distance(geom, pts):
    """or_distance over rows of pts -> (d, nearest)."""
    og, keep = make_geom(geom)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    d = np.zeros(len(pts))
    nb = np.zeros((len(pts), 3))
    tmp = np.zeros(3)
    for i, x in enumerate(pts):
        d[i] = lib().or_distance(C.byref(og), np.ascontiguousarray(x), tmp)
        nb[i] = tmp
    return d, nb


def real_sh(lmax: int, direction) -> np.ndarray:
    Y = np.zeros((lmax + 1) ** 2)
    lib().or_real_sh(lmax, np.ascontiguousarray(direction, dtype=np.float64), Y)
    return Y


def dirichlet(data, pts) -> np.ndarray:
    od, keep = make_data(data)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    return np.array([lib().or_dirichlet(C.byref(od), np.ascontiguousarray(x)) for x in pts])


def neumann_exact(data, pts, normals) -> np.ndarray:
    od, keep = make_data(data)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    nrm = np.ascontiguousarray(normals, dtype=np.float64).reshape(-1, 3)
    return np.array([lib().or_neumann_exact(C.byref(od), np.ascontiguousarray(x),
                                            np.ascontiguousarray(n)) for x, n in zip(pts, nrm)])


def walk(geom, data, y, walk_id, point, patch, opts):
    og, k1 = make_geom(geom)
    od, k2 = make_data(data)
    sc = C.c_double(0.0)
    st = C.c_uint64(0)
    ok = lib().or_walk(C.byref(og), C.byref(od), np.ascontiguousarray(y, dtype=np.float64),
                       walk_id, point, patch, C.byref(opts), C.byref(sc), C.byref(st))
    return bool(ok), sc.value, st.value


def wos_points(geom, data, y, point_ids, patch_ids, walks, opts):
    """or_wos_points -> dict(sum, sum2, steps, capped) per node."""
    og, k1 = make_geom(geom)
    od, k2 = make_data(data)
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1, 3)
    n = len(y)
    pt = np.ascontiguousarray(np.broadcast_to(np.asarray(point_ids, dtype=np.uint32), (n,)))
    pa = np.ascontiguousarray(np.broadcast_to(np.asarray(patch_ids, dtype=np.uint32), (n,)))
    wk = np.ascontiguousarray(np.broadcast_to(np.asarray(walks, dtype=np.int64), (n,)))
    s1 = np.zeros(n); s2 = np.zeros(n)
    st = np.zeros(n, dtype=np.uint64); cp = np.zeros(n, dtype=np.uint64)
    lib().or_wos_points(C.byref(og), C.byref(od), n, y, pt, pa, wk, C.byref(opts), s1, s2, st, cp)
    return dict(sum=s1, sum2=s2, steps=st, capped=cp)


def wos_estimates(res, walks):
    """Mean and standard error (Eq. bw87) from sums."""
    N = np.asarray(walks, dtype=np.float64) - res["capped"].astype(np.float64)
    U = res["sum"] / N
    var = (res["sum2"] - N * U * U) / (N * (N - 1.0))
    return U, np.sqrt(np.maximum(var, 0.0))


def patch_frame(geom, c, a) -> OrPatch:
    og, keep = make_geom(geom)
    p = OrPatch()
    rc = lib().or_patch_frame(C.byref(og), np.ascontiguousarray(c, dtype=np.float64), float(a),
                              C.byref(p))
    if rc != 0:
        raise ValueError("unsupported patch (ball meets more than one face)")
    return p


def gamma_nodes(p: OrPatch, nt: int, nph: int):
    P = nt * nph
    Yl = np.zeros((P, 3)); yg = np.zeros((P, 3)); W = np.zeros(P)
    lib().or_gamma_nodes(C.byref(p), nt, nph, Yl, yg, W)
    return Yl, yg, W


def panels(p: OrPatch, nr: int, ns: int):
    n = nr * ns
    Xl = np.zeros((n, 3)); xg = np.zeros((n, 3)); ng = np.zeros((n, 3))
    ar = np.zeros(n); prm = np.zeros((n, 7))
    rc = lib().or_panels(C.byref(p), nr, ns, Xl, xg, ng, ar, prm)
    if rc != 0:
        raise ValueError("or_panels: fewer sectors than the wrapped patch's sub-ranges")
    return dict(Xloc=Xl, x=xg, normal=ng, area=ar, prm=prm)


def green(a, X, Y) -> float:
    return lib().or_green(float(a), np.ascontiguousarray(X, dtype=np.float64),
                          np.ascontiguousarray(Y, dtype=np.float64))


def green_grad_y(a, X, Y) -> np.ndarray:
    g = np.zeros(3)
    lib().or_green_grad_y(float(a), np.ascontiguousarray(X, dtype=np.float64),
                          np.ascontiguousarray(Y, dtype=np.float64), g)
    return g


def poisson(a, X, Y) -> float:
    return lib().or_poisson(float(a), np.ascontiguousarray(X, dtype=np.float64),
                            np.ascontiguousarray(Y, dtype=np.float64))


def panel_integral(p: OrPatch, data, kind: int, X, prm, sing=None, rtol=1e-13) -> float:
    od, keep = make_data(data) if data is not None else (None, None)
    s = None
    if sing is not None:
        sarr = np.ascontiguousarray(sing, dtype=np.float64)
        s = sarr.ctypes.data_as(C.c_void_p)
    return lib().or_panel_integral(C.byref(p), C.byref(od) if od is not None else None, kind,
                                   np.ascontiguousarray(X, dtype=np.float64),
                                   np.ascontiguousarray(prm, dtype=np.float64), s, rtol)


def assemble(p: OrPatch, data, nr, ns, nt, nph, U, rtol=1e-13):
    od, keep = make_data(data)
    n = nr * ns
    A = np.zeros((n, n)); b = np.zeros(n)
    rc = lib().or_assemble(C.byref(p), C.byref(od), nr, ns, nt, nph,
                           np.ascontiguousarray(U, dtype=np.float64), rtol, A, b)
    if rc != 0:
        raise ValueError("or_assemble: fewer sectors than the wrapped patch's sub-ranges")
    return A, b


def lu_solve(A, b) -> np.ndarray:
    A = np.array(A, dtype=np.float64, order="C")
    b = np.array(b, dtype=np.float64)
    x = np.zeros(len(b))
    rc = lib().or_lu_solve(len(b), A, b, x)
    if rc != 0:
        raise np.linalg.LinAlgError(f"zero pivot at column {rc - 1}")
    return x


def solve_patch(geom, data, c, a, nt, nph, nr, ns, walks, patch_id, opts, U_in=None, rtol=1e-13):
    """or_solve_patch -> dict(U, SE, steps, q)."""
    og, k1 = make_geom(geom)
    od, k2 = make_data(data)
    P, n = nt * nph, nr * ns
    U = np.zeros(P); SE = np.zeros(P); st = np.zeros(1, dtype=np.uint64); q = np.zeros(n)
    uin = None
    if U_in is not None:
        uarr = np.ascontiguousarray(U_in, dtype=np.float64)
        uin = uarr.ctypes.data_as(C.c_void_p)
    rc = lib().or_solve_patch(C.byref(og), C.byref(od), np.ascontiguousarray(c, dtype=np.float64),
                              float(a), nt, nph, nr, ns, int(walks), patch_id, C.byref(opts), uin,
                              rtol, U, SE, st, q)
    if rc != 0:
        raise RuntimeError(f"or_solve_patch failed ({rc})")
    return dict(U=U, SE=SE, steps=int(st[0]), q=q)


def potential(y, normals, area, q, g, targets) -> np.ndarray:
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1, 3)
    t = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(len(t))
    lib().or_potential(len(y), y, np.ascontiguousarray(normals, dtype=np.float64),
                       np.ascontiguousarray(area, dtype=np.float64),
                       np.ascontiguousarray(q, dtype=np.float64),
                       np.ascontiguousarray(g, dtype=np.float64), len(t), t, out)
    return out


def potential_majorants(y, area, q, g, targets) -> tuple:
    """(b0, b1) per target: sum |A q| / (4 pi r) and sum |A g| / (4 pi r^2)."""
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1, 3)
    t = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 3)
    b0 = np.zeros(len(t))
    b1 = np.zeros(len(t))
    lib().or_potential_majorants(len(y), y, np.ascontiguousarray(area, dtype=np.float64),
                                 np.ascontiguousarray(q, dtype=np.float64),
                                 np.ascontiguousarray(g, dtype=np.float64), len(t), t, b0, b1)
    return b0, b1


def owned(x, owner_patch, centers) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    cen = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 3)
    keep = np.zeros(len(x), dtype=np.uint8)
    lib().or_owned(len(x), x, np.ascontiguousarray(owner_patch, dtype=np.int64), len(cen), cen, keep)
    return keep.astype(bool)


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(n: int) -> None:
    lib().or_set_num_threads(int(n))


def single_point(geom, data, x, a, ng1, ng2, delta, walks=0, patch=0, opts=None, U_in=None):
    """or_single_point: Neumann data at one point of a flat boundary piece by
    Sigma1' + Sigma2' (Sec. 4.1, Eq. bw64-bw88).  Returns dict(sigma1, sigma2, q,
    se, U) or None if x is not on a supported flat piece."""
    og, k1 = make_geom(geom)
    od, k2 = make_data(data)
    o = opts if opts is not None else wos_opts()
    nn = ng1 * ng1
    U = np.zeros(nn)
    out = np.zeros(4)
    uin = None
    if U_in is not None:
        uin = np.ascontiguousarray(U_in, dtype=np.float64)
        assert uin.shape == (nn,)
    rc = lib().or_single_point(C.byref(og), C.byref(od), np.ascontiguousarray(x, dtype=np.float64), float(a),
                               int(ng1), int(ng2), float(delta), int(walks), int(patch), C.byref(o),
                               None if uin is None else uin.ctypes.data_as(C.c_void_p), out,
                               U.ctypes.data_as(C.c_void_p))
    if rc != 0:
        return None
    return dict(sigma1=out[0], sigma2=out[1], q=out[2], se=out[3], U=U)



def green_dnn(a, X, nx, Y, ny) -> float:
    """or_green_dnn: d2G/dn_x dn_y of the whole-sphere Dirichlet Green's function."""
    f = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    return lib().or_green_dnn(float(a), f(X), f(nx), f(Y), f(ny))


def second_kind_flat(p: OrPatch, data, nt, nph, nr, ns, U, ng2=20) -> np.ndarray:
    """or_second_kind_flat: Neumann data of a disk patch by the second-kind
    local BIE (Eq. bw55-bw59), hemisphere values U at or_gamma_nodes(p, nt, nph)."""
    od, keep = make_data(data)
    q = np.zeros(nr * ns)
    rc = lib().or_second_kind_flat(C.byref(p), C.byref(od), int(nt), int(nph), int(nr), int(ns),
                                   np.ascontiguousarray(U, dtype=np.float64), int(ng2), q)
    if rc != 0:
        raise ValueError("second-kind rows need a disk patch")
    return q


def set_sk_self_order(n: int) -> int:
    """Gauss order per direction of the second kind's self-panel rule (default
    20); returns the previous order."""
    return int(lib().or_set_sk_self_order(int(n)))


def second_kind(p: OrPatch, data, nt, nph, nr, ns, U, rtol=1e-10, want_system=False):
    """or_second_kind: Neumann data of a disk or cap patch by the second-kind
    local BIE (Eq. bw55-bw59) with the harmonic-linear regularisation of the
    finite part; hemisphere values U at or_gamma_nodes(p, nt, nph).  With
    want_system also returns (A, b) of (1/2 I - D) q = b.  rtol: the adaptive
    panel rules' relative tolerance; below ~1e-11 the rules next to x_i chase
    the rounding of g - l (O(r^2) against g = O(1)) and slow down."""
    od, keep = make_data(data)
    n = nr * ns
    q = np.zeros(n)
    A = np.zeros((n, n)) if want_system else None
    b = np.zeros(n) if want_system else None
    rc = lib().or_second_kind(C.byref(p), C.byref(od), int(nt), int(nph), int(nr), int(ns),
                              np.ascontiguousarray(U, dtype=np.float64), float(rtol),
                              None if A is None else A.ctypes.data_as(C.c_void_p),
                              None if b is None else b.ctypes.data_as(C.c_void_p), q)
    if rc != 0:
        raise ValueError(f"or_second_kind: LU status {rc}")
    return (q, A, b) if want_system else q


__all__ = [n for n in dir() if not n.startswith("_")]
