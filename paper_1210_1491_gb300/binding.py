"""Thin ctypes binding of libdtn.so (include/dtn.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels; this module only turns
torch tensors into device pointers and Python values into the C structs.  If
the library is missing it raises instead of computing anything itself.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdtn.so")

PREC_FP64 = 0
PREC_MIXED = 1

GEOM_BALL_INTERIOR = 0
GEOM_BOX_INTERIOR = 1
GEOM_BOX_MINUS_BOXES = 2
GEOM_HALF_SPACE = 3
GEOM_DISK_EXTERIOR = 4
GEOM_BALL_EXTERIOR = 5

DATA_POINT_SOURCE = 0
DATA_HARMONIC_SH = 1
DATA_CONSTANT = 2

STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA runtime error",
          4: "refinement did not converge", 5: "timed out", 6: "unsupported patch or geometry",
          7: "walks cut at max_steps"}


class DtnError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)} (status {code})")
        self.code = code


class GeometryDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("center", C.c_double * 3), ("radius", C.c_double),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("n_boxes", C.c_int32),
                ("boxes", C.POINTER(C.c_double)), ("cell_size", C.c_double), ("truncation", C.c_double)]


class DirichletDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("x0", C.c_double * 3), ("strength", C.c_double),
                ("lmax", C.c_int32), ("clm", C.POINTER(C.c_double)), ("center", C.c_double * 3),
                ("scale", C.c_double), ("constant", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("prec", C.c_int32), ("epsilon", C.c_double), ("seed", C.c_uint64),
                ("max_steps", C.c_uint64), ("max_refine_iters", C.c_int32), ("refine_tol", C.c_double),
                ("u_provided", C.c_int32), ("walk_chunk", C.c_int32), ("wos_blocks_per_sm", C.c_int32),
                ("graph_capture", C.c_int32), ("record_stages", C.c_int32), ("wos_refill", C.c_int32),
                ("bie_kind", C.c_int32), ("ring_order", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("walk_chunk", C.c_int32), ("wos_blocks_per_sm", C.c_int32), ("wos_refill", C.c_int32),
                ("ns_per_walk_step", C.c_float)]


class PatchBatch(C.Structure):
    _fields_ = [("n_patches", C.c_int64), ("centers", C.c_void_p), ("radius", C.c_void_p),
                ("n_theta", C.c_void_p), ("n_phi", C.c_void_p), ("n_rings", C.c_void_p),
                ("n_sectors", C.c_void_p), ("walks_per_point", C.c_void_p),
                ("patch_id_base", C.c_uint32), ("patch_ids", C.c_void_p)]


class PatchResult(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in (
        "gamma_xyz", "gamma_w", "u_gamma_mean", "u_gamma_se", "gamma_steps", "gamma_capped",
        "colloc_xyz", "normals", "areas", "dirichlet", "neumann", "matrix", "rhs", "refine_iters",
        "residual", "patch_status")]


class ServerConfig(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("max_batch_patches", C.c_int64),
                ("memory_budget", C.c_int64), ("opts", SolveOpts), ("split_sms", C.c_int32)]


class ServerInfo(C.Structure):
    _fields_ = [("budget_bytes", C.c_int64), ("device_free_bytes", C.c_int64), ("held_bytes", C.c_int64),
                ("peak_held_bytes", C.c_int64), ("batches", C.c_int64), ("queries", C.c_int64),
                ("rejected", C.c_int64), ("max_concurrent", C.c_int32), ("busy_ms", C.c_double),
                ("overlap_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Query(C.Structure):
    _fields_ = [("n_patches", C.c_int64), ("centers", C.c_void_p), ("radius", C.c_void_p),
                ("n_theta", C.c_void_p), ("n_phi", C.c_void_p), ("n_rings", C.c_void_p),
                ("n_sectors", C.c_void_p), ("walks_per_point", C.c_void_p), ("patch_ids", C.c_void_p)]


class FmmOpts(C.Structure):
    _fields_ = [("order", C.c_int32), ("leaf_sources", C.c_int32), ("leaf_targets", C.c_int32),
                ("max_level", C.c_int32), ("theta", C.c_double)]


class FmmStats(C.Structure):
    _fields_ = [("source_cells", C.c_int64), ("target_cells", C.c_int64), ("m2l_pairs", C.c_int64),
                ("p2p_pairs", C.c_int64), ("p2p_terms", C.c_int64), ("source_levels", C.c_int32),
                ("target_levels", C.c_int32), ("traversal_passes", C.c_int32), ("restarts", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["dtn_create_geometry", "dtn_destroy_geometry", "dtn_set_dirichlet", "dtn_query_patch_sizes",
           "dtn_solve_patches", "dtn_eval_potential", "dtn_gather_owned", "dtn_wos_points",
           "dtn_distance", "dtn_philox4x32_10", "dtn_eval_dirichlet", "dtn_status_string",
           "dtn_last_cuda_error", "dtn_server_create", "dtn_server_submit", "dtn_server_poll",
           "dtn_server_drain", "dtn_server_destroy", "dtn_stage_times", "dtn_autotune_walks",
           "dtn_wos_points_noalloc", "dtn_single_point_neumann", "dtn_eval_potential_fmm",
           "dtn_philox_fields21", "dtn_release_workspace", "dtn_server_stats"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libdtn.so (build it first with paper_1210_1491_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libdtn.so not found at {path}: run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(path)
    vp, i64, i32, u64, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_double
    sig = {
        "dtn_create_geometry": ([C.POINTER(GeometryDesc), C.POINTER(vp)], i32),
        "dtn_destroy_geometry": ([vp], i32),
        "dtn_set_dirichlet": ([vp, C.POINTER(DirichletDesc)], i32),
        "dtn_query_patch_sizes": ([C.POINTER(PatchBatch), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)], i32),
        "dtn_solve_patches": ([vp, C.POINTER(PatchBatch), C.POINTER(SolveOpts), C.POINTER(PatchResult), vp], i32),
        "dtn_eval_potential": ([vp, i64, vp, vp, vp, vp, vp, vp, vp, i64, vp, vp, i32, vp], i32),
        "dtn_gather_owned": ([i64, vp, vp, i64, vp, vp, vp, vp, vp], i32),
        "dtn_wos_points": ([vp, i64, vp, vp, vp, vp, C.POINTER(SolveOpts), vp, vp, vp, vp, vp], i32),
        "dtn_distance": ([vp, i64, vp, vp, vp, i32, vp], i32),
        "dtn_philox4x32_10": ([i64, vp, u64, vp, vp], i32),
        "dtn_philox_fields21": ([i64, vp, u64, vp, vp, vp, vp], i32),
        "dtn_eval_dirichlet": ([vp, i64, vp, vp, vp], i32),
        "dtn_status_string": ([i32], C.c_char_p),
        "dtn_last_cuda_error": ([], i32),
        "dtn_server_create": ([vp, C.POINTER(ServerConfig), C.POINTER(vp)], i32),
        "dtn_server_submit": ([vp, C.POINTER(Query), C.POINTER(i64)], i32),
        "dtn_server_poll": ([vp, i64, C.POINTER(i32), vp, vp, C.POINTER(dbl), vp], i32),
        "dtn_server_stats": ([vp, C.POINTER(ServerInfo)], i32),
        "dtn_release_workspace": ([vp], i32),
        "dtn_server_drain": ([vp], i32),
        "dtn_server_destroy": ([vp], i32),
        "dtn_stage_times": ([vp, C.POINTER(C.c_float)], i32),
        "dtn_autotune_walks": ([vp, C.POINTER(PatchBatch), C.POINTER(SolveOpts), C.POINTER(Tuning), vp], i32),
        "dtn_wos_points_noalloc": ([vp, i64, vp, vp, vp, vp, C.POINTER(SolveOpts), vp, vp, vp, vp, vp], i32),
        "dtn_single_point_neumann": ([vp, i64, vp, dbl, i32, i32, dbl, vp, C.c_uint32, C.POINTER(SolveOpts),
                                      vp, vp, vp, vp, vp, vp, vp], i32),
        "dtn_eval_potential_fmm": ([vp, i64, vp, vp, vp, vp, vp, vp, vp, i64, vp, vp, C.POINTER(FmmOpts),
                                    C.POINTER(FmmStats), vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(code: int, what: str):
    if code != 0:
        # a failed CUDA runtime call: name it (cudaError_t value)
        cu = load().dtn_last_cuda_error() if code in (2, 3) else 0
        raise DtnError(code, what + (f" [cudaError {cu}]" if cu else ""))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(t.ctypes.data)
    raise TypeError(type(t))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(t, dtype):
    """Device tensor of dtype on cuda:0 (copies only when needed)."""
    return torch.as_tensor(t).to(device="cuda", dtype=dtype).contiguous()


def _host_f64(t):
    """Host float64 array (per-patch shape parameters live on the host)."""
    if isinstance(t, torch.Tensor):
        t = t.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(-1))


def solve_opts(prec=PREC_MIXED, epsilon=1e-4, seed=0, max_steps=0, max_refine_iters=0, refine_tol=0.0,
               u_provided=False, walk_chunk=0, wos_blocks_per_sm=0, graph_capture=False,
               record_stages=False, wos_refill=0, bie_kind=0, ring_order=0) -> SolveOpts:
    o = SolveOpts()
    o.prec, o.epsilon, o.seed, o.max_steps = int(prec), float(epsilon), int(seed), int(max_steps)
    o.max_refine_iters, o.refine_tol, o.u_provided = int(max_refine_iters), float(refine_tol), int(u_provided)
    o.walk_chunk, o.wos_blocks_per_sm, o.graph_capture = int(walk_chunk), int(wos_blocks_per_sm), int(graph_capture)
    o.record_stages = int(record_stages)
    o.wos_refill = int(wos_refill)
    o.bie_kind, o.ring_order = int(bie_kind), int(ring_order)
    return o


def autotune_walks(geom, centers, radius, hb, opts: SolveOpts, stream=None) -> dict:
    """dtn_autotune_walks: pick and cache the walk-kernel launch parameters."""
    c = _dev(centers, torch.float64).reshape(-1, 3)
    rad = _host_f64(radius)
    t = Tuning()
    b = hb.struct(c, rad)
    _check(load().dtn_autotune_walks(geom.handle, C.byref(b), C.byref(opts), C.byref(t), _stream(stream)),
           "dtn_autotune_walks")
    return dict(walk_chunk=t.walk_chunk, wos_blocks_per_sm=t.wos_blocks_per_sm, wos_refill=t.wos_refill,
                ns_per_walk_step=t.ns_per_walk_step)


class Geometry:
    """dtn_create_geometry / dtn_set_dirichlet / dtn_destroy_geometry."""

    def __init__(self, kind, center=(0, 0, 0), radius=1.0, lo=(0, 0, 0), hi=(1, 1, 1), boxes=None,
                 cell_size=0.0, truncation=0.0):
        L = load()
        d = GeometryDesc()
        d.kind = int(kind)
        d.center[:] = [float(v) for v in center]
        d.radius = float(radius)
        d.lo[:] = [float(v) for v in lo]
        d.hi[:] = [float(v) for v in hi]
        self._boxes = None
        if boxes is not None and len(boxes):
            self._boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 6)
            d.n_boxes = int(self._boxes.shape[0])
            d.boxes = self._boxes.ctypes.data_as(C.POINTER(C.c_double))
        d.cell_size = float(cell_size)
        d.truncation = float(truncation)
        h = C.c_void_p()
        _check(L.dtn_create_geometry(C.byref(d), C.byref(h)), "dtn_create_geometry")
        self.handle = h
        self.kind = int(kind)

    @classmethod
    def from_spec(cls, g, cell_size=0.0):
        """From any object with kind/center/radius/lo/hi/boxes (and truncation) attributes."""
        return cls(g.kind, g.center, g.radius, g.lo, g.hi, g.boxes, cell_size, getattr(g, "truncation", 0.0))

    def set_dirichlet(self, kind, x0=(0, 0, 0), strength=1.0, lmax=0, clm=None, center=(0, 0, 0),
                      scale=1.0, constant=0.0):
        d = DirichletDesc()
        d.kind = int(kind)
        d.x0[:] = [float(v) for v in x0]
        d.strength = float(strength)
        d.lmax = int(lmax)
        self._clm = None
        if clm is not None:
            self._clm = np.ascontiguousarray(clm, dtype=np.float64)
            d.clm = self._clm.ctypes.data_as(C.POINTER(C.c_double))
        d.center[:] = [float(v) for v in center]
        d.scale = float(scale)
        d.constant = float(constant)
        _check(load().dtn_set_dirichlet(self.handle, C.byref(d)), "dtn_set_dirichlet")
        return self

    def set_data_spec(self, d):
        return self.set_dirichlet(d.kind, d.x0, d.strength, d.lmax, d.clm, d.center, d.scale, d.constant)

    def stage_times(self):
        """ms of (setup, walks, assembly, solve) of the last recorded solve."""
        ms = (C.c_float * 4)()
        _check(load().dtn_stage_times(self.handle, ms), "dtn_stage_times")
        return [float(v) for v in ms]

    def release_workspace(self):
        """dtn_release_workspace: free the device workspaces the calls have grown."""
        _check(load().dtn_release_workspace(self.handle), "dtn_release_workspace")

    def close(self):
        if getattr(self, "handle", None):
            load().dtn_destroy_geometry(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostBatch:
    """Host-side per-patch size arrays of a dtn_patch_batch (kept alive here)."""

    def __init__(self, n_theta, n_phi, n_rings, n_sectors, walks, patch_ids=None, patch_id_base=0):
        self.nt = np.ascontiguousarray(n_theta, dtype=np.int32)
        self.nph = np.ascontiguousarray(n_phi, dtype=np.int32)
        self.nr = np.ascontiguousarray(n_rings, dtype=np.int32)
        self.ns = np.ascontiguousarray(n_sectors, dtype=np.int32)
        self.walks = np.ascontiguousarray(walks, dtype=np.int64)
        self.pids = None if patch_ids is None else np.ascontiguousarray(patch_ids, dtype=np.uint32)
        self.base = int(patch_id_base)
        self.n = int(self.nt.shape[0])

    def struct(self, centers_dev, radius_host) -> PatchBatch:
        b = PatchBatch()
        b.n_patches = self.n
        b.centers = _ptr(centers_dev)
        b.radius = _ptr(radius_host)
        b.n_theta, b.n_phi = _ptr(self.nt), _ptr(self.nph)
        b.n_rings, b.n_sectors = _ptr(self.nr), _ptr(self.ns)
        b.walks_per_point = _ptr(self.walks)
        b.patch_id_base = self.base
        b.patch_ids = _ptr(self.pids) if self.pids is not None else None
        return b

    def sizes(self):
        b = self.struct(None, None)
        pt, gt, mt = C.c_int64(), C.c_int64(), C.c_int64()
        _check(load().dtn_query_patch_sizes(C.byref(b), C.byref(pt), C.byref(gt), C.byref(mt)),
               "dtn_query_patch_sizes")
        return pt.value, gt.value, mt.value


def alloc_result(hb: HostBatch, want_matrix=False, want_geometry=True, device="cuda"):
    pt, gt, mt = hb.sizes()
    f64 = dict(dtype=torch.float64, device=device)
    r = dict(
        u_gamma_mean=torch.zeros(gt, **f64), u_gamma_se=torch.zeros(gt, **f64),
        gamma_steps=torch.zeros(gt, dtype=torch.int64, device=device),
        gamma_capped=torch.zeros(gt, dtype=torch.int32, device=device),
        neumann=torch.zeros(pt, **f64), dirichlet=torch.zeros(pt, **f64),
        refine_iters=torch.zeros(hb.n, dtype=torch.int32, device=device),
        residual=torch.zeros(hb.n, **f64),
        patch_status=torch.zeros(hb.n, dtype=torch.int32, device=device),
    )
    if want_geometry:
        r.update(gamma_xyz=torch.zeros(gt, 3, **f64), gamma_w=torch.zeros(gt, **f64),
                 colloc_xyz=torch.zeros(pt, 3, **f64), normals=torch.zeros(pt, 3, **f64),
                 areas=torch.zeros(pt, **f64))
    if want_matrix:
        r.update(matrix=torch.zeros(mt, **f64), rhs=torch.zeros(pt, **f64))
    return r


def _result_struct(r: dict) -> PatchResult:
    s = PatchResult()
    for name, _ in PatchResult._fields_:
        setattr(s, name, _ptr(r.get(name)) if r.get(name) is not None else None)
    return s


def solve_patches(geom: Geometry, centers, radius, hb: HostBatch, opts: SolveOpts, result=None,
                  stream=None, **alloc_kw):
    """dtn_solve_patches on device tensors; returns the result dict of tensors."""
    c = _dev(centers, torch.float64).reshape(-1, 3)
    rad = _host_f64(radius)
    if result is None:
        result = alloc_result(hb, **alloc_kw)
    b = hb.struct(c, rad)
    rs = _result_struct(result)
    _check(load().dtn_solve_patches(geom.handle, C.byref(b), C.byref(opts), C.byref(rs), _stream(stream)),
           "dtn_solve_patches")
    result["_keep"] = (c, rad)
    return result


def eval_potential(geom: Geometry, xyz, normals, areas, neumann, dirichlet, targets, prec=PREC_MIXED,
                   out=None, stream=None, index=None, n_index=None):
    x = _dev(xyz, torch.float64).reshape(-1, 3)
    n = _dev(normals, torch.float64).reshape(-1, 3)
    a = _dev(areas, torch.float64).reshape(-1)
    q = _dev(neumann, torch.float64).reshape(-1)
    g = None if dirichlet is None else _dev(dirichlet, torch.float64).reshape(-1)
    t = _dev(targets, torch.float64).reshape(-1, 3)
    if out is None:
        out = torch.empty(t.shape[0], dtype=torch.float64, device="cuda")
    idx = None if index is None else _dev(index, torch.int64).reshape(-1)
    cnt = None if n_index is None else _dev(n_index, torch.int64)
    if idx is not None and cnt is None and idx.numel() < x.shape[0]:
        raise ValueError("index without n_index must hold one entry per panel array row")
    _check(load().dtn_eval_potential(geom.handle, x.shape[0], _ptr(x), _ptr(n), _ptr(a), _ptr(q), _ptr(g),
                                     _ptr(idx), _ptr(cnt), t.shape[0], _ptr(t), _ptr(out), int(prec),
                                     _stream(stream)),
           "dtn_eval_potential")
    return out


def fmm_opts(order=10, theta=0.6, leaf_sources=128, leaf_targets=64, max_level=20) -> FmmOpts:
    """FMM options; the defaults are the fastest setting measured on 10^6 sphere panels x 10^6 targets
    at relative error ~3e-6 against the FP64 direct sum."""
    return FmmOpts(int(order), int(leaf_sources), int(leaf_targets), int(max_level), float(theta))


def eval_potential_fmm(geom: Geometry, xyz, normals, areas, neumann, dirichlet, targets, opts: FmmOpts = None,
                       out=None, stream=None, index=None, n_index=None, want_stats=False):
    """dtn_eval_potential_fmm: the sum of eval_potential by the fast multipole method."""
    x = _dev(xyz, torch.float64).reshape(-1, 3)
    n = _dev(normals, torch.float64).reshape(-1, 3)
    a = _dev(areas, torch.float64).reshape(-1)
    q = _dev(neumann, torch.float64).reshape(-1)
    g = None if dirichlet is None else _dev(dirichlet, torch.float64).reshape(-1)
    t = _dev(targets, torch.float64).reshape(-1, 3)
    if out is None:
        out = torch.empty(t.shape[0], dtype=torch.float64, device="cuda")
    idx = None if index is None else _dev(index, torch.int64).reshape(-1)
    cnt = None if n_index is None else _dev(n_index, torch.int64)
    if idx is not None and cnt is None and idx.numel() < x.shape[0]:
        raise ValueError("index without n_index must hold one entry per panel array row")
    o = opts if opts is not None else fmm_opts()
    st = FmmStats()
    _check(load().dtn_eval_potential_fmm(geom.handle, x.shape[0], _ptr(x), _ptr(n), _ptr(a), _ptr(q), _ptr(g),
                                         _ptr(idx), _ptr(cnt), t.shape[0], _ptr(t), _ptr(out), C.byref(o),
                                         C.byref(st), _stream(stream)),
           "dtn_eval_potential_fmm")
    return (out, st.as_dict()) if want_stats else out


def gather_owned(colloc_xyz, owner, centers, stream=None):
    """dtn_gather_owned -> (keep mask, kept indices) as device tensors."""
    x = _dev(colloc_xyz, torch.float64).reshape(-1, 3)
    o = _dev(owner, torch.int64).reshape(-1)
    c = _dev(centers, torch.float64).reshape(-1, 3)
    keep = torch.empty(x.shape[0], dtype=torch.uint8, device="cuda")
    kept = torch.empty(x.shape[0], dtype=torch.int64, device="cuda")
    nk = torch.empty(1, dtype=torch.int64, device="cuda")   # written by the library
    _check(load().dtn_gather_owned(x.shape[0], _ptr(x), _ptr(o), c.shape[0], _ptr(c), _ptr(keep), _ptr(kept),
                                   _ptr(nk), _stream(stream)), "dtn_gather_owned")
    return keep, kept, nk


def wos_points(geom: Geometry, y, point_ids, patch_ids, walks, opts: SolveOpts, stream=None):
    yy = _dev(y, torch.float64).reshape(-1, 3)
    n = yy.shape[0]
    pt = _dev(np.broadcast_to(np.asarray(point_ids, dtype=np.uint32), (n,)).astype(np.int64), torch.int64)
    pa = _dev(np.broadcast_to(np.asarray(patch_ids, dtype=np.uint32), (n,)).astype(np.int64), torch.int64)
    pt32 = pt.to(torch.int32).contiguous()
    pa32 = pa.to(torch.int32).contiguous()
    w = np.ascontiguousarray(np.broadcast_to(np.asarray(walks, dtype=np.int64), (n,)))
    mean = torch.empty(n, dtype=torch.float64, device="cuda")
    se = torch.empty(n, dtype=torch.float64, device="cuda")
    steps = torch.empty(n, dtype=torch.int64, device="cuda")
    capped = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(load().dtn_wos_points(geom.handle, n, _ptr(yy), _ptr(pt32), _ptr(pa32), _ptr(w), C.byref(opts),
                                 _ptr(mean), _ptr(se), _ptr(steps), _ptr(capped), _stream(stream)),
           "dtn_wos_points")
    return dict(mean=mean, se=se, steps=steps, capped=capped)


def wos_points_noalloc(geom: Geometry, y, point_ids, patch_ids, walks, opts: SolveOpts, out=None,
                       stream=None):
    """dtn_wos_points_noalloc: the library allocates nothing (the caller's tensors
    in `out`, if given, receive mean / se / steps / capped)."""
    yy = _dev(y, torch.float64).reshape(-1, 3)
    n = yy.shape[0]
    pt32 = _dev(np.broadcast_to(np.asarray(point_ids, dtype=np.uint32), (n,)).astype(np.int64),
                torch.int64).to(torch.int32).contiguous()
    pa32 = _dev(np.broadcast_to(np.asarray(patch_ids, dtype=np.uint32), (n,)).astype(np.int64),
                torch.int64).to(torch.int32).contiguous()
    w = np.ascontiguousarray(np.broadcast_to(np.asarray(walks, dtype=np.int64), (n,)))
    if out is None:
        out = dict(mean=torch.empty(n, dtype=torch.float64, device="cuda"),
                   se=torch.empty(n, dtype=torch.float64, device="cuda"),
                   steps=torch.empty(n, dtype=torch.int64, device="cuda"),
                   capped=torch.empty(n, dtype=torch.int32, device="cuda"))
    _check(load().dtn_wos_points_noalloc(geom.handle, n, _ptr(yy), _ptr(pt32), _ptr(pa32), _ptr(w), C.byref(opts),
                                         _ptr(out["mean"]), _ptr(out.get("se")), _ptr(out.get("steps")),
                                         _ptr(out.get("capped")), _stream(stream)),
           "dtn_wos_points_noalloc")
    return out


def single_point_neumann(geom: Geometry, x, a, ng1, ng2, delta, walks, opts: SolveOpts, patch_id_base=0,
                         want_nodes=False, stream=None):
    """dtn_single_point_neumann: q = Sigma1' + Sigma2' at points x (n x 3) of flat
    boundary pieces -> dict of device tensors (sigma1, sigma2, q, se, status, U)."""
    xx = _dev(x, torch.float64).reshape(-1, 3)
    n = xx.shape[0]
    w = np.ascontiguousarray(np.broadcast_to(np.asarray(walks, dtype=np.int64), (n,)))
    out = dict(sigma1=torch.empty(n, dtype=torch.float64, device="cuda"),
               sigma2=torch.empty(n, dtype=torch.float64, device="cuda"),
               q=torch.empty(n, dtype=torch.float64, device="cuda"),
               se=torch.empty(n, dtype=torch.float64, device="cuda"),
               status=torch.empty(n, dtype=torch.int32, device="cuda"))
    if want_nodes:
        out["U"] = torch.empty(n * int(ng1) * int(ng1), dtype=torch.float64, device="cuda")
    _check(load().dtn_single_point_neumann(geom.handle, n, _ptr(xx), float(a), int(ng1), int(ng2), float(delta),
                                           _ptr(w), int(patch_id_base), C.byref(opts), _ptr(out["sigma1"]),
                                           _ptr(out["sigma2"]), _ptr(out["q"]), _ptr(out["se"]),
                                           _ptr(out["status"]), _ptr(out.get("U")), _stream(stream)),
           "dtn_single_point_neumann")
    out["_keep"] = (xx, w)
    return out


def distance(geom: Geometry, x, prec=PREC_FP64, stream=None):
    xx = _dev(x, torch.float64).reshape(-1, 3)
    d = torch.empty(xx.shape[0], dtype=torch.float64, device="cuda")
    nb = torch.empty(xx.shape[0], 3, dtype=torch.float64, device="cuda")
    _check(load().dtn_distance(geom.handle, xx.shape[0], _ptr(xx), _ptr(d), _ptr(nb), int(prec), _stream(stream)),
           "dtn_distance")
    return d, nb


def philox(ctr, seed: int, stream=None):
    """dtn_philox4x32_10 on a (n, 4) uint32 counter array -> (n, 4) uint32 numpy array."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    cd = torch.from_numpy(c.view(np.int32)).to("cuda")
    out = torch.empty_like(cd)
    _check(load().dtn_philox4x32_10(c.shape[0], _ptr(cd), int(seed), _ptr(out), _stream(stream)),
           "dtn_philox4x32_10")
    return out.cpu().numpy().view(np.uint32)


def philox_fields21(ctr, seed: int, stream=None):
    """dtn_philox_fields21 on a (n, 4) uint32 counter array -> numpy (fields (n, 6)
    uint32, uniforms (n, 6) float32, directions (n, 3, 3) float32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    cd = torch.from_numpy(c.view(np.int32)).to("cuda")
    n = c.shape[0]
    f = torch.empty(n, 6, dtype=torch.int32, device="cuda")
    u = torch.empty(n, 6, dtype=torch.float32, device="cuda")
    d = torch.empty(n, 3, 3, dtype=torch.float32, device="cuda")
    _check(load().dtn_philox_fields21(n, _ptr(cd), int(seed), _ptr(f), _ptr(u), _ptr(d), _stream(stream)),
           "dtn_philox_fields21")
    return f.cpu().numpy().view(np.uint32), u.cpu().numpy(), d.cpu().numpy()


def eval_dirichlet(geom: Geometry, x, stream=None):
    xx = _dev(x, torch.float64).reshape(-1, 3)
    out = torch.empty(xx.shape[0], dtype=torch.float64, device="cuda")
    _check(load().dtn_eval_dirichlet(geom.handle, xx.shape[0], _ptr(xx), _ptr(out), _stream(stream)),
           "dtn_eval_dirichlet")
    return out


class Server:
    """dtn_server_*: continuous-batching request server (host arrays in, host arrays out)."""

    def __init__(self, geom: Geometry, opts: SolveOpts, max_inflight=2, max_batch_patches=4096,
                 memory_budget=0, split_sms=True):
        cfg = ServerConfig()
        cfg.max_inflight, cfg.max_batch_patches, cfg.memory_budget = int(max_inflight), int(max_batch_patches), int(memory_budget)
        cfg.opts = opts
        cfg.split_sms = 1 if split_sms else 0
        h = C.c_void_p()
        _check(load().dtn_server_create(geom.handle, C.byref(cfg), C.byref(h)), "dtn_server_create")
        self.handle = h
        self._geom = geom
        self._sizes = {}

    def submit(self, centers, radius, n_theta, n_phi, n_rings, n_sectors, walks, patch_ids) -> int:
        arrs = [np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 3),
                np.ascontiguousarray(radius, dtype=np.float64),
                np.ascontiguousarray(n_theta, dtype=np.int32), np.ascontiguousarray(n_phi, dtype=np.int32),
                np.ascontiguousarray(n_rings, dtype=np.int32), np.ascontiguousarray(n_sectors, dtype=np.int32),
                np.ascontiguousarray(walks, dtype=np.int64), np.ascontiguousarray(patch_ids, dtype=np.uint32)]
        q = Query()
        q.n_patches = arrs[0].shape[0]
        (q.centers, q.radius, q.n_theta, q.n_phi, q.n_rings, q.n_sectors, q.walks_per_point,
         q.patch_ids) = [_ptr(a) for a in arrs]
        t = C.c_int64()
        _check(load().dtn_server_submit(self.handle, C.byref(q), C.byref(t)), "dtn_server_submit")
        self._sizes[t.value] = (int(np.sum(arrs[4].astype(np.int64) * arrs[5])),
                                int(np.sum(arrs[2].astype(np.int64) * arrs[3])), q.n_patches)
        return t.value

    def poll(self, ticket: int):
        """None while the query runs; then a dict with its status, latency and (unless
        it did not run: DTN_E_CUDA, DTN_E_OUT_OF_MEMORY) neumann, u and patch_status."""
        npan, nnode, npat = self._sizes[ticket]
        q = np.zeros(npan)
        u = np.zeros(nnode)
        ps = np.zeros(npat, dtype=np.int32)
        done = C.c_int32()
        lat = C.c_double()
        st = load().dtn_server_poll(self.handle, ticket, C.byref(done), _ptr(q), _ptr(u), C.byref(lat), _ptr(ps))
        if not done.value:
            _check(st, "dtn_server_poll")
            return None
        if st in (1, 2, 3):   # invalid ticket, out of memory, CUDA: no result
            return dict(status=st, latency_s=lat.value, neumann=None, u=None, patch_status=None)
        return dict(status=st, neumann=q, u=u, patch_status=ps, latency_s=lat.value)

    def stats(self) -> dict:
        info = ServerInfo()
        _check(load().dtn_server_stats(self.handle, C.byref(info)), "dtn_server_stats")
        return info.as_dict()

    def drain(self):
        _check(load().dtn_server_drain(self.handle), "dtn_server_drain")

    def close(self):
        if getattr(self, "handle", None):
            load().dtn_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
