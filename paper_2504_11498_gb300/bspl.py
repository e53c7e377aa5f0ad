"""Python binding of libbspl (include/bspl.h): argument marshalling only.

Every computation runs in the CUDA library; this module maps torch tensors to
the C structs and calls the ``extern "C"`` entry points with the same names.
PyTorch provides device memory and the stream.  The module refuses to work
without the compiled library: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbspl.so")

OK, EINVAL, ENOSPACE, ECUDA, ENOTCONV, ETIMEOUT = 0, 1, 2, 3, 4, 5
FP64, MIXED, LEARNED_MIXED, CLIP_MIXED = 0, 1, 2, 3
Q_CONVERGED, Q_FALLBACK, Q_AT_END, Q_NONCONV, Q_OFF_CURVE, Q_INVALID = 1, 2, 4, 8, 16, 32
GROUP = 32
CREC64, CREC32, SREC64, SREC32, GREC64, GREC32 = 18, 24, 54, 72, 12, 12
SPAN_NET = 8 * 8 * 3
OP_DECOMPOSE_CURVES, OP_DECOMPOSE_SURFACES, OP_QUERY_CURVES, OP_QUERY_SURFACES = 1, 2, 3, 4
OP_QUERY_CURVES_LEARNED, OP_MLP_TRAIN, OP_SMLP_TRAIN, OP_QUERY_SURFACES_LEARNED = 5, 6, 7, 8
OP_REFINE_CURVES = 9
# learned seed (include/bspl_mlp.h)
MLP_IN, MLP_HIDDEN, MLP_NPARAM, MLP_NBF16, MLP_MAX_BATCH = 16, 128, 35332, 2048 + 4 * 16384 + 128, 65536
MLP_OFF = {"W1": 0, "b1": 2048, "W2": 2176, "b2": 18560, "W3": 18688, "b3": 35072, "w4": 35200, "b4": 35328}
MLP_CURVE, MLP_SURFACE = 0, 1
# the surface seed network (bspl_mlp.h BSPL_SMLP_*): 64 inputs (51 used) -> 2
SMLP_IN, SMLP_OUT, SMLP_NPARAM, SMLP_NBF16 = 64, 2, 41604, 8192 + 4 * 16384 + 256
SMLP_OFF = {"W1": 0, "b1": 8192, "W2": 8320, "b2": 24704, "W3": 24832, "b3": 41216, "W4": 41344, "b4": 41600}
NET = {MLP_CURVE: (MLP_IN, 1, MLP_NPARAM, MLP_NBF16, OP_MLP_TRAIN),
       MLP_SURFACE: (SMLP_IN, SMLP_OUT, SMLP_NPARAM, SMLP_NBF16, OP_SMLP_TRAIN)}
NCOUNTERS = 14
COUNTER_NAMES = ["queries", "seg_tested", "grp_tested", "candidates", "newton", "fallback", "nonconv",
                 "newton32_iters", "newton64_iters", "iso_pairs", "cert_cells", "cert_leaves", "cert_overflow",
                 "classified"]


class BsplError(RuntimeError):
    pass


class bspl_curves(C.Structure):
    _fields_ = [("n", C.c_int64), ("degree", C.c_void_p), ("knot_off", C.c_void_p), ("knots", C.c_void_p),
                ("cp_off", C.c_void_p), ("cps", C.c_void_p), ("weights", C.c_void_p)]


class bspl_surfaces(C.Structure):
    _fields_ = [("n", C.c_int64), ("deg_u", C.c_void_p), ("deg_v", C.c_void_p), ("n_u", C.c_void_p),
                ("n_v", C.c_void_p), ("knot_u_off", C.c_void_p), ("knots_u", C.c_void_p),
                ("knot_v_off", C.c_void_p), ("knots_v", C.c_void_p), ("cp_off", C.c_void_p), ("cps", C.c_void_p)]


class bspl_segments(C.Structure):
    _fields_ = [("is_surface", C.c_int32), ("n", C.c_int64), ("capacity", C.c_int64), ("grp_capacity", C.c_int64),
                ("seg_off", C.c_void_p), ("ctrl", C.c_void_p), ("prange", C.c_void_p), ("diag", C.c_void_p),
                ("rec64", C.c_void_p), ("rec32", C.c_void_p), ("grp_off", C.c_void_p), ("grp64", C.c_void_p),
                ("grp32", C.c_void_p), ("patch_span", C.c_void_p), ("patch_box", C.c_void_p),
                ("span_net", C.c_void_p), ("span_net32", C.c_void_p), ("n_cp_total", C.c_int64),
                ("tol_rel", C.c_double), ("patch_net32", C.c_void_p), ("spline_rank", C.c_void_p)]


class bspl_options(C.Structure):
    _fields_ = [("prec", C.c_int32), ("samples", C.c_int32), ("newton_max", C.c_int32), ("fp32_steps", C.c_int32),
                ("sort_queries", C.c_int32), ("occupancy", C.c_int32), ("pairs_per_query", C.c_int32),
                ("mlp", C.c_void_p),
                ("counters", C.c_void_p), ("stage_events", C.c_void_p), ("cert_depth", C.c_int32)]


NSTAGE_EVENTS = 9
STAGE_NAMES = ["sort", "cull", "classify", "seed", "fp32", "fp64", "select", "leftovers"]


class bspl_mlp(C.Structure):
    _fields_ = [("params", C.c_void_p), ("wbf16", C.c_void_p), ("kind", C.c_int32)]


EXPORTS = ["bspl_graph_begin", "bspl_graph_end", "bspl_graph_launch", "bspl_graph_destroy",
           "bspl_project_curves_noalloc", "bspl_measure_fma_peak", "bspl_workspace_bytes", "bspl_decompose", "bspl_project_curves", "bspl_invert_curves",
           "bspl_project_surfaces", "bspl_invert_surfaces", "bspl_eval_curves", "bspl_eval_surfaces",
           "bspl_refine_curves", "bspl_status_string"]

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libbspl.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise BsplError(f"{LIB_PATH} is missing: build it with paper_2504_11498_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            vp, i64, st = C.c_void_p, C.c_int64, C.c_int
            L.bspl_workspace_bytes.restype = C.c_size_t
            L.bspl_workspace_bytes.argtypes = [C.c_int, i64, i64, i64, i64]
            L.bspl_decompose.restype = st
            L.bspl_decompose.argtypes = [C.c_int, vp, C.c_double, C.POINTER(bspl_segments), C.POINTER(i64), vp,
                                         C.c_size_t, vp]
            for name in ("bspl_project_curves", "bspl_invert_curves", "bspl_project_surfaces",
                         "bspl_invert_surfaces"):
                f = getattr(L, name)
                f.restype = st
                f.argtypes = [C.POINTER(bspl_segments), i64, vp, vp, C.POINTER(bspl_options), vp, vp, vp, vp,
                              C.c_size_t, vp]
            L.bspl_eval_curves.restype = st
            L.bspl_eval_curves.argtypes = [C.POINTER(bspl_curves), i64, vp, vp, vp, vp]
            L.bspl_refine_curves.restype = st
            L.bspl_refine_curves.argtypes = [C.POINTER(bspl_curves), vp, C.c_int, i64, vp, vp, C.c_int32, vp, vp,
                                             vp, vp, vp, C.c_size_t, vp]
            L.bspl_eval_surfaces.restype = st
            L.bspl_eval_surfaces.argtypes = [C.POINTER(bspl_surfaces), i64, vp, vp, vp, vp]
            L.bspl_status_string.restype = C.c_char_p
            L.bspl_status_string.argtypes = [st]
            L.bspl_project_curves_noalloc.restype = st
            L.bspl_project_curves_noalloc.argtypes = [C.POINTER(bspl_segments), i64, vp, vp, C.POINTER(bspl_options),
                                                      vp, vp, vp, vp]
            L.bspl_graph_begin.restype = st
            L.bspl_graph_begin.argtypes = [vp]
            L.bspl_graph_end.restype = st
            L.bspl_graph_end.argtypes = [vp, C.POINTER(vp), C.POINTER(i64)]
            L.bspl_graph_launch.restype = st
            L.bspl_graph_launch.argtypes = [vp, vp]
            L.bspl_graph_destroy.restype = None
            L.bspl_graph_destroy.argtypes = [vp]
            L.bspl_measure_fma_peak.restype = C.c_int
            L.bspl_measure_fma_peak.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), vp, vp]
            mp = C.POINTER(bspl_mlp)
            sp = C.POINTER(bspl_segments)
            f32 = C.c_float
            for name, args in (("bspl_mlp_check", [vp]), ("bspl_mlp_sync", [mp, vp]),
                               ("bspl_mlp_forward", [mp, i64, vp, vp, vp]),
                               ("bspl_mlp_features", [sp, i64, vp, vp, vp, vp, vp]),
                               ("bspl_mlp_labels", [sp, i64, vp, vp, vp, vp, vp]),
                               ("bspl_mlp_collect_pairs", [sp, i64, vp, vp, i64, vp, vp, vp, vp, C.c_size_t, vp]),
                               ("bspl_mlp_loss_grad", [mp, i64, vp, vp, vp, vp, vp, C.c_size_t, vp]),
                               ("bspl_mlp_adam", [mp, vp, vp, vp, C.c_int32, f32, f32, f32, f32, vp]),
                               ("bspl_mlp_train", [mp, vp, vp, i64, vp, vp, C.c_int32, C.c_int32, f32, C.c_uint64,
                                                   C.c_int32, vp, vp, C.c_size_t, vp]),
                               ("bspl_smlp_features", [sp, i64, vp, vp, vp, vp, vp]),
                               ("bspl_smlp_labels", [sp, i64, vp, vp, vp, vp, vp]),
                               ("bspl_smlp_collect_pairs", [sp, i64, vp, vp, i64, vp, vp, vp, vp, C.c_size_t, vp])):
                f = getattr(L, name)
                f.restype = st
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc, what, allow=(OK,)):
    if rc not in allow:
        name = lib().bspl_status_string(rc).decode()
        raise BsplError(f"{what} failed: {name} ({rc})")
    return rc


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(x, dtype, device):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype).to(device)


# ------------------------------------------------------------------ inputs

class DeviceCurves:
    """A CSR curve set (see synth.CurveSet) resident on the GPU; with a
    ``weights`` attribute that is not None (one weight per control point)
    the curves are rational."""

    def __init__(self, cs, device="cuda"):
        self.n = int(len(cs.degree))
        self.degree = _dev(cs.degree, torch.int32, device)
        self.knot_off = _dev(cs.knot_off, torch.int64, device)
        self.knots = _dev(cs.knots, torch.float64, device)
        self.cp_off = _dev(cs.cp_off, torch.int64, device)
        self.cps = _dev(np.asarray(cs.cps).reshape(-1, 3), torch.float64, device)
        w = getattr(cs, "weights", None)
        self.weights = None if w is None else _dev(np.asarray(w).reshape(-1), torch.float64, device)
        self.n_cp_total = int(cs.cp_off[-1])
        self.c = bspl_curves(self.n, _ptr(self.degree), _ptr(self.knot_off), _ptr(self.knots), _ptr(self.cp_off),
                             _ptr(self.cps), None if self.weights is None else _ptr(self.weights))


class DeviceSurfaces:
    """A CSR surface set (see synth.SurfaceSet) resident on the GPU."""

    def __init__(self, ss, device="cuda"):
        self.n = int(len(ss.deg_u))
        self.deg_u = _dev(ss.deg_u, torch.int32, device)
        self.deg_v = _dev(ss.deg_v, torch.int32, device)
        self.n_u = _dev(ss.n_u, torch.int32, device)
        self.n_v = _dev(ss.n_v, torch.int32, device)
        self.knot_u_off = _dev(ss.knot_u_off, torch.int64, device)
        self.knots_u = _dev(ss.knots_u, torch.float64, device)
        self.knot_v_off = _dev(ss.knot_v_off, torch.int64, device)
        self.knots_v = _dev(ss.knots_v, torch.float64, device)
        self.cp_off = _dev(ss.cp_off, torch.int64, device)
        self.cps = _dev(np.asarray(ss.cps).reshape(-1, 3), torch.float64, device)
        self.n_cp_total = int(ss.cp_off[-1])
        self.c = bspl_surfaces(self.n, _ptr(self.deg_u), _ptr(self.deg_v), _ptr(self.n_u), _ptr(self.n_v),
                               _ptr(self.knot_u_off), _ptr(self.knots_u), _ptr(self.knot_v_off),
                               _ptr(self.knots_v), _ptr(self.cp_off), _ptr(self.cps))


# ------------------------------------------------------------ decomposition

class Segments:
    """Decomposition output + query tables (torch tensors owned here)."""

    def __init__(self, splines, is_surface: bool, capacity: int, device="cuda"):
        n = splines.n
        self.is_surface = bool(is_surface)
        self.n = n
        self.capacity = int(capacity)
        cap = max(self.capacity, 1)
        self.grp_capacity = n + cap // GROUP + 1
        f64, f32, i64 = torch.float64, torch.float32, torch.int64
        z = lambda shape, dt: torch.zeros(shape, dtype=dt, device=device)
        self.seg_off = z(n + 1, i64)
        self.diag = z(n, f64)
        self.grp_off = z(n + 1, i64)
        if is_surface:
            self.ctrl = z((cap, 4, 4, 3), f64)
            self.prange = z((cap, 4), f64)
            self.rec64 = z((cap, SREC64), f64)
            self.rec32 = z((cap, SREC32), f32)
            self.patch_span = z(cap, i64)
            self.patch_box = z((cap, 4), f64)
            self.span_net = z((splines.n_cp_total, SPAN_NET), f64)
            self.span_net32 = z((splines.n_cp_total, SPAN_NET), f32)
            self.patch_net32 = z((cap, SPAN_NET), f32)
        else:
            self.ctrl = z((cap, 4, 3), f64)
            self.prange = z((cap, 2), f64)
            self.rec64 = z((cap, CREC64), f64)
            self.rec32 = z((cap, CREC32), f32)
            self.patch_span = self.patch_box = self.span_net = self.span_net32 = self.patch_net32 = None
        self.spline_rank = z(max(n, 1), torch.int32)
        self.grp64 = z((self.grp_capacity, GREC64), f64)
        self.grp32 = z((self.grp_capacity, GREC32), f32)
        self.n_cp_total = splines.n_cp_total
        self.total = 0
        self.tol_rel = 0.0
        self.c = self._struct()

    def _struct(self):
        return bspl_segments(int(self.is_surface), self.n, self.capacity, self.grp_capacity, _ptr(self.seg_off),
                             _ptr(self.ctrl), _ptr(self.prange), _ptr(self.diag), _ptr(self.rec64),
                             _ptr(self.rec32), _ptr(self.grp_off), _ptr(self.grp64), _ptr(self.grp32),
                             _ptr(self.patch_span), _ptr(self.patch_box), _ptr(self.span_net), _ptr(self.span_net32),
                             self.n_cp_total,
                             self.tol_rel, _ptr(self.patch_net32), _ptr(self.spline_rank))

    def view(self):
        """Host copies (seg_off, ctrl, prange) trimmed to the segment count."""
        k = self.total
        return self.seg_off.cpu().numpy(), self.ctrl[:k].cpu().numpy(), self.prange[:k].cpu().numpy()


def workspace_bytes(op, n_splines, n_cp_total, n_seg, n_q):
    return int(lib().bspl_workspace_bytes(op, n_splines, n_cp_total, n_seg, n_q))


def _ws(nbytes, device="cuda"):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def bspl_decompose(is_surface, splines, tol_rel, seg_struct, ws, stream=None):
    """Raw call: returns (status, n_seg_total)."""
    tot = C.c_int64(0)
    rc = lib().bspl_decompose(int(is_surface), C.byref(splines.c), float(tol_rel), C.byref(seg_struct),
                              C.byref(tot), _ptr(ws), ws.numel(), _stream(stream))
    return rc, tot.value


def decompose(splines, tol_rel: float, is_surface: bool | None = None, stream=None,
              allow_capped: bool = False) -> Segments:
    """Two-phase decomposition: count, allocate, fill.

    BSPL_ENOTCONV (a span or span pair reached the subdivision depth cap or
    its piece cap, so some accepted pieces exceed the tolerance) raises
    BsplError unless ``allow_capped``; the status is kept in ``segs.status``."""
    if is_surface is None:
        is_surface = isinstance(splines, DeviceSurfaces)
    op = OP_DECOMPOSE_SURFACES if is_surface else OP_DECOMPOSE_CURVES
    ws = _ws(workspace_bytes(op, splines.n, splines.n_cp_total, 0, 0), splines.cp_off.device)
    probe = Segments(splines, is_surface, 0, splines.cp_off.device)
    probe.c.ctrl = None
    rc, total = bspl_decompose(is_surface, splines, tol_rel, probe.c, ws, stream)
    ok = (OK, ENOTCONV) if allow_capped else (OK,)
    _check(rc, "bspl_decompose(count)", ok)
    segs = Segments(splines, is_surface, total, splines.cp_off.device)
    rc, total2 = bspl_decompose(is_surface, splines, tol_rel, segs.c, ws, stream)
    _check(rc, "bspl_decompose(fill)", ok)
    assert total2 == total
    segs.total = total
    segs.tol_rel = float(tol_rel)
    segs.status = rc
    segs.c = segs._struct()
    return segs


# ----------------------------------------------------------------- queries

@dataclass
class QueryResult:
    param: torch.Tensor  # t [n] (curves) or uv [n][2] (surfaces)
    dist: torch.Tensor
    status: torch.Tensor


def make_options(prec=FP64, samples=0, newton_max=0, fp32_steps=0, sort_queries=1, counters=None, mlp=None,
                 occupancy=0, stage_events=None, pairs_per_query=0, cert_depth=0):
    """mlp: an ``Mlp`` (learned seed for prec=LEARNED_MIXED) or None;
    stage_events: NSTAGE_EVENTS torch.cuda.Event(enable_timing=True) that the
    learned path records at its stage boundaries (profiling)."""
    ev = None
    if stage_events is not None:
        assert len(stage_events) == NSTAGE_EVENTS
        s = torch.cuda.current_stream()
        for e in stage_events:
            if not e.cuda_event:
                e.record(s)  # creates the event
        ev = (C.c_void_p * NSTAGE_EVENTS)(*[e.cuda_event for e in stage_events])
    o = bspl_options(int(prec), int(samples), int(newton_max), int(fp32_steps), int(sort_queries), int(occupancy),
                     int(pairs_per_query), C.cast(C.pointer(mlp.c), C.c_void_p) if mlp is not None else C.c_void_p(0),
                     _ptr(counters) if counters is not None else None,
                     C.cast(ev, C.c_void_p) if ev is not None else None, int(cert_depth))
    o._keep = (mlp, ev)  # what the pointers refer to stays alive with the options
    return o


class QueryBuffers:
    """Preallocated outputs + workspace for repeated query calls."""

    def __init__(self, segs: Segments, n_q: int, device="cuda", learned: bool = False):
        self.n_q = int(n_q)
        shape = (n_q, 2) if segs.is_surface else (n_q,)
        self.param = torch.empty(shape, dtype=torch.float64, device=device)
        self.dist = torch.empty(n_q, dtype=torch.float64, device=device)
        self.status = torch.empty(n_q, dtype=torch.uint8, device=device)
        if segs.is_surface:
            op = OP_QUERY_SURFACES_LEARNED if learned else OP_QUERY_SURFACES
        else:
            op = OP_QUERY_CURVES_LEARNED if learned else OP_QUERY_CURVES
        self.ws = _ws(workspace_bytes(op, segs.n, segs.n_cp_total, segs.total, n_q), device)


def _query(fn_name, segs, q_idx, q_xyz, opts, bufs, stream):
    L = lib()
    fn = getattr(L, fn_name)
    rc = fn(C.byref(segs.c), int(q_idx.numel()), _ptr(q_idx), _ptr(q_xyz), C.byref(opts), _ptr(bufs.param),
            _ptr(bufs.dist), _ptr(bufs.status), _ptr(bufs.ws), bufs.ws.numel(), _stream(stream))
    _check(rc, fn_name)
    return QueryResult(bufs.param, bufs.dist, bufs.status)


def _learned(opts):
    return opts is not None and opts.prec in (LEARNED_MIXED, CLIP_MIXED)


def bspl_project_curves(segs, q_curve, q_xyz, opts=None, bufs=None, stream=None):
    bufs = bufs or QueryBuffers(segs, q_curve.numel(), q_xyz.device, _learned(opts))
    return _query("bspl_project_curves", segs, q_curve, q_xyz, opts or make_options(), bufs, stream)


def bspl_invert_curves(segs, q_curve, q_xyz, opts=None, bufs=None, stream=None):
    bufs = bufs or QueryBuffers(segs, q_curve.numel(), q_xyz.device, _learned(opts))
    return _query("bspl_invert_curves", segs, q_curve, q_xyz, opts or make_options(), bufs, stream)


def bspl_project_surfaces(segs, q_surf, q_xyz, opts=None, bufs=None, stream=None):
    bufs = bufs or QueryBuffers(segs, q_surf.numel(), q_xyz.device, _learned(opts))
    return _query("bspl_project_surfaces", segs, q_surf, q_xyz, opts or make_options(), bufs, stream)


def bspl_invert_surfaces(segs, q_surf, q_xyz, opts=None, bufs=None, stream=None):
    bufs = bufs or QueryBuffers(segs, q_surf.numel(), q_xyz.device, _learned(opts))
    return _query("bspl_invert_surfaces", segs, q_surf, q_xyz, opts or make_options(), bufs, stream)


NOALLOC_MAX_QUERIES = 1 << 20
NOALLOC_MAX_SPLINES = 1 << 18
SCRATCH_BYTES = 8 << 20  # BSPL_NOALLOC_SCRATCH_BYTES


def bspl_project_curves_noalloc(segs, q_curve, q_xyz, opts=None, out=None, stream=None):
    """Projection through the scratch-free entry point: for callers that
    cannot give the library a workspace allocation (see include/bspl.h).
    ``out`` optionally holds preallocated (t, dist, status) tensors."""
    n = q_curve.numel()
    if out is None:
        out = (torch.empty(n, dtype=torch.float64, device=q_xyz.device),
               torch.empty(n, dtype=torch.float64, device=q_xyz.device),
               torch.empty(n, dtype=torch.uint8, device=q_xyz.device))
    t, d, st = out
    rc = lib().bspl_project_curves_noalloc(C.byref(segs.c), n, _ptr(q_curve), _ptr(q_xyz),
                                           C.byref(opts or make_options()), _ptr(t), _ptr(d), _ptr(st),
                                           _stream(stream))
    _check(rc, "bspl_project_curves_noalloc")
    return QueryResult(t, d, st)


class Graph:
    """Query calls captured once as a CUDA graph (include/bspl_graph.h) and
    replayed: ``with Graph(stream) as g: <calls on that stream>`` then
    ``g.replay()``.  ``n_kernels`` is the number of kernel launches a replay
    makes.  The calls must use preallocated buffers (a replay reads and writes
    the same device addresses).

    A graph released while a capture is open on this thread (for instance
    the one ``g`` held before ``with Graph() as g`` rebinds it, which happens
    after the new capture began) is destroyed when that capture ends:
    destroying it inside the capture would invalidate the capture."""

    _open = threading.local()

    @classmethod
    def _state(cls):
        st = cls._open
        if not hasattr(st, "depth"):
            st.depth, st.pending = 0, []
        return st

    def __init__(self, stream=None):
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.exec = C.c_void_p(0)
        self.n_kernels = 0
        self._ctx = None

    def __enter__(self):
        self._ctx = torch.cuda.stream(self.stream)
        self._ctx.__enter__()
        _check(lib().bspl_graph_begin(_stream(self.stream)), "bspl_graph_begin")
        Graph._state().depth += 1
        return self

    def __exit__(self, exc_type, exc, tb):
        n = C.c_int64(0)
        rc = lib().bspl_graph_end(_stream(self.stream), C.byref(self.exec), C.byref(n))
        st = Graph._state()
        st.depth -= 1
        if st.depth == 0:
            for ex in st.pending:
                lib().bspl_graph_destroy(ex)
            st.pending = []
        self._ctx.__exit__(exc_type, exc, tb)
        if exc_type is None:
            _check(rc, "bspl_graph_end")
        self.n_kernels = int(n.value)
        return False

    def replay(self, stream=None):
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().bspl_graph_launch(self.exec, _stream(s)), "bspl_graph_launch")

    def __del__(self):
        try:
            if self.exec and self.exec.value:
                st = Graph._state()
                if st.depth > 0:
                    st.pending.append(self.exec)
                else:
                    lib().bspl_graph_destroy(self.exec)
        except Exception:
            pass


def bspl_eval_curves(curves: DeviceCurves, q_curve, t, stream=None):
    out = torch.empty((q_curve.numel(), 3), dtype=torch.float64, device=t.device)
    rc = lib().bspl_eval_curves(C.byref(curves.c), q_curve.numel(), _ptr(q_curve), _ptr(t), _ptr(out),
                                _stream(stream))
    _check(rc, "bspl_eval_curves")
    return out


REFINE_EVALS = 64


def refine_workspace(curves: DeviceCurves, n_q: int, device="cuda"):
    """Workspace for bspl_refine_curves to group its n_q queries by curve."""
    return _ws(workspace_bytes(OP_REFINE_CURVES, curves.n, curves.n_cp_total, 0, n_q), device)


def bspl_refine_curves(curves: DeviceCurves, q_curve, q_xyz, res: "QueryResult", invert: bool = False,
                       diag=None, max_iter: int = 0, evals=None, ws=None, stream=None):
    """Refines a curve projection / inversion result in place on the
    original curves (include/bspl.h, bspl_refine_curves); diag: the per-curve
    diagonals (e.g. the segments' diag) for the OFF_CURVE bit of inversions;
    evals: optional int64 device tensor [REFINE_EVALS] accumulating the
    evaluations made per curve degree; ws: optional workspace
    (refine_workspace) with which the queries are processed grouped by curve."""
    rc = lib().bspl_refine_curves(C.byref(curves.c), _ptr(diag) if diag is not None else None, int(invert),
                                  q_curve.numel(), _ptr(q_curve), _ptr(q_xyz), int(max_iter), _ptr(res.param),
                                  _ptr(res.dist), _ptr(res.status), _ptr(evals) if evals is not None else None,
                                  _ptr(ws) if ws is not None else None, ws.numel() if ws is not None else 0,
                                  _stream(stream))
    _check(rc, "bspl_refine_curves")
    return res


def bspl_eval_surfaces(surfs: DeviceSurfaces, q_surf, uv, stream=None):
    out = torch.empty((q_surf.numel(), 3), dtype=torch.float64, device=uv.device)
    rc = lib().bspl_eval_surfaces(C.byref(surfs.c), q_surf.numel(), _ptr(q_surf), _ptr(uv), _ptr(out),
                                  _stream(stream))
    _check(rc, "bspl_eval_surfaces")
    return out


def measure_fma_peak(fp64: bool, iters: int = 4096, reps: int = 5, stream=None) -> float:
    """FP32 or FP64 FMA-chain throughput of the current GPU in FLOP/s."""
    sink = torch.zeros(2, dtype=torch.float64, device="cuda")
    out = C.c_double(0.0)
    rc = lib().bspl_measure_fma_peak(int(fp64), int(iters), int(reps), C.byref(out), _ptr(sink), _stream(stream))
    _check(rc, "bspl_measure_fma_peak")
    return out.value


# ------------------------------------------------------------ learned seed

class Mlp:
    """Parameters of a learned seed network on the GPU (include/bspl_mlp.h):
    FP32 master weights, the BF16 copy the kernels read, and Adam's moments.
    kind MLP_CURVE (16 -> 1) or MLP_SURFACE (64 -> 2)."""

    def __init__(self, params, device="cuda", kind=MLP_CURVE):
        self.kind = int(kind)
        self.n_in, self.n_out, npar, nbf, self.train_op = NET[self.kind]
        self.params = torch.tensor(np.array(params, np.float32)).to(device).contiguous()
        assert self.params.numel() == npar
        self.wbf16 = torch.zeros(nbf, dtype=torch.int16, device=device)
        self.adam_m = torch.zeros(npar, dtype=torch.float32, device=device)
        self.adam_v = torch.zeros(npar, dtype=torch.float32, device=device)
        self.step = 0
        self.c = bspl_mlp(self.params.data_ptr(), self.wbf16.data_ptr(), self.kind)
        self.sync()

    def sync(self, stream=None):
        _check(lib().bspl_mlp_sync(C.byref(self.c), _stream(stream)), "bspl_mlp_sync")

    def forward(self, X, stream=None):
        X = X.contiguous()
        shape = (X.shape[0],) if self.n_out == 1 else (X.shape[0], self.n_out)
        t = torch.empty(shape, dtype=torch.float32, device=X.device)
        _check(lib().bspl_mlp_forward(C.byref(self.c), X.shape[0], _ptr(X), _ptr(t), _stream(stream)),
               "bspl_mlp_forward")
        return t

    def loss_grad(self, X, y, stream=None):
        n = X.shape[0]
        grad = torch.empty(self.params.numel(), dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        ws = _ws(workspace_bytes(self.train_op, 0, 0, 0, n), X.device)
        _check(lib().bspl_mlp_loss_grad(C.byref(self.c), n, _ptr(X.contiguous()), _ptr(y.contiguous()), _ptr(grad),
                                        _ptr(loss), _ptr(ws), ws.numel(), _stream(stream)), "bspl_mlp_loss_grad")
        return loss, grad

    def adam(self, grad, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self.step += 1
        _check(lib().bspl_mlp_adam(C.byref(self.c), _ptr(grad), _ptr(self.adam_m), _ptr(self.adam_v), self.step,
                                   float(lr), float(beta1), float(beta2), float(eps), _stream(stream)),
               "bspl_mlp_adam")

    def train(self, X, y, epochs, batch=8192, lr=1e-3, seed=0, stream=None):
        """Returns the per-epoch mean loss (device tensor)."""
        n = X.shape[0]
        loss = torch.empty(epochs, dtype=torch.float32, device=X.device)
        ws = _ws(workspace_bytes(self.train_op, 0, 0, 0, batch), X.device)
        _check(lib().bspl_mlp_train(C.byref(self.c), _ptr(self.adam_m), _ptr(self.adam_v), n, _ptr(X.contiguous()),
                                    _ptr(y.contiguous()), int(epochs), int(batch), float(lr), int(seed) & (2**64 - 1),
                                    self.step, _ptr(loss), _ptr(ws), ws.numel(), _stream(stream)), "bspl_mlp_train")
        self.step += epochs * ((n + batch - 1) // batch)
        return loss

    # versioned checkpoint: magic, version, nparam, step, CRC32 of the payload,
    # then params, Adam m and v (FP32, little endian)
    _MAGIC = b"BSPLMLP\0"

    def save(self, path):
        import struct
        import zlib
        payload = b"".join(t.detach().cpu().numpy().astype("<f4").tobytes()
                           for t in (self.params, self.adam_m, self.adam_v))
        # version 1: the curve network; version 2: the surface network
        hdr = self._MAGIC + struct.pack("<IIqI", 1 + self.kind, self.params.numel(), self.step,
                                        zlib.crc32(payload))
        with open(path, "wb") as f:
            f.write(hdr + payload)

    @classmethod
    def load(cls, path, device="cuda"):
        import struct
        import zlib
        raw = open(path, "rb").read()
        if raw[:8] != cls._MAGIC:
            raise BsplError(f"{path}: not an MLP checkpoint")
        ver, npar, step, crc = struct.unpack("<IIqI", raw[8:28])
        payload = raw[28:]
        kind = ver - 1
        if kind not in NET or npar != NET[kind][2] or len(payload) != 12 * npar or zlib.crc32(payload) != crc:
            raise BsplError(f"{path}: corrupt or incompatible MLP checkpoint")
        a = np.frombuffer(payload, "<f4").reshape(3, npar)
        m = cls(a[0], device, kind)
        m.adam_m.copy_(torch.from_numpy(a[1].copy()))
        m.adam_v.copy_(torch.from_numpy(a[2].copy()))
        m.step = step
        return m


def mlp_check(stream=None):
    """BSPL_ETIMEOUT if a tensor-core wait gave up since the last check."""
    return lib().bspl_mlp_check(_stream(stream))


def bspl_mlp_features(segs, pair_q, pair_seg, q_xyz, stream=None):
    X = torch.empty((pair_q.numel(), MLP_IN), dtype=torch.float32, device=q_xyz.device)
    _check(lib().bspl_mlp_features(C.byref(segs.c), pair_q.numel(), _ptr(pair_q), _ptr(pair_seg), _ptr(q_xyz),
                                   _ptr(X), _stream(stream)), "bspl_mlp_features")
    return X


def bspl_mlp_labels(segs, pair_q, pair_seg, q_xyz, stream=None):
    y = torch.empty(pair_q.numel(), dtype=torch.float32, device=q_xyz.device)
    _check(lib().bspl_mlp_labels(C.byref(segs.c), pair_q.numel(), _ptr(pair_q), _ptr(pair_seg), _ptr(q_xyz),
                                 _ptr(y), _stream(stream)), "bspl_mlp_labels")
    return y


def bspl_mlp_collect_pairs(segs, q_curve, q_xyz, cap, stream=None):
    """(pair_q, pair_seg) of the seeded pairs written (at most cap) and the
    number of seeded pairs found."""
    dev = q_xyz.device
    pq = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    ps = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    n = torch.zeros(2, dtype=torch.int64, device=dev)
    ws = _ws(workspace_bytes(OP_QUERY_CURVES_LEARNED, segs.n, 0, 0, q_curve.numel()), dev)
    _check(lib().bspl_mlp_collect_pairs(C.byref(segs.c), q_curve.numel(), _ptr(q_curve), _ptr(q_xyz), int(cap),
                                        _ptr(pq), _ptr(ps), _ptr(n), _ptr(ws), ws.numel(), _stream(stream)),
           "bspl_mlp_collect_pairs")
    written, found = (int(v) for v in n.tolist())
    return pq[:written], ps[:written], found


# ------------------------------------------------------ surface seed network

def bspl_smlp_features(segs, pair_q, pair_patch, q_xyz, stream=None):
    X = torch.empty((pair_q.numel(), SMLP_IN), dtype=torch.float32, device=q_xyz.device)
    _check(lib().bspl_smlp_features(C.byref(segs.c), pair_q.numel(), _ptr(pair_q), _ptr(pair_patch), _ptr(q_xyz),
                                    _ptr(X), _stream(stream)), "bspl_smlp_features")
    return X


def bspl_smlp_labels(segs, pair_q, pair_patch, q_xyz, stream=None):
    uv = torch.empty((pair_q.numel(), 2), dtype=torch.float32, device=q_xyz.device)
    _check(lib().bspl_smlp_labels(C.byref(segs.c), pair_q.numel(), _ptr(pair_q), _ptr(pair_patch), _ptr(q_xyz),
                                  _ptr(uv), _stream(stream)), "bspl_smlp_labels")
    return uv


def bspl_smlp_collect_pairs(segs, q_surf, q_xyz, cap, stream=None):
    """(pair_q, pair_patch) of the (query, patch) pairs the learned surface
    path seeds (at most cap written) and the number found."""
    dev = q_xyz.device
    pq = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    pp = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    n = torch.zeros(2, dtype=torch.int64, device=dev)
    ws = _ws(workspace_bytes(OP_QUERY_SURFACES_LEARNED, segs.n, 0, 0, q_surf.numel()), dev)
    _check(lib().bspl_smlp_collect_pairs(C.byref(segs.c), q_surf.numel(), _ptr(q_surf), _ptr(q_xyz), int(cap),
                                         _ptr(pq), _ptr(pp), _ptr(n), _ptr(ws), ws.numel(), _stream(stream)),
           "bspl_smlp_collect_pairs")
    written, found = (int(v) for v in n.tolist())
    return pq[:written], pp[:written], found
