"""Thin Python binding of libd2.so (include/d2.h), same call names.

Argument marshalling only: every step of the assignment step runs in the
CUDA library.  Tensors are torch tensors (device or host) or numpy arrays
(host); pointers and sizes are passed straight through the C ABI.  If the
library cannot be loaded this module raises -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libd2.so")

D2_OK, D2_EINVAL, D2_ENOMEM, D2_ENOTCONVERGED = 0, -1, -2, -3
D2_ETIMEOUT, D2_ECUDA, D2_EUNSUPPORTED, D2_ENOCENTROIDS = -4, -5, -6, -7
D2_F64, D2_F32, D2_BF16 = 0, 1, 2
D2_PREC_AUTO, D2_PREC_FP64, D2_PREC_FP32, D2_PREC_TC = 0, 1, 2, 3
D2_TC_AUTO, D2_TC_OFF, D2_TC_ON = 0, 1, 2
D2_START_AUTO, D2_START_RANKED, D2_START_VOGEL = 0, 1, 2
D2_SEG_SLICES, D2_SEG_CONSTRAINED = 0, 1
D2_UPDATE_CONSTRAINED, D2_UPDATE_ALG1 = 0, 1
D2_CERTIFY_CANDIDATES, D2_CERTIFY_ALL = 0, 1
MAX_SUPPORT = 64

EXPORTS = ["d2_ctx_create", "d2_ctx_destroy", "d2_set_stream", "d2_sync", "d2_strerror",
           "d2_version", "d2_set_centroids", "d2_get_centroids", "d2_cost_matrix",
           "d2_mallows_batch", "d2_assign", "d2_update_locations", "d2_cluster_level",
           "d2_get_stats", "d2_update_locations_noalloc", "d2_server_create", "d2_server_submit",
           "d2_server_poll", "d2_server_stats", "d2_server_destroy", "d2_segment",
           "d2_set_cost_table", "d2_assign_multi", "d2_update_weights", "d2_cluster_level_ex",
           "d2_mallows_all"]


class D2Bags(ctypes.Structure):
    _fields_ = [("loc", ctypes.c_void_p), ("w", ctypes.c_void_p), ("off", ctypes.c_void_p),
                ("count", ctypes.c_int64), ("dim", ctypes.c_int32), ("loc_dtype", ctypes.c_int32),
                ("w_dtype", ctypes.c_int32), ("max_support", ctypes.c_int32)]


class D2Config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("pivot_budget", ctypes.c_int32),
                ("group_lanes", ctypes.c_int32), ("cost_tc", ctypes.c_int32),
                ("tile_budget_mib", ctypes.c_int32), ("start_rule", ctypes.c_int32),
                ("segmentation", ctypes.c_int32), ("split_iters", ctypes.c_int32),
                ("eps_tol", ctypes.c_double), ("centroid_update", ctypes.c_int32),
                ("joint_max_iter", ctypes.c_int32), ("joint_tol", ctypes.c_double),
                ("certify", ctypes.c_int32), ("tc_wait_probe", ctypes.c_int32),
                ("no_prune", ctypes.c_int32), ("joint_cold_start", ctypes.c_int32),
                ("warm_budget_mib", ctypes.c_int32)]


class D2Flows(ctypes.Structure):
    _fields_ = [("cell", ctypes.c_void_p), ("w", ctypes.c_void_p), ("stride", ctypes.c_int64)]


class D2Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("pairs_screened", ctypes.c_int64),
                ("pivots_screened", ctypes.c_int64), ("pairs_exact", ctypes.c_int64),
                ("pivots_exact", ctypes.c_int64), ("joint_rounds", ctypes.c_int64),
                ("joint_master_pivots", ctypes.c_int64), ("pairs_certified", ctypes.c_int64),
                ("cells_checked", ctypes.c_int64)]


class D2Error(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (%d)" % (what, strerror(code), code))
        self.code = code


_lib = None


def load(path=None):
    """Load libd2.so; raises OSError if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError("libd2.so not built: %s (run `python -m paper_1302_0435_gb300.build`)" % p)
    lib = ctypes.CDLL(p)
    vp = ctypes.c_void_p
    i64 = ctypes.c_int64
    i32 = ctypes.c_int32
    lib.d2_ctx_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(D2Config)]
    lib.d2_ctx_destroy.argtypes = [vp]
    lib.d2_set_stream.argtypes = [vp, vp]
    lib.d2_sync.argtypes = [vp]
    lib.d2_strerror.argtypes = [i32]
    lib.d2_strerror.restype = ctypes.c_char_p
    lib.d2_version.restype = ctypes.c_char_p
    lib.d2_set_centroids.argtypes = [vp, ctypes.POINTER(D2Bags)]
    lib.d2_get_centroids.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.d2_cost_matrix.argtypes = [vp, ctypes.POINTER(D2Bags), i64, i64, i32, vp]
    lib.d2_mallows_batch.argtypes = [vp, ctypes.POINTER(D2Bags), vp, vp, i64, vp,
                                     ctypes.POINTER(D2Flows), vp]
    lib.d2_assign.argtypes = [vp, ctypes.POINTER(D2Bags), vp, vp, vp, vp, ctypes.POINTER(D2Flows)]
    lib.d2_mallows_all.argtypes = [vp, ctypes.POINTER(D2Bags), vp, vp, vp]
    lib.d2_update_locations.argtypes = [vp, ctypes.POINTER(D2Bags), vp, vp, ctypes.POINTER(D2Flows)]
    lib.d2_cluster_level.argtypes = [vp, ctypes.POINTER(D2Bags), vp, i32, i64, i32, vp, vp, vp]
    lib.d2_get_stats.argtypes = [ctypes.POINTER(D2Stats)]
    lib.d2_segment.argtypes = [vp, ctypes.POINTER(D2Bags), vp, i64, i32, vp, ctypes.POINTER(i64)]
    lib.d2_set_cost_table.argtypes = [vp, vp, i32]
    lib.d2_assign_multi.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(D2Bags), vp, vp]
    lib.d2_update_weights.argtypes = [vp, ctypes.POINTER(D2Bags), vp, vp, i32, ctypes.c_double,
                                      vp, vp]
    lib.d2_cluster_level_ex.argtypes = [vp, ctypes.POINTER(D2Bags), vp, i32, i64, i32, vp, vp, vp,
                                        vp]
    lib.d2_server_create.argtypes = [ctypes.POINTER(vp), vp, i32, i64]
    lib.d2_server_submit.argtypes = [vp, ctypes.POINTER(D2Bags), ctypes.POINTER(i64)]
    lib.d2_server_poll.argtypes = [vp, i64, vp, vp, ctypes.POINTER(ctypes.c_double), i32]
    lib.d2_server_stats.argtypes = [vp, vp, vp, vp, vp]
    lib.d2_server_destroy.argtypes = [vp]
    lib.d2_update_locations_noalloc.argtypes = [ctypes.POINTER(D2Bags), vp, vp, ctypes.POINTER(D2Flows),
                                                i64, vp, i32, vp, vp, vp]
    _lib = lib
    return lib


def strerror(code):
    return load().d2_strerror(int(code)).decode()


def _ptr(x):
    """Raw address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr()


def _check(rc, what):
    if rc != D2_OK:
        raise D2Error(rc, what)


_DT = {"f64": D2_F64, "f32": D2_F32, "bf16": D2_BF16}


class BagsRef:
    """A bag batch as the C ABI sees it, holding references to its arrays.
    max_support: the largest bag's support count if known (0: the library
    scans the offsets, which waits for the stream)."""

    def __init__(self, loc, w, off, count, dim, loc_dtype, w_dtype, max_support=0):
        self.loc, self.w, self.off = loc, w, off
        self.s = D2Bags(_ptr(loc), _ptr(w), _ptr(off), int(count), int(dim), int(loc_dtype),
                        int(w_dtype), int(max_support))

    @property
    def count(self):
        return self.s.count


def bags_from_synth(b, device=None, pinned=False):
    """Marshal a synth.Bags into host numpy arrays (device=None), pinned host
    tensors (pinned=True) or device tensors (device='cuda:0')."""
    if b.loc_dtype == "bf16":
        loc_np = np.ascontiguousarray(b.loc_bits.view(np.int16))
    else:
        loc_np = np.ascontiguousarray(b.loc)
    w_np = np.ascontiguousarray(b.w)
    off_np = np.ascontiguousarray(b.off.astype(np.int64))
    # the largest bag, declared so that calls need not scan the offsets (only
    # when every bag fits the kernels; otherwise the library's scan reports it)
    sizes = np.diff(off_np)
    mx = int(sizes.max()) if sizes.size else 0
    ms = mx if 1 <= mx <= MAX_SUPPORT and sizes.min() >= 1 else 0
    if device is None and not pinned:
        return BagsRef(loc_np, w_np, off_np, b.count, b.dim, _DT[b.loc_dtype], _DT[b.w_dtype], ms)
    import torch
    tl = torch.from_numpy(loc_np)
    if b.loc_dtype == "bf16":
        tl = tl.view(torch.bfloat16)
    tw, to = torch.from_numpy(w_np), torch.from_numpy(off_np)
    if pinned:
        tl, tw, to = tl.pin_memory(), tw.pin_memory(), to.pin_memory()
    else:
        tl, tw, to = tl.to(device), tw.to(device), to.to(device)
    return BagsRef(tl, tw, to, b.count, b.dim, _DT[b.loc_dtype], _DT[b.w_dtype], ms)


class Context:
    """d2_ctx_create / d2_ctx_destroy."""

    def __init__(self, device=0, precision=D2_PREC_AUTO, pivot_budget=0, group_lanes=0,
                 cost_tc=D2_TC_AUTO, tile_budget_mib=0, start_rule=D2_START_AUTO,
                 segmentation=D2_SEG_SLICES, split_iters=0, eps_tol=0.0,
                 centroid_update=D2_UPDATE_CONSTRAINED, joint_max_iter=0, joint_tol=0.0,
                 certify=D2_CERTIFY_CANDIDATES, tc_wait_probe=0, no_prune=False,
                 joint_cold_start=False, warm_budget_mib=0):
        lib = load()
        self.h = ctypes.c_void_p()
        cfg = D2Config(precision, pivot_budget, group_lanes, cost_tc, tile_budget_mib, start_rule,
                       segmentation, split_iters, float(eps_tol), int(centroid_update),
                       int(joint_max_iter), float(joint_tol), int(certify), int(tc_wait_probe),
                       int(bool(no_prune)), int(bool(joint_cold_start)), int(warm_budget_mib))
        _check(lib.d2_ctx_create(ctypes.byref(self.h), int(device), ctypes.byref(cfg)), "d2_ctx_create")
        self._cents = None

    def close(self):
        if self.h:
            load().d2_ctx_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def d2_set_stream(ctx, stream):
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    h = getattr(stream, "cuda_stream", stream)
    _check(load().d2_set_stream(ctx.h, h), "d2_set_stream")


def d2_sync(ctx):
    _check(load().d2_sync(ctx.h), "d2_sync")


def d2_set_centroids(ctx, cents):
    ref = cents if isinstance(cents, BagsRef) else bags_from_synth(cents)
    _check(load().d2_set_centroids(ctx.h, ctypes.byref(ref.s)), "d2_set_centroids")


def d2_get_centroids(ctx, dim):
    """Resident centroids as numpy (loc [T, dim] f64, w [T] f64, off [K+1])."""
    lib = load()
    k = ctypes.c_int64()
    t = ctypes.c_int64()
    _check(lib.d2_get_centroids(ctx.h, None, None, None, ctypes.byref(k), ctypes.byref(t)),
           "d2_get_centroids")
    loc = np.empty((t.value, dim))
    w = np.empty(t.value)
    off = np.empty(k.value + 1, dtype=np.int64)
    _check(lib.d2_get_centroids(ctx.h, _ptr(loc), _ptr(w), _ptr(off), None, None), "d2_get_centroids")
    return loc, w, off


def d2_get_centroids_into(ctx, loc_out):
    """Resident centroid locations into a caller buffer ([T, dim] float64,
    host or device)."""
    _check(load().d2_get_centroids(ctx.h, _ptr(loc_out), None, None, None, None),
           "d2_get_centroids")


def d2_cost_matrix(ctx, objs, i, j, precision, m, n):
    C = np.empty((m, n))
    _check(load().d2_cost_matrix(ctx.h, ctypes.byref(objs.s), int(i), int(j), int(precision), _ptr(C)),
           "d2_cost_matrix")
    return C


def _flows(flows):
    if flows is None:
        return None
    cell, w = flows
    stride = cell.shape[-1]
    return D2Flows(_ptr(cell), _ptr(w), stride)


def d2_mallows_batch(ctx, objs, pair_obj, pair_cen, dist2, flows=None, status=None):
    """dist2/status/flows are caller buffers (torch or numpy); flows = (cell, w)
    with shape [npairs, stride].  Returns the status code (raises on errors
    other than D2_ENOTCONVERGED)."""
    f = _flows(flows)
    rc = load().d2_mallows_batch(ctx.h, ctypes.byref(objs.s), _ptr(pair_obj), _ptr(pair_cen),
                                 int(len(pair_obj)), _ptr(dist2), ctypes.byref(f) if f else None,
                                 _ptr(status))
    if rc not in (D2_OK, D2_ENOTCONVERGED):
        _check(rc, "d2_mallows_batch")
    return rc


def d2_assign(ctx, objs, labels, dist2, omega=None, eps=None, flows=None):
    f = _flows(flows)
    rc = load().d2_assign(ctx.h, ctypes.byref(objs.s), _ptr(omega), _ptr(labels), _ptr(dist2),
                          _ptr(eps), ctypes.byref(f) if f else None)
    if rc not in (D2_OK, D2_ENOTCONVERGED):
        _check(rc, "d2_assign")
    return rc


def d2_mallows_all(ctx, objs, dist2_all, labels=None, dist2=None):
    """D^2 of every (object, resident centroid) pair into dist2_all [N, K]
    (FP64, certified), plus the argmin labels / dist2 if given."""
    rc = load().d2_mallows_all(ctx.h, ctypes.byref(objs.s), _ptr(dist2_all), _ptr(labels),
                               _ptr(dist2))
    if rc not in (D2_OK, D2_ENOTCONVERGED):
        _check(rc, "d2_mallows_all")
    return rc


def d2_update_locations(ctx, objs, labels, omega=None, flows=None):
    f = _flows(flows)
    rc = load().d2_update_locations(ctx.h, ctypes.byref(objs.s), _ptr(omega), _ptr(labels),
                                    ctypes.byref(f) if f else None)
    if rc not in (D2_OK, D2_ENOTCONVERGED):
        _check(rc, "d2_update_locations")
    return rc


def d2_update_weights(ctx, objs, labels, max_iter=512, tol=1e-9, omega=None, eps=None,
                      iters=None):
    """Alg. 1 Step 1: resident centroid weights from the joint LP of
    Eq. (WeightedD2).  eps [K] float64 / iters [K] int32 outputs are
    optional.  Returns D2_OK, or D2_ENOTCONVERGED if a cluster was not
    certified within max_iter rounds."""
    rc = load().d2_update_weights(ctx.h, ctypes.byref(objs.s), _ptr(omega), _ptr(labels),
                                  int(max_iter), float(tol), _ptr(eps), _ptr(iters))
    if rc not in (D2_OK, D2_ENOTCONVERGED):
        _check(rc, "d2_update_weights")
    return rc


def d2_cluster_level(ctx, objs, K, seg_size, iters, out_loc, out_cent_weight, labels, omega=None):
    rc = load().d2_cluster_level(ctx.h, ctypes.byref(objs.s), _ptr(omega), int(K), int(seg_size),
                                 int(iters), _ptr(out_loc), _ptr(out_cent_weight), _ptr(labels))
    if rc not in (D2_OK, D2_ENOTCONVERGED):
        _check(rc, "d2_cluster_level")
    return rc


def d2_cluster_level_ex(ctx, objs, K, seg_size, iters, out_loc, out_support_w, out_cent_weight,
                        labels, omega=None):
    rc = load().d2_cluster_level_ex(ctx.h, ctypes.byref(objs.s), _ptr(omega), int(K),
                                    int(seg_size), int(iters), _ptr(out_loc), _ptr(out_support_w),
                                    _ptr(out_cent_weight), _ptr(labels))
    if rc not in (D2_OK, D2_ENOTCONVERGED):
        _check(rc, "d2_cluster_level_ex")
    return rc


def d2_set_cost_table(ctx, table):
    """Symbol ground costs: table [A, A] FP64 (numpy or tensor); None removes."""
    if table is None:
        _check(load().d2_set_cost_table(ctx.h, None, 0), "d2_set_cost_table")
        return
    if isinstance(table, np.ndarray):
        table = np.ascontiguousarray(table, dtype=np.float64)
    A = int(table.shape[0])
    _check(load().d2_set_cost_table(ctx.h, _ptr(table), A), "d2_set_cost_table")


def d2_assign_multi(ctxs, objs_list, labels, dist2):
    """Combined distance of several bag types: ctxs[b] holds type b's
    centroids, objs_list[b] type b's bags (BagsRef)."""
    B = len(ctxs)
    hs = (ctypes.c_void_p * B)(*[c.h for c in ctxs])
    bags = (D2Bags * B)(*[o.s for o in objs_list])
    rc = load().d2_assign_multi(hs, B, bags, _ptr(labels), _ptr(dist2))
    if rc not in (D2_OK, D2_ENOTCONVERGED):
        _check(rc, "d2_assign_multi")
    return rc


def d2_segment(ctx, objs, tau, iters, omega=None, seg_id=None):
    """Initial data segmentation (Alg. 3 Step 1).  Returns (seg_id array,
    number of segments); seg_id may be a caller buffer (numpy or device
    tensor of int32)."""
    out = seg_id if seg_id is not None else np.empty(objs.count, dtype=np.int32)
    m = ctypes.c_int64()
    _check(load().d2_segment(ctx.h, ctypes.byref(objs.s), _ptr(omega), int(tau), int(iters),
                             _ptr(out), ctypes.byref(m)), "d2_segment")
    return out, m.value


def d2_get_stats():
    st = D2Stats()
    _check(load().d2_get_stats(ctypes.byref(st)), "d2_get_stats")
    return {k: int(getattr(st, k)) for k in ("kernel_launches", "pairs_screened", "pivots_screened",
                                              "pairs_exact", "pivots_exact", "joint_rounds",
                                              "joint_master_pivots", "pairs_certified",
                                              "cells_checked")}


def d2_update_locations_noalloc(objs, labels, flows, K, cent_off, cent_loc_dtype, cent_loc64,
                                cent_loc32, omega=None, stream=None):
    """Allocation-free location update on caller-owned device centroid
    arrays (see include/d2.h).  All tensors must be on the device."""
    f = _flows(flows)
    h = getattr(stream, "cuda_stream", stream)
    rc = load().d2_update_locations_noalloc(ctypes.byref(objs.s), _ptr(omega), _ptr(labels),
                                            ctypes.byref(f), int(K), _ptr(cent_off),
                                            int(cent_loc_dtype), _ptr(cent_loc64), _ptr(cent_loc32), h)
    _check(rc, "d2_update_locations_noalloc")
    return rc


class Server:
    """d2_server_*: continuous batching of assignment requests against the
    context's resident centroids."""

    def __init__(self, ctx, slots=8, mem_budget=0):
        self.h = ctypes.c_void_p()
        _check(load().d2_server_create(ctypes.byref(self.h), ctx.h, int(slots), int(mem_budget)),
               "d2_server_create")
        self.ctx = ctx
        self._keep = {}

    def submit(self, bags):
        """bags: host BagsRef (numpy arrays); returns a ticket."""
        t = ctypes.c_int64()
        _check(load().d2_server_submit(self.h, ctypes.byref(bags.s), ctypes.byref(t)), "d2_server_submit")
        self._keep[t.value] = bags.count
        return t.value

    def poll(self, ticket, timeout_ms=-1):
        """Returns (status, labels, dist2, latency_ms); status D2_ETIMEOUT
        means not done yet."""
        n = self._keep[ticket]
        lab = np.empty(n, dtype=np.int32)
        d2v = np.empty(n)
        lat = ctypes.c_double()
        rc = load().d2_server_poll(self.h, int(ticket), _ptr(lab), _ptr(d2v), ctypes.byref(lat),
                                   int(timeout_ms))
        if rc == D2_ETIMEOUT:
            return rc, None, None, None
        del self._keep[ticket]
        return rc, lab, d2v, lat.value

    def stats(self):
        v = [ctypes.c_int64() for _ in range(4)]
        _check(load().d2_server_stats(self.h, *[ctypes.byref(x) for x in v]), "d2_server_stats")
        return dict(zip(["admitted", "completed", "peak_inflight", "queued"], [x.value for x in v]))

    def close(self):
        if self.h:
            load().d2_server_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
