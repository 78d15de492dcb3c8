"""Thin ctypes binding of the C ABI in ``include/frw.h``.

Functions carry the C names and only marshal arguments; every step of the walk
runs in ``libfrw.so`` (CUDA kernels for sm_103a).  There is no CPU path: if the
library cannot be built or loaded, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import json
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_uint8, c_uint32, c_uint64, c_void_p

import numpy as np

from . import build as _build

(FRW_OK, FRW_EINVAL, FRW_ENOMEM, FRW_ETIMEOUT, FRW_EDEVICE, FRW_ENOTCONV, FRW_ECAPACITY, FRW_ENOTFOUND,
 FRW_ECANCELED) = range(9)
FRW_FP64_GEOM, FRW_FP32_GEOM = 0, 1
FRW_TRANSITION_MICROWALK, FRW_TRANSITION_FDM = 0, 1
FRW_FDM_MAX_N = 24
FRW_TAB_SGF, FRW_TAB_FLUX_PAR, FRW_TAB_FLUX_PERP, FRW_TAB_SGF_HOM, FRW_TAB_FLUX_HOM = range(5)

EXPORTS = ("frw_default_options", "frw_create", "frw_destroy", "frw_set_stream", "frw_load_structure",
           "frw_unload_structure", "frw_extract", "frw_extract_batch", "frw_walk_records",
           "frw_microwalk_cubes", "frw_microwalk_cubes_noalloc", "frw_table", "frw_strerror", "frw_last_error",
           "frw_submit", "frw_poll", "frw_wait", "frw_plan_create", "frw_plan_run", "frw_plan_destroy",
           "frw_get_tuning", "frw_set_tuning", "frw_autotune", "frw_extract_sums", "frw_extract_matrix",
           "frw_cancel", "frw_get_serve_info", "frw_fdm_cubes", "frw_load_structure_boxes",
           "frw_extract_batch_sums", "frw_load_structure_ex")


class frw_box(ctypes.Structure):
    _fields_ = [("lo", c_double * 3), ("hi", c_double * 3)]


class frw_block(ctypes.Structure):
    _fields_ = [("lo", c_double * 3), ("hi", c_double * 3), ("mat", c_int32), ("reserved", c_int32)]


FRW_VOXEL_NONE = 255


class frw_structure(ctypes.Structure):
    _fields_ = [("domain", frw_box), ("grounded_walls", c_int32), ("n_boxes", c_int32), ("n_cond", c_int32),
                ("n_mat", c_int32), ("background_mat", c_int32), ("n_blocks", c_int32),
                ("vox_dims", c_int32 * 3), ("reserved", c_int32),
                ("boxes", c_void_p), ("box_conductor", c_void_p), ("eps_r", c_void_p), ("blocks", c_void_p),
                ("voxel_mat", c_void_p)]


class frw_options(ctypes.Structure):
    _fields_ = [("N", c_int32), ("precision", c_int32), ("seed", c_uint64), ("first_cube_mode", c_int32),
                ("hybrid", c_int32), ("gauss_offset_frac", c_double), ("max_hops", c_int32),
                ("slots", c_int32), ("table_capacity", c_int32), ("mw_warps_per_cta", c_int32),
                ("mw_ctas_per_sm", c_int32), ("geom_threads", c_int32), ("serve_jobs", c_int32),
                ("serve_arena_mb", c_int32), ("mwe_factor", c_int32), ("idle_timeout_ms", c_int32),
                ("transition", c_int32), ("reserved", c_int32)]


class frw_extract_params(ctypes.Structure):
    _fields_ = [("walk_budget", c_uint64), ("sigma_target", c_double), ("request_id", c_uint64),
                ("batch", c_uint64), ("walk_begin", c_uint64)]


class frw_job(ctypes.Structure):
    _fields_ = [("structure_id", c_int32), ("master", c_int32), ("walk_budget", c_uint64),
                ("sigma_target", c_double), ("request_id", c_uint64), ("batch", c_uint64)]


class frw_tuning(ctypes.Structure):
    _fields_ = [("pool_per_cta", c_int32), ("hops_per_epoch", c_int32), ("suspend_lanes", c_int32),
                ("mw_warps_per_cta", c_int32), ("mw_ctas_per_sm", c_int32), ("suspend_min_steps", c_int32),
                ("geo_warps", c_int32), ("unstaged", c_int32),
                ("walks_per_s", c_double), ("mw_steps_per_s", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class frw_serve_info(ctypes.Structure):
    _fields_ = [("submitted", c_uint64), ("completed", c_uint64), ("cancelled", c_uint64), ("refused", c_uint64),
                ("runs", c_uint64), ("runs_failed", c_uint64), ("last_status", c_uint32), ("reserved", c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class frw_stats(ctypes.Structure):
    _fields_ = [("walks", c_uint64), ("hops", c_uint64), ("micro_steps", c_uint64), ("truncated", c_uint64),
                ("branch", c_uint64 * 3), ("strat_hops", c_uint64), ("hom_hops", c_uint64),
                ("mw_hops", c_uint64), ("tables_built", c_uint64), ("rounds", c_uint64), ("seconds", c_double),
                ("geom_ms", c_double), ("fill_ms", c_double), ("mw_ms", c_double), ("launches", c_uint64),
                ("mw_jobs", c_uint64), ("walks_issued", c_uint64), ("kernel_ms", c_double),
                ("reduce_ms", c_double), ("stage_bytes", c_uint64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "branch"}
        d["branch"] = list(self.branch)
        return d


class FRWError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"frw error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load (building in-tree if needed) libfrw.so and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build(checked=os.environ.get("FRW_CHECKED") == "1")
    L = ctypes.CDLL(path)
    P = POINTER
    L.frw_default_options.argtypes = [P(frw_options)]
    L.frw_default_options.restype = None
    L.frw_create.argtypes = [P(c_void_p), c_int, P(frw_options)]
    L.frw_destroy.argtypes = [c_void_p]
    L.frw_destroy.restype = None
    L.frw_set_stream.argtypes = [c_void_p, c_void_p]
    L.frw_load_structure.argtypes = [c_void_p, P(frw_box), P(frw_box), c_int32, P(c_double), c_int32, c_int32,
                                     P(frw_block), c_int32, P(c_int32)]
    L.frw_load_structure_ex.argtypes = [c_void_p, POINTER(frw_structure), POINTER(c_int32)]
    L.frw_load_structure_boxes.argtypes = [c_void_p, P(frw_box), P(frw_box), P(c_int32), c_int32, c_int32,
                                           P(c_double), c_int32, c_int32, P(frw_block), c_int32, P(c_int32)]
    L.frw_unload_structure.argtypes = [c_void_p, c_int32]
    L.frw_extract.argtypes = [c_void_p, c_int32, c_int32, P(frw_extract_params), P(c_double), P(c_double),
                              P(frw_stats)]
    L.frw_extract_batch.argtypes = [c_void_p, P(frw_job), c_int32, P(c_double), P(c_double), P(frw_stats)]
    L.frw_walk_records.argtypes = [c_void_p, c_int32, c_int32, c_uint64, c_uint64, c_uint64, P(c_double),
                                   P(c_int32), P(c_uint32), P(c_uint64), P(c_int32)]
    L.frw_microwalk_cubes.argtypes = [c_void_p, c_int32, c_int32, c_void_p, P(c_double), c_int32, c_uint64,
                                      c_uint64, c_void_p, c_void_p]
    L.frw_microwalk_cubes_noalloc.argtypes = [c_int32, c_int32, c_void_p, P(c_double), c_int32, c_uint64, c_uint64,
                                              c_uint64, c_void_p, c_void_p, c_void_p]
    L.frw_fdm_cubes.argtypes = [c_void_p, c_int32, c_int32, c_void_p, P(c_double), c_int32, c_void_p, c_void_p,
                                c_void_p, c_void_p]
    L.frw_table.argtypes = [c_void_p, c_int32, P(c_int32), P(c_double), c_int32, P(c_uint32), P(c_uint8),
                            P(c_double), P(c_double)]
    L.frw_submit.argtypes = [c_void_p, POINTER(frw_job), POINTER(c_uint64)]
    L.frw_poll.argtypes = [c_void_p, c_uint64, POINTER(c_int32)]
    L.frw_cancel.argtypes = [c_void_p, c_uint64]
    L.frw_get_serve_info.argtypes = [c_void_p, POINTER(frw_serve_info)]
    L.frw_wait.argtypes = [c_void_p, c_uint64, c_double, P(c_double), P(c_double), POINTER(frw_stats)]
    L.frw_plan_create.argtypes = [c_void_p, POINTER(frw_job), c_int32, POINTER(c_void_p)]
    L.frw_plan_run.argtypes = [c_void_p, c_uint64, P(c_double), P(c_double), POINTER(frw_stats)]
    L.frw_plan_destroy.argtypes = [c_void_p]
    L.frw_plan_destroy.restype = None
    L.frw_get_tuning.argtypes = [c_void_p, POINTER(frw_tuning)]
    L.frw_set_tuning.argtypes = [c_void_p, POINTER(frw_tuning)]
    L.frw_autotune.argtypes = [c_void_p, POINTER(frw_job), c_int32, c_uint64, POINTER(frw_tuning)]
    L.frw_extract_sums.argtypes = [c_void_p, c_int32, c_int32, POINTER(frw_extract_params), P(c_uint64),
                                   POINTER(c_uint64), POINTER(frw_stats)]
    L.frw_extract_batch_sums.argtypes = [c_void_p, c_int32, c_int32, POINTER(frw_extract_params), P(c_uint64),
                                         P(c_uint64), POINTER(frw_stats)]
    L.frw_extract_matrix.argtypes = [c_void_p, c_int32, POINTER(frw_extract_params), P(c_double), P(c_double),
                                     P(c_double), POINTER(frw_stats)]
    L.frw_strerror.argtypes = [c_int]
    L.frw_strerror.restype = ctypes.c_char_p
    L.frw_last_error.argtypes = [c_void_p]
    L.frw_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("frw_default_options", "frw_destroy", "frw_strerror", "frw_last_error", "frw_plan_destroy"):
            getattr(L, name).restype = c_int
    _lib = L
    return L


def _ptr(a, ct):
    return a.ctypes.data_as(POINTER(ct)) if a is not None else None


def _check(ctx, rc, allow=(FRW_OK,)):
    if rc not in allow:
        msg = lib().frw_last_error(ctx).decode() if ctx else ""
        raise FRWError(rc, (lib().frw_strerror(rc).decode() + (": " + msg if msg else "")))
    return rc


# ---------------------------------------------------------------------------
def frw_strerror(code: int) -> str:
    return lib().frw_strerror(code).decode()


def frw_last_error(ctx) -> str:
    return lib().frw_last_error(ctx).decode()


def frw_default_options(**kw) -> frw_options:
    o = frw_options()
    lib().frw_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def frw_create(device: int = 0, options: frw_options | None = None):
    ctx = c_void_p()
    rc = lib().frw_create(ctypes.byref(ctx), int(device), ctypes.byref(options) if options is not None else None)
    _check(None, rc)
    return ctx


def frw_destroy(ctx) -> None:
    lib().frw_destroy(ctx)


def frw_set_stream(ctx, stream_handle: int | None) -> None:
    _check(ctx, lib().frw_set_stream(ctx, c_void_p(stream_handle or 0)))


def frw_load_structure(ctx, s) -> int:
    """Load a :class:`workloads.Structure` (host arrays are copied); structures
    with multi-box conductors go through frw_load_structure_boxes."""
    dom = frw_box((c_double * 3)(*s.domain_lo), (c_double * 3)(*s.domain_hi))
    cond = (frw_box * s.n_boxes)()
    for k in range(s.n_boxes):
        cond[k].lo = (c_double * 3)(*s.cond_lo[k])
        cond[k].hi = (c_double * 3)(*s.cond_hi[k])
    blk = (frw_block * max(1, s.n_blocks))()
    for b in range(s.n_blocks):
        blk[b].lo = (c_double * 3)(*s.block_lo[b])
        blk[b].hi = (c_double * 3)(*s.block_hi[b])
        blk[b].mat = int(s.block_mat[b])
    eps = np.ascontiguousarray(s.eps, np.float64)
    sid = c_int32(-1)
    vm = getattr(s, "voxel_mat", None)
    if vm is not None:
        vm = np.ascontiguousarray(vm, np.uint8)
        cid = None if s.cond_id is None else np.ascontiguousarray(s.cond_id, np.int32)
        d = frw_structure()
        d.domain = dom
        d.grounded_walls = 1
        d.n_boxes, d.n_cond = s.n_boxes, s.n_cond
        d.n_mat, d.background_mat = len(eps), int(s.background)
        d.n_blocks = s.n_blocks
        d.vox_dims = (c_int32 * 3)(*vm.shape)
        d.boxes = ctypes.cast(cond, c_void_p)
        d.box_conductor = None if cid is None else cid.ctypes.data
        d.eps_r = eps.ctypes.data
        d.blocks = ctypes.cast(blk, c_void_p)
        d.voxel_mat = vm.ctypes.data
        _check(ctx, lib().frw_load_structure_ex(ctx, ctypes.byref(d), ctypes.byref(sid)))
        return sid.value
    if s.cond_id is None:
        rc = lib().frw_load_structure(ctx, ctypes.byref(dom), cond, s.n_cond, _ptr(eps, c_double), len(eps),
                                      int(s.background), blk, s.n_blocks, ctypes.byref(sid))
    else:
        cid = np.ascontiguousarray(s.cond_id, np.int32)
        rc = lib().frw_load_structure_boxes(ctx, ctypes.byref(dom), cond, _ptr(cid, c_int32), s.n_boxes, s.n_cond,
                                            _ptr(eps, c_double), len(eps), int(s.background), blk, s.n_blocks,
                                            ctypes.byref(sid))
    _check(ctx, rc)
    return sid.value


def frw_unload_structure(ctx, sid: int) -> None:
    _check(ctx, lib().frw_unload_structure(ctx, int(sid)))


def frw_extract(ctx, sid: int, master: int, n_cond: int, walk_budget: int, sigma_target: float = 0.0,
                request_id: int = 0, batch: int = 0, walk_begin: int = 0):
    """-> (C row [n_cond+1], stderr row, stats dict, converged flag)."""
    p = frw_extract_params(int(walk_budget), float(sigma_target), int(request_id), int(batch), int(walk_begin))
    C = np.zeros(n_cond + 1)
    se = np.zeros(n_cond + 1)
    st = frw_stats()
    rc = lib().frw_extract(ctx, int(sid), int(master), ctypes.byref(p), _ptr(C, c_double), _ptr(se, c_double),
                           ctypes.byref(st))
    _check(ctx, rc, (FRW_OK, FRW_ENOTCONV))
    return C, se, st.as_dict(), rc == FRW_OK


def frw_extract_sums(ctx, sid: int, master: int, n_cond: int, walk_budget: int, request_id: int = 0,
                     batch: int = 0, walk_begin: int = 0):
    """-> (exact sums as 4 (n_cond + 1) uint64 words, walks counted, stats); budget mode."""
    p = frw_extract_params(int(walk_budget), 0.0, int(request_id), int(batch), int(walk_begin))
    words = np.zeros(4 * (n_cond + 1), np.uint64)
    n = c_uint64(0)
    st = frw_stats()
    _check(ctx, lib().frw_extract_sums(ctx, int(sid), int(master), ctypes.byref(p), _ptr(words, c_uint64),
                                       ctypes.byref(n), ctypes.byref(st)))
    return words, int(n.value), st.as_dict()


def frw_extract_batch_sums(ctx, sid: int, master: int, n_cond: int, walk_budget: int, request_id: int = 0,
                           batch: int = 0, walk_begin: int = 0):
    """-> (per-batch exact sums, shape (n_batches, 4 (n_cond + 1)) uint64, walks per
    batch, stats); budget mode, walk_begin a multiple of the batch size."""
    b = int(batch) if batch else 16384
    nb = (int(walk_budget) + b - 1) // b
    p = frw_extract_params(int(walk_budget), 0.0, int(request_id), int(batch), int(walk_begin))
    words = np.zeros((max(nb, 1), 4 * (n_cond + 1)), np.uint64)
    cnt = np.zeros(max(nb, 1), np.uint64)
    st = frw_stats()
    _check(ctx, lib().frw_extract_batch_sums(ctx, int(sid), int(master), ctypes.byref(p), _ptr(words, c_uint64),
                                             _ptr(cnt, c_uint64), ctypes.byref(st)))
    return words[:nb], cnt[:nb], st.as_dict()


def frw_extract_matrix(ctx, sid: int, n_cond: int, walk_budget: int, sigma_target: float = 0.0,
                       request_id: int = 0, batch: int = 0):
    """-> (C (n, n+1), stderr (n, n+1), C_sym (n, n), stats list, all converged)."""
    p = frw_extract_params(int(walk_budget), float(sigma_target), int(request_id), int(batch), 0)
    C = np.zeros((n_cond, n_cond + 1))
    se = np.zeros((n_cond, n_cond + 1))
    Cs = np.zeros((n_cond, n_cond))
    st = (frw_stats * n_cond)()
    rc = lib().frw_extract_matrix(ctx, int(sid), ctypes.byref(p), _ptr(C, c_double), _ptr(se, c_double),
                                  _ptr(Cs, c_double), st)
    _check(ctx, rc, (FRW_OK, FRW_ENOTCONV))
    return C, se, Cs, [x.as_dict() for x in st], rc == FRW_OK


def frw_extract_batch(ctx, jobs, n_conds):
    """jobs: list of dicts (structure_id, master, walk_budget, sigma_target, request_id, batch);
    n_conds: conductor count of each job's structure.  -> list of (C, stderr, stats) and converged flag."""
    n = len(jobs)
    arr = (frw_job * max(1, n))()
    for i, j in enumerate(jobs):
        arr[i] = frw_job(int(j["structure_id"]), int(j["master"]), int(j["walk_budget"]),
                         float(j.get("sigma_target", 0.0)), int(j.get("request_id", 0)), int(j.get("batch", 0)))
    tot = sum(nc + 1 for nc in n_conds)
    C = np.zeros(max(1, tot))
    se = np.zeros(max(1, tot))
    st = (frw_stats * max(1, n))()
    rc = lib().frw_extract_batch(ctx, arr, n, _ptr(C, c_double), _ptr(se, c_double), st)
    _check(ctx, rc, (FRW_OK, FRW_ENOTCONV))
    out, off = [], 0
    for i, nc in enumerate(n_conds):
        out.append((C[off:off + nc + 1].copy(), se[off:off + nc + 1].copy(), st[i].as_dict()))
        off += nc + 1
    return out, rc == FRW_OK


def _jobs_array(jobs):
    arr = (frw_job * max(1, len(jobs)))()
    for i, j in enumerate(jobs):
        arr[i] = frw_job(int(j["structure_id"]), int(j["master"]), int(j["walk_budget"]),
                         float(j.get("sigma_target", 0.0)), int(j.get("request_id", 0)), int(j.get("batch", 0)))
    return arr


class Plan:
    """A fixed job set replayed through a captured CUDA graph (frw_plan_*)."""

    def __init__(self, ctx, jobs, n_conds):
        self.ctx = ctx
        self.n_conds = list(n_conds)
        h = c_void_p(0)
        _check(ctx, lib().frw_plan_create(ctx, _jobs_array(jobs), len(jobs), ctypes.byref(h)))
        self.h = h

    def run(self, request_offset=0):
        n = len(self.n_conds)
        tot = sum(nc + 1 for nc in self.n_conds)
        C = np.zeros(max(1, tot))
        se = np.zeros(max(1, tot))
        st = (frw_stats * max(1, n))()
        rc = lib().frw_plan_run(self.h, int(request_offset), _ptr(C, c_double), _ptr(se, c_double), st)
        _check(self.ctx, rc, (FRW_OK, FRW_ENOTCONV))
        out, off = [], 0
        for i, nc in enumerate(self.n_conds):
            out.append((C[off:off + nc + 1].copy(), se[off:off + nc + 1].copy(), st[i].as_dict()))
            off += nc + 1
        return out, rc == FRW_OK

    def close(self):
        if self.h:
            lib().frw_plan_destroy(self.h)
            self.h = None


def frw_get_tuning(ctx) -> dict:
    t = frw_tuning()
    _check(ctx, lib().frw_get_tuning(ctx, ctypes.byref(t)))
    return t.as_dict()


def frw_set_tuning(ctx, **kw):
    t = frw_tuning()
    _check(ctx, lib().frw_get_tuning(ctx, ctypes.byref(t)))
    for k, v in kw.items():
        setattr(t, k, v)
    _check(ctx, lib().frw_set_tuning(ctx, ctypes.byref(t)))


def frw_autotune(ctx, sample_jobs, sample_walks) -> dict:
    t = frw_tuning()
    _check(ctx, lib().frw_autotune(ctx, _jobs_array(sample_jobs), len(sample_jobs), int(sample_walks),
                                   ctypes.byref(t)))
    return t.as_dict()


def frw_submit(ctx, job) -> int:
    """Queue one extraction (dict as in frw_extract_batch); returns its ticket."""
    j = frw_job(int(job["structure_id"]), int(job["master"]), int(job["walk_budget"]),
                float(job.get("sigma_target", 0.0)), int(job.get("request_id", 0)), int(job.get("batch", 0)))
    t = c_uint64(0)
    _check(ctx, lib().frw_submit(ctx, ctypes.byref(j), ctypes.byref(t)))
    return int(t.value)


def frw_cancel(ctx, ticket: int):
    _check(ctx, lib().frw_cancel(ctx, int(ticket)))


def frw_poll(ctx, ticket: int) -> bool:
    d = c_int32(0)
    _check(ctx, lib().frw_poll(ctx, int(ticket), ctypes.byref(d)))
    return bool(d.value)


def frw_wait(ctx, ticket: int, n_cond: int, timeout_s: float = -1.0):
    """-> (C, stderr, stats, converged), or None if timeout_s passed first."""
    C = np.zeros(n_cond + 1)
    se = np.zeros(n_cond + 1)
    st = frw_stats()
    rc = lib().frw_wait(ctx, int(ticket), float(timeout_s), _ptr(C, c_double), _ptr(se, c_double), ctypes.byref(st))
    if rc == FRW_ETIMEOUT:
        return None
    _check(ctx, rc, (FRW_OK, FRW_ENOTCONV))
    return C, se, st.as_dict(), rc == FRW_OK


def frw_walk_records(ctx, sid: int, master: int, request_id: int, walk_begin: int, n_walks: int):
    n = int(n_walks)
    om = np.zeros(n)
    k = np.zeros(n, np.int32)
    hops = np.zeros(n, np.uint32)
    steps = np.zeros(n, np.uint64)
    br = np.zeros(n, np.int32)
    rc = lib().frw_walk_records(ctx, int(sid), int(master), int(request_id), int(walk_begin), n,
                                _ptr(om, c_double), _ptr(k, c_int32), _ptr(hops, c_uint32),
                                _ptr(steps, c_uint64), _ptr(br, c_int32))
    _check(ctx, rc)
    return {"omega": om, "k": k, "hops": hops, "steps": steps, "branch": br}


def pack_cubes(cubes) -> np.ndarray:
    """:class:`workloads.CubeSet` -> int32 records of 64 words (see frw_microwalk_cubes)."""
    rec = np.zeros((cubes.n, 64), np.int32)
    rec[:, 0] = cubes.bg
    rec[:, 1] = cubes.nblk
    for b in range(cubes.ranges.shape[1]):
        rec[:, 2 + 7 * b:8 + 7 * b] = cubes.ranges[:, b, :]
        rec[:, 8 + 7 * b] = cubes.mat[:, b]
    return rec


def frw_microwalk_cubes(ctx, N: int, n_cubes: int, d_cubes_ptr: int, eps, samples_per_cube: int,
                        request_id: int, d_exit_ptr: int, d_steps_ptr: int) -> None:
    e = np.ascontiguousarray(eps, np.float64)
    rc = lib().frw_microwalk_cubes(ctx, int(N), int(n_cubes), c_void_p(d_cubes_ptr), _ptr(e, c_double), len(e),
                                   int(samples_per_cube), int(request_id), c_void_p(d_exit_ptr or 0),
                                   c_void_p(d_steps_ptr or 0))
    _check(ctx, rc)


def frw_microwalk_cubes_noalloc(N: int, n_cubes: int, d_cubes_ptr: int, eps, seed: int, samples_per_cube: int,
                                request_id: int, d_exit_ptr: int, d_steps_ptr: int, stream_handle: int = 0) -> int:
    """Allocation-free MicroWalk on the current device; returns the status code."""
    e = np.ascontiguousarray(eps, np.float64)
    return lib().frw_microwalk_cubes_noalloc(int(N), int(n_cubes), c_void_p(d_cubes_ptr), _ptr(e, c_double), len(e),
                                             int(seed), int(samples_per_cube), int(request_id),
                                             c_void_p(d_exit_ptr or 0), c_void_p(d_steps_ptr or 0),
                                             c_void_p(stream_handle or 0))


def frw_fdm_cubes(ctx, N: int, n_cubes: int, d_cubes_ptr: int, eps, d_u_ptr: int = 0, d_P_ptr: int = 0,
                  d_exit_ptr: int = 0, d_iters_ptr: int = 0) -> None:
    """FD-based transitions (Algorithm 2) of stand-alone cubes; device pointers."""
    e = np.ascontiguousarray(eps, np.float64)
    rc = lib().frw_fdm_cubes(ctx, int(N), int(n_cubes), c_void_p(d_cubes_ptr), _ptr(e, c_double), len(e),
                             c_void_p(d_u_ptr or 0), c_void_p(d_P_ptr or 0), c_void_p(d_exit_ptr or 0),
                             c_void_p(d_iters_ptr or 0))
    _check(ctx, rc)


def frw_table(ctx, N: int, kind: int, profile=None, eps=None):
    """-> (thresholds u32[6N^2], negative flags u8[6N^2], total, values f64[6N^2])."""
    P = 6 * N * N
    thr = np.zeros(P, np.uint32)
    neg = np.zeros(P, np.uint8)
    tot = np.zeros(1)
    vals = np.zeros(P)
    prof = np.ascontiguousarray(profile, np.int32) if profile is not None else None
    e = np.ascontiguousarray(eps, np.float64) if eps is not None else None
    rc = lib().frw_table(ctx, int(kind), _ptr(prof, c_int32), _ptr(e, c_double), 0 if e is None else len(e),
                         _ptr(thr, c_uint32), _ptr(neg, c_uint8), _ptr(tot, c_double), _ptr(vals, c_double))
    _check(ctx, rc)
    return thr, neg, float(tot[0]), vals


def decode_exit(packed: np.ndarray) -> np.ndarray:
    """Packed exit nodes -> (n, 3) int coordinates (one of them -1 or N)."""
    p = np.asarray(packed, np.int64)
    return np.stack([(p & 255) - 1, ((p >> 8) & 255) - 1, ((p >> 16) & 255) - 1], axis=1)


_TUNE_KEYS = ("pool_per_cta", "hops_per_epoch", "suspend_lanes", "suspend_min_steps", "mw_warps_per_cta",
              "mw_ctas_per_sm")


class Context:
    """Convenience owner of a context (destroyed on close / garbage collection)."""

    def __init__(self, device: int = 0, **opts):
        self.options = frw_default_options(**opts)
        self.N = self.options.N
        self.device = device
        self.ctx = frw_create(device, self.options)
        self._n_cond = {}
        self._tickets = {}

    def close(self):
        if self.ctx:
            frw_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def load(self, s) -> int:
        sid = frw_load_structure(self.ctx, s)
        self._n_cond[sid] = s.n_cond
        return sid

    def unload(self, sid):
        frw_unload_structure(self.ctx, sid)
        self._n_cond.pop(sid, None)

    def extract(self, sid, master, walk_budget, sigma_target=0.0, request_id=0, batch=0, walk_begin=0):
        return frw_extract(self.ctx, sid, master, self._n_cond.get(sid, 0), walk_budget, sigma_target,
                           request_id, batch, walk_begin)

    def extract_batch(self, jobs):
        return frw_extract_batch(self.ctx, jobs, [self._n_cond.get(j["structure_id"], 0) for j in jobs])

    def matrix(self, sid, walk_budget, sigma_target=0.0, request_id=0, batch=0):
        return frw_extract_matrix(self.ctx, sid, self._n_cond[sid], walk_budget, sigma_target, request_id, batch)

    def plan(self, jobs) -> Plan:
        return Plan(self.ctx, jobs, [self._n_cond.get(j["structure_id"], 0) for j in jobs])

    def tuning(self) -> dict:
        return frw_get_tuning(self.ctx)

    def set_tuning(self, **kw):
        frw_set_tuning(self.ctx, **kw)

    def autotune(self, sample_jobs, sample_walks=200_000, cache=None) -> dict:
        """frw_autotune on the sample jobs.  With `cache` (a JSON file path), settings
        are kept per (device name, N, geometry precision, MicroWalk-E factor): a
        cached entry is applied without tuning, a new one is written after tuning."""
        key = None
        if cache:
            try:
                import torch
                dev = torch.cuda.get_device_name(self.device)
            except Exception:
                dev = f"cuda:{self.device}"
            key = f"{dev}|N={self.N}|precision={self.options.precision}|mwe={self.options.mwe_factor}"
            try:
                with open(cache) as f:
                    data = json.load(f)
            except (OSError, ValueError):
                data = {}
            if key in data:
                t = data[key]
                self.set_tuning(**{k: t[k] for k in _TUNE_KEYS})
                return self.tuning()
        t = frw_autotune(self.ctx, sample_jobs, sample_walks)
        if key:
            data[key] = t
            tmp = f"{cache}.{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return t

    def submit(self, job) -> int:
        t = frw_submit(self.ctx, job)
        self._tickets[t] = self._n_cond.get(job["structure_id"], 0)
        return t

    def poll(self, ticket) -> bool:
        return frw_poll(self.ctx, ticket)

    def cancel(self, ticket):
        frw_cancel(self.ctx, ticket)

    def serve_info(self) -> dict:
        i = frw_serve_info()
        _check(self.ctx, lib().frw_get_serve_info(self.ctx, ctypes.byref(i)))
        return i.as_dict()

    def wait(self, ticket, timeout_s=-1.0):
        r = frw_wait(self.ctx, ticket, self._tickets[ticket], timeout_s)
        if r is not None:
            self._tickets.pop(ticket, None)
        return r

    def walk_records(self, sid, master, n_walks, request_id=0, walk_begin=0):
        return frw_walk_records(self.ctx, sid, master, request_id, walk_begin, n_walks)

    def table(self, kind, profile=None, eps=None):
        return frw_table(self.ctx, self.N, kind, profile, eps)
