"""Python binding of the C-ABI race checker (libhirace.so).

Argument marshalling only: every step of the check runs in the library's
CUDA kernels.  PyTorch is used for device memory and streams (tensors are
passed by ``data_ptr()``, streams by ``cuda_stream``).  There is no CPU
fallback: if the shared library is missing, importing the checker raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

RACE_DTYPE = np.dtype([("word", "<u4"), ("tid", "<u4"), ("kernel", "<u2"), ("epoch", "<u2"),
                       ("region", "<u2"), ("op", "u1"), ("prior", "u1")])
assert RACE_DTYPE.itemsize == 16

HR_OK = 0
STATUS = {0: "HR_OK", 1: "HR_ERR_INVALID", 2: "HR_ERR_OOM", 3: "HR_ERR_CUDA", 4: "HR_ERR_ORDER",
          5: "HR_ERR_RANGE", 6: "HR_ERR_CLOCK_OVERFLOW", 7: "HR_ERR_CONTENTION", 8: "HR_ERR_TIMEOUT",
          9: "HR_ERR_UNSUPPORTED", 10: "HR_ERR_CAPACITY", 11: "HR_ERR_NOT_READY"}
STATUS_CODE = {v: k for k, v in STATUS.items()}
FLAG_TRUNCATED = 1
REPORT_FIRST, REPORT_EVERY_EPOCH = 0, 1
SPACE_GLOBAL, SPACE_SHARED = 0, 1
SYNC_KERNEL = 0


class HrRegionDesc(ctypes.Structure):
    _fields_ = [("n_words", ctypes.c_uint64), ("block_dim", ctypes.c_uint32), ("warp_size", ctypes.c_uint32),
                ("space", ctypes.c_uint32), ("shadow_bytes", ctypes.c_uint8), ("tid_bits", ctypes.c_uint8),
                ("report_mode", ctypes.c_uint8), ("reserved", ctypes.c_uint8), ("report_capacity", ctypes.c_uint64)]


class HrGeom(ctypes.Structure):
    _fields_ = [("block_dim", ctypes.c_uint32), ("warp_size", ctypes.c_uint32), ("bd_magic", ctypes.c_uint64),
                ("ws_magic", ctypes.c_uint64), ("bd_shift", ctypes.c_uint32), ("ws_shift", ctypes.c_uint32),
                ("shadow_bytes", ctypes.c_uint32), ("tid_bits", ctypes.c_uint32), ("report_mode", ctypes.c_uint32),
                ("pad", ctypes.c_uint32)]


class HrFilter(ctypes.Structure):
    """Mirror of hr_filter (include/hirace.h): selective monitoring."""
    _fields_ = [("word_lo", ctypes.c_uint64), ("word_hi", ctypes.c_uint64), ("block_lo", ctypes.c_uint32),
                ("block_hi", ctypes.c_uint32), ("lane_mask", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("sym_lo", ctypes.c_uint32), ("sym_hi", ctypes.c_uint32), ("sym_stride", ctypes.c_uint64)]


class HrJob(ctypes.Structure):
    _fields_ = [("region", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("trace", ctypes.c_void_p),
                ("n", ctypes.c_uint64)]


class HrView(ctypes.Structure):
    """Mirror of hr_view (include/hirace_device.cuh): what an instrumented kernel gets by value."""
    _fields_ = [("shadow", ctypes.c_void_p), ("ring", ctypes.c_void_p), ("n_races", ctypes.c_void_p),
                ("error", ctypes.c_void_p), ("flags", ctypes.c_void_p), ("table", ctypes.c_void_p),
                ("n_words", ctypes.c_uint64), ("ring_cap", ctypes.c_uint64), ("geom", HrGeom),
                ("kernel", ctypes.c_uint32), ("region", ctypes.c_uint32), ("filter", HrFilter)]


assert ctypes.sizeof(HrView) == 168


class HiRaceError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s%s" % (STATUS.get(status, "status %d" % status), (": " + what) if what else ""))


_lib = None


def load_library():
    """Load libhirace.so from the package directory (built by ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("HIRACE_LIB", _build.LIB)   # a custom build of the same C-ABI
    if not os.path.exists(path):
        raise RuntimeError("libhirace.so is not built (run __graft_entry__.build()); "
                           "the checker has no CPU fallback")
    lib = ctypes.CDLL(path)
    P, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    lib.hr_init.argtypes = [ctypes.POINTER(P), ctypes.POINTER(HrRegionDesc), u32, u64, P]
    lib.hr_init_with_buffers.argtypes = [ctypes.POINTER(P), ctypes.POINTER(HrRegionDesc), u32, u64,
                                         ctypes.POINTER(P), ctypes.POINTER(P), P]
    lib.hr_set_filter.argtypes = [P, u32, ctypes.POINTER(HrFilter), P]
    lib.hr_check_trace_host.argtypes = [P, u32, P, u64, u64, P]
    lib.hr_batch_job_times.argtypes = [P, ctypes.POINTER(u64), u32]
    lib.hr_check_trace.argtypes = [P, u32, P, u64, P]
    lib.hr_check_trace_plain.argtypes = [P, u32, P, u64, P]
    lib.hr_check_trace_kbase.argtypes = [P, u32, P, u64, u32, P]
    lib.hr_sync.argtypes = [P, u32, u32, P]
    lib.hr_report.argtypes = [P, u32, P, u64, ctypes.POINTER(u64), ctypes.POINTER(u32)]
    lib.hr_counters.argtypes = [P, u32, ctypes.POINTER(u64 * 4)]
    lib.hr_reset.argtypes = [P, u32, P]
    lib.hr_destroy.argtypes = [P]
    lib.hr_variant_count.restype = u32
    lib.hr_variant_desc.argtypes = [u32, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]
    lib.hr_variant_desc.restype = i32
    lib.hr_set_variant.argtypes = [P, u32]
    lib.hr_set_variant.restype = i32
    lib.hr_get_variant.argtypes = [P, ctypes.POINTER(u32)]
    lib.hr_get_variant.restype = i32
    lib.hr_autotune.argtypes = [P, u32, P, u64, P, ctypes.POINTER(u32), ctypes.POINTER(ctypes.c_float), u32]
    lib.hr_autotune.restype = i32
    lib.hr_set_limits.argtypes = [P, u64, u32, u32]
    lib.hr_set_limits.restype = i32
    lib.hr_profile_enable.argtypes = [P, i32]
    lib.hr_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(u64), ctypes.POINTER(u64)]
    lib.hr_check_batch.argtypes = [P, ctypes.POINTER(HrJob), u32, P]
    lib.hr_check_batch.restype = i32
    lib.hr_batch_reserve.argtypes = [P, u32, u64]
    lib.hr_batch_reserve.restype = i32
    lib.hr_region_reconfigure.argtypes = [P, u32, u64, u32, u32, P]
    lib.hr_region_reconfigure.restype = i32
    lib.hr_device_view.argtypes = [P, u32, ctypes.POINTER(HrView)]
    lib.hr_device_view.restype = i32
    lib.hr_status_str.argtypes = [i32]
    lib.hr_status_str.restype = ctypes.c_char_p
    lib.hr_fsm_table.argtypes = [P, ctypes.POINTER(u32)]
    lib.hr_fsm_state_name.argtypes = [u32]
    lib.hr_fsm_state_name.restype = ctypes.c_char_p
    lib.hr_version.restype = ctypes.c_char_p
    for name in ("hr_init", "hr_check_trace", "hr_check_trace_plain", "hr_check_trace_kbase", "hr_sync", "hr_report", "hr_counters",
                 "hr_reset", "hr_destroy", "hr_fsm_table", "hr_profile_enable", "hr_profile_read"):
        getattr(lib, name).restype = i32
    _lib = lib
    return lib


def fsm_table():
    """(table[2048] uint8, n_states) of the flat FSM; host only, no GPU needed."""
    lib = load_library()
    out = np.zeros(2048, np.uint8)
    n = ctypes.c_uint32(0)
    rc = lib.hr_fsm_table(out.ctypes.data, ctypes.byref(n))
    if rc:
        raise HiRaceError(rc)
    return out, int(n.value)


def variants():
    """[(id, dict(aggregate, records_per_lane, consumer_warps, binned))] of the checker: the
    per-wave kernel's shapes, and the binned checker (reported with zero lanes and warps)."""
    lib = load_library()
    out = []
    for i in range(lib.hr_variant_count()):
        a, r, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        lib.hr_variant_desc(i, ctypes.byref(a), ctypes.byref(r), ctypes.byref(c))
        out.append((i, dict(aggregate=bool(a.value), records_per_lane=r.value, consumer_warps=c.value,
                            binned=c.value == 0)))
    return out


def binned_variant() -> int:
    """Variant id of the binned checker (per-segment shadow in shared memory)."""
    return next(i for i, d in variants() if d["binned"])


def state_name(state: int) -> str:
    return load_library().hr_fsm_state_name(state).decode()


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr_and_count(trace):
    if trace.device.type != "cuda":
        raise ValueError("trace must be a CUDA tensor")
    if not trace.is_contiguous():
        raise ValueError("trace must be contiguous")
    nbytes = trace.numel() * trace.element_size()
    if nbytes % 16:
        raise ValueError("trace size must be a multiple of 16 bytes")
    return ctypes.c_void_p(trace.data_ptr()), nbytes // 16


class Checker:
    """One checker context with one shadow store per region.

    ``regions`` is a list of dicts with keys n_words, block_dim and optional
    warp_size (32), space (global), report_capacity (0 = the default),
    shadow_bytes (8, or 4 for the compact packing), tid_bits (compact
    packing: tid width, 0 = 16) and report_mode (REPORT_FIRST: the first racy
    epoch of each word per kernel; REPORT_EVERY_EPOCH: every racy epoch).
    """

    def __init__(self, regions, report_capacity: int = 1 << 20, stream=None, buffers=None):
        """``buffers``: optional caller-owned device tensors, one per region, as
        ``shadow`` or ``(shadow, ring)`` (ring may be None); they must stay alive
        and untouched while the checker lives (hr_init_with_buffers)."""
        self._lib = load_library()
        arr = (HrRegionDesc * len(regions))()
        for i, r in enumerate(regions):
            arr[i].n_words = int(r["n_words"])
            arr[i].block_dim = int(r["block_dim"])
            arr[i].warp_size = int(r.get("warp_size", 32))
            arr[i].space = int(r.get("space", SPACE_GLOBAL))
            arr[i].shadow_bytes = int(r.get("shadow_bytes", 0))
            arr[i].tid_bits = int(r.get("tid_bits", 0))
            arr[i].report_mode = int(r.get("report_mode", REPORT_FIRST))
            arr[i].reserved = 0
            arr[i].report_capacity = int(r.get("report_capacity", 0))
        self.regions = [dict(r) for r in regions]
        self.report_capacity = report_capacity
        ctx = ctypes.c_void_p()
        self._buffers = None
        if buffers is None:
            rc = self._lib.hr_init(ctypes.byref(ctx), arr, len(regions), report_capacity, _stream_handle(stream))
        else:
            if len(buffers) != len(regions):
                raise ValueError("one buffer entry per region")
            pairs = [b if isinstance(b, (tuple, list)) else (b, None) for b in buffers]
            for i, (sh, ring) in enumerate(pairs):
                need = int(regions[i]["n_words"]) * (24 if int(regions[i].get("report_mode", 0)) else
                                                     4 if int(regions[i].get("shadow_bytes", 8)) == 4 else 8)
                if not sh.is_cuda or sh.numel() * sh.element_size() < need:
                    raise ValueError("shadow buffer %d must be a device tensor of >= %d bytes" % (i, need))
                cap = int(regions[i].get("report_capacity", 0)) or report_capacity
                if ring is not None and (not ring.is_cuda or ring.numel() * ring.element_size() < 16 * cap):
                    raise ValueError("ring buffer %d must be a device tensor of >= %d bytes" % (i, 16 * cap))
            sh_arr = (ctypes.c_void_p * len(pairs))(*[sh.data_ptr() for sh, _ in pairs])
            ring_arr = (ctypes.c_void_p * len(pairs))(*[(r.data_ptr() if r is not None else None) for _, r in pairs])
            self._buffers = pairs   # keep the tensors alive with the context
            rc = self._lib.hr_init_with_buffers(ctypes.byref(ctx), arr, len(regions), report_capacity, sh_arr,
                                                ring_arr, _stream_handle(stream))
        if rc:
            raise HiRaceError(rc, "hr_init")
        self._ctx = ctx

    def _check(self, rc, what):
        if rc:
            raise HiRaceError(rc, what)

    def check_trace(self, region: int, trace, stream=None, aggregate: bool = True, kernel_base: int = 0):
        """Queue a check of a device-resident trace (16-byte records)."""
        ptr, n = _ptr_and_count(trace)
        st = _stream_handle(stream)
        if kernel_base:
            if not aggregate:
                raise ValueError("kernel_base is only offered by the aggregated checker")
            rc = self._lib.hr_check_trace_kbase(self._ctx, region, ptr, n, kernel_base, st)
        else:
            fn = self._lib.hr_check_trace if aggregate else self._lib.hr_check_trace_plain
            rc = fn(self._ctx, region, ptr, n, st)
        self._check(rc, "hr_check_trace")

    def batch_job_times(self, n: int) -> np.ndarray:
        """Per-job completion times (ns after the batch started) of the last check_batch."""
        buf = (ctypes.c_uint64 * max(1, n))()
        self._check(self._lib.hr_batch_job_times(self._ctx, buf, n), "hr_batch_job_times")
        return np.frombuffer(buf, dtype=np.uint64)[:n].copy()

    def check_trace_host(self, region: int, trace, chunk_records: int = 0, stream=None):
        """Queue a check of a trace in host memory (a CPU tensor or a numpy array of
        16-byte records; page-locked for overlap), copied in chunks that overlap the
        checks.  Keep `trace` alive until the stream has passed this call."""
        import torch
        if isinstance(trace, np.ndarray):
            ptr, n = trace.ctypes.data, trace.nbytes // 16
        else:
            if trace.is_cuda:
                raise ValueError("check_trace_host takes host memory; use check_trace for device traces")
            ptr, n = trace.data_ptr(), trace.numel() * trace.element_size() // 16
        self._check(self._lib.hr_check_trace_host(self._ctx, region, ctypes.c_void_p(ptr), n, chunk_records,
                                                  _stream_handle(stream)), "hr_check_trace_host")

    def check_batch(self, jobs, stream=None):
        """Queue one batched check: ``jobs`` is a list of (region, device trace tensor)
        with distinct regions."""
        arr = (HrJob * max(1, len(jobs)))()
        keep = []
        for i, (region, trace) in enumerate(jobs):
            ptr, n = _ptr_and_count(trace)
            arr[i].region = region
            arr[i].reserved = 0
            arr[i].trace = ptr
            arr[i].n = n
            keep.append(trace)
        self._check(self._lib.hr_check_batch(self._ctx, arr, len(jobs), _stream_handle(stream)), "hr_check_batch")

    def batch_reserve(self, max_jobs: int, max_waves: int = 1 << 18):
        self._check(self._lib.hr_batch_reserve(self._ctx, max_jobs, max_waves), "hr_batch_reserve")

    def sync(self, region: int, stream=None):
        self._check(self._lib.hr_sync(self._ctx, region, SYNC_KERNEL, _stream_handle(stream)), "hr_sync")

    def report(self, region: int, cap: int | None = None):
        """(races, status, n_total, flags); waits for the region's work."""
        if cap is None:
            cap = int(self.regions[region].get("report_capacity", 0) or self.report_capacity)
        out = np.zeros(max(cap, 1), RACE_DTYPE)
        n_total = ctypes.c_uint64(0)
        flags = ctypes.c_uint32(0)
        rc = self._lib.hr_report(self._ctx, region, out.ctypes.data, cap, ctypes.byref(n_total),
                                 ctypes.byref(flags))
        if rc in (STATUS_CODE["HR_ERR_INVALID"], STATUS_CODE["HR_ERR_CUDA"]):
            raise HiRaceError(rc, "hr_report")
        ring_cap = int(self.regions[region].get("report_capacity", 0) or self.report_capacity)
        n = min(int(n_total.value), cap, ring_cap)
        return out[:n], int(rc), int(n_total.value), int(flags.value)

    def counters(self, region: int):
        buf = (ctypes.c_uint64 * 4)()
        self._check(self._lib.hr_counters(self._ctx, region, ctypes.byref(buf)), "hr_counters")
        return dict(accesses=buf[0], cas=buf[1], retries=buf[2], merged=buf[3])

    def reconfigure(self, region: int, n_words: int, block_dim: int, warp_size: int = 32, stream=None):
        """Reuse a region for a job of another shape (n_words within its allocation)."""
        self._check(self._lib.hr_region_reconfigure(self._ctx, region, n_words, block_dim, warp_size,
                                                    _stream_handle(stream)), "hr_region_reconfigure")
        self.regions[region] = dict(self.regions[region], n_words=n_words, block_dim=block_dim, warp_size=warp_size)

    def reset(self, region: int, stream=None):
        self._check(self._lib.hr_reset(self._ctx, region, _stream_handle(stream)), "hr_reset")

    def device_view(self, region: int) -> HrView:
        """The by-value view an instrumented kernel needs (kernel ordinal = hr_sync count)."""
        v = HrView()
        self._check(self._lib.hr_device_view(self._ctx, region, ctypes.byref(v)), "hr_device_view")
        return v

    def set_filter(self, region: int, word_lo: int = 0, word_hi: int = 0, block_lo: int = 0, block_hi: int = 0,
                   lane_mask: int = 0xFFFFFFFF, sym_lo: int = 0, sym_hi: int = 0, sym_stride: int = 0, stream=None):
        """Monitor only words [word_lo, word_hi) (word_hi 0: all), blocks
        [block_lo, block_hi) (block_hi 0: all) and the lanes in lane_mask;
        blocks [sym_lo, sym_hi) (sym_hi 0: none) form a symmetric group checked
        through block sym_lo, member m's words shifted by m * sym_stride."""
        f = HrFilter(word_lo, word_hi, block_lo, block_hi, lane_mask, 0, sym_lo, sym_hi, sym_stride)
        self._check(self._lib.hr_set_filter(self._ctx, region, ctypes.byref(f), _stream_handle(stream)),
                    "hr_set_filter")

    def clear_filter(self, region: int, stream=None):
        self._check(self._lib.hr_set_filter(self._ctx, region, None, _stream_handle(stream)), "hr_set_filter")

    def set_variant(self, variant: int):
        self._check(self._lib.hr_set_variant(self._ctx, variant), "hr_set_variant")

    def variant(self) -> int:
        v = ctypes.c_uint32()
        self._check(self._lib.hr_get_variant(self._ctx, ctypes.byref(v)), "hr_get_variant")
        return v.value

    def autotune(self, region: int, trace, stream=None):
        """Time every kernel variant on this trace, keep the fastest; returns (best, [ms...])."""
        ptr, n = _ptr_and_count(trace)
        nv = self._lib.hr_variant_count()
        ms = (ctypes.c_float * nv)()
        best = ctypes.c_uint32()
        self._check(self._lib.hr_autotune(self._ctx, region, ptr, n, _stream_handle(stream), ctypes.byref(best), ms,
                                          nv), "hr_autotune")
        return best.value, list(ms)

    def autotune_cached(self, region: int, trace, key: str, stream=None):
        """Autotune once per workload key; the choice is kept in the JSON file named
        by $HIRACE_TUNE_CACHE (no file: tune every time)."""
        import json
        path = os.environ.get("HIRACE_TUNE_CACHE")
        cache = {}
        if path and os.path.exists(path):
            with open(path) as f:
                cache = json.load(f)
        if key in cache:
            self.set_variant(int(cache[key]))
            return int(cache[key]), None
        best, ms = self.autotune(region, trace, stream)
        if path:
            cache[key] = best
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        return best, ms

    def set_limits(self, wait_ns: int = 4_000_000_000, cas_retry_cap: int = 4096, test_flags: int = 0):
        """Bounds of device waits (ns) and CAS retries; test_flags=1 holds stage 1 (tests only)."""
        self._check(self._lib.hr_set_limits(self._ctx, wait_ns, cas_retry_cap, test_flags), "hr_set_limits")

    def profile(self, on: bool = True):
        self._check(self._lib.hr_profile_enable(self._ctx, int(on)), "hr_profile_enable")

    def profile_read(self):
        """dict(check_ms, prepass_ms, calls, launches) summed since the last read."""
        a, b = ctypes.c_double(0), ctypes.c_double(0)
        c, d = ctypes.c_uint64(0), ctypes.c_uint64(0)
        self._check(self._lib.hr_profile_read(self._ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                              ctypes.byref(d)), "hr_profile_read")
        return dict(check_ms=a.value, prepass_ms=b.value, calls=c.value, launches=d.value)

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.hr_destroy(self._ctx)
            self._ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def race_keys(races) -> set:
    """{(kernel, word, epoch)} of a race array."""
    return {(int(k), int(w), int(e)) for k, w, e in zip(races["kernel"], races["word"], races["epoch"])}


# ---------------------------------------------------------------------------
# Hand-instrumented synthetic kernels (libhirace_workloads.so)
# ---------------------------------------------------------------------------

_wl = None


def load_workloads():
    """Stencil, histogram and reduction kernels, instrumented with hr_access()."""
    global _wl
    if _wl is not None:
        return _wl
    if not os.path.exists(_build.WORKLOADS_LIB):
        raise RuntimeError("libhirace_workloads.so is not built (run __graft_entry__.build())")
    lib = ctypes.CDLL(_build.WORKLOADS_LIB)
    P, u32, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int
    VP = ctypes.POINTER(HrView)
    lib.hrw_stencil.argtypes = [VP, P, P, u32, u32, u32, P]
    lib.hrw_histogram.argtypes = [VP, P, u32, P, u32, u32, P]
    lib.hrw_reduce.argtypes = [VP, P, u32, u32, i32, P]
    lib.hrw_smem_reduce.argtypes = [VP, i32, P, P, u32, u32, i32, P]
    for f in (lib.hrw_stencil, lib.hrw_histogram, lib.hrw_reduce, lib.hrw_smem_reduce):
        f.restype = i32
    _wl = lib
    return lib


def run_stencil(view, d_in, d_out, block=256, racy_stride=0, stream=None):
    rc = load_workloads().hrw_stencil(ctypes.byref(view) if view is not None else None, d_in.data_ptr(),
                                      d_out.data_ptr(), d_in.numel(), block, racy_stride, _stream_handle(stream))
    if rc:
        raise RuntimeError("hrw_stencil failed (%d)" % rc)


def run_histogram(view, d_keys, d_bins, block=256, racy_stride=0, stream=None):
    rc = load_workloads().hrw_histogram(ctypes.byref(view) if view is not None else None, d_keys.data_ptr(),
                                        d_keys.numel(), d_bins.data_ptr(), block, racy_stride, _stream_handle(stream))
    if rc:
        raise RuntimeError("hrw_histogram failed (%d)" % rc)


def run_smem_reduce(view, d_in, d_out, mode, block=256, drop_level=-1, stream=None):
    """Block reduction through a __shared__ buffer: mode 0 plain, 1 monitored
    through the region's global shadow, 2 through a shared-memory shadow."""
    rc = load_workloads().hrw_smem_reduce(ctypes.byref(view) if view is not None else None, mode, d_in.data_ptr(),
                                          d_out.data_ptr(), d_in.numel(), block, drop_level, _stream_handle(stream))
    if rc:
        raise RuntimeError("hrw_smem_reduce failed (%d)" % rc)


def run_reduce(view, d_data, block=256, drop_level=-1, stream=None):
    rc = load_workloads().hrw_reduce(ctypes.byref(view) if view is not None else None, d_data.data_ptr(),
                                     d_data.numel(), block, drop_level, _stream_handle(stream))
    if rc:
        raise RuntimeError("hrw_reduce failed (%d)" % rc)

