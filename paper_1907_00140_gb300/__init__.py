"""Python binding of libchl.so, the GB300 canonical hub labeling library.

Thin marshalling over the C ABI declared in ``include/chl.h``: every function
of that header is exposed under the same name with the same arguments
(pointers as ints, ``void* stream`` as an int). Arrays may be numpy arrays
(host memory, ``CHL_MEM_HOST``) or torch CUDA tensors (device memory,
``CHL_MEM_DEVICE``); the helpers below only pass pointers and sizes. All
computation happens inside libchl.so on the GPU; there is no CPU fallback, and
calling into this module without a built library raises.

Method: PLaNT (Lakhotia et al., arXiv 1907.00140, Sec. 5.2, Algorithm 3)
builds one shortest-path tree per root in rank order and labels a vertex with
the root exactly when no higher-ranked vertex lies on any of its shortest
paths from the root; queries merge the two rank-sorted label lists (Sec. 6).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "build", "lib", "Server", "CHL_OK", "CHL_EINVAL", "CHL_ENOMEM", "CHL_ECUDA", "CHL_ETIMEOUT",
    "CHL_EOVERFLOW", "CHL_MEM_DEVICE", "CHL_MEM_HOST", "CHL_FLAG_WIDE_KEYS", "CHL_FLAG_PARENTS", "CHL_FLAG_NO_HYBRID", "CHL_FLAG_DENSE_ROOT_LABELS", "ChlError", "chl_csr", "chl_build_opts",
    "chl_build_stats", "chl_build", "chl_query", "chl_labels_info", "chl_labels_stats",
    "chl_labels_view", "chl_labels_copy", "chl_labels_free", "chl_last_error", "chl_version",
    "chl_query_noalloc", "chl_query_partitioned", "chl_query_grouped", "query_partitioned",
    "chl_tune", "chl_tune_report", "tune",
    "Labels", "build_labels", "query",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
_SOURCES = ["chl_api.cu", "chl_graph.cu", "chl_tree.cu", "chl_labels.cu", "chl_query.cu",
            "chl_serve.cu"]
LIB_PATH = os.path.join(_HERE, "libchl.so")
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]

CHL_OK, CHL_EINVAL, CHL_ENOMEM, CHL_ECUDA, CHL_ETIMEOUT, CHL_EOVERFLOW = range(6)
CHL_MEM_DEVICE, CHL_MEM_HOST = 0, 1
CHL_FLAG_WIDE_KEYS = 1
CHL_FLAG_PARENTS = 2
CHL_FLAG_NO_HYBRID = 4
CHL_FLAG_DENSE_ROOT_LABELS = 8
_NAMES = {0: "CHL_OK", 1: "CHL_EINVAL", 2: "CHL_ENOMEM", 3: "CHL_ECUDA", 4: "CHL_ETIMEOUT",
          5: "CHL_EOVERFLOW"}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _sources():
    return [os.path.join(_CSRC, s) for s in _SOURCES]


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = _sources() + [os.path.join(_CSRC, "chl_common.cuh"), os.path.join(_INCLUDE, "chl.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libchl.so for sm_103a in-tree (nvcc, one translation unit per
    source, compiled in parallel) if it is missing or older than its sources."""
    if not force and not _stale():
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [_nvcc(), *ARCH_FLAGS, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-shared", "-t", "0", "-o", tmp, *_sources()]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
    if verbose:
        print(r.stdout + r.stderr)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


# ------------------------------------------------------------------ ABI structs
class chl_csr(C.Structure):
    _fields_ = [("n", C.c_uint32), ("num_arcs", C.c_uint64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("w", C.c_void_p), ("mem", C.c_int)]


class chl_build_opts(C.Structure):
    _fields_ = [("root_begin", C.c_uint32), ("root_end", C.c_uint32),
                ("threads_per_tree", C.c_int32), ("bucket_delta", C.c_int32),
                ("window_buckets", C.c_int32), ("slots", C.c_int32), ("mode", C.c_int32),
                ("flags", C.c_int32), ("label_capacity", C.c_uint64), ("common_hubs", C.c_int32),
                ("pruned_bucket_delta", C.c_int32), ("psi_threshold", C.c_float),
                ("pruned_threads_per_tree", C.c_int32), ("switch_ratio", C.c_float),
                ("round_limit", C.c_uint32), ("query_stage_kb", C.c_int32),
                ("small_tree_expansions", C.c_uint32), ("small_threads_per_tree", C.c_int32),
                ("big_tree_bucket_delta", C.c_int32), ("overlap_phases", C.c_int32)]


class chl_tune_report(C.Structure):
    _fields_ = [("trials", C.c_int32), ("sample_roots", C.c_uint32), ("best_tree_ms", C.c_double),
                ("best_expanded", C.c_uint64), ("best_arcs", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class chl_server_opts(C.Structure):
    _fields_ = [("query_slots", C.c_int32), ("max_batch", C.c_uint64), ("batching", C.c_int32),
                ("build_workers", C.c_int32), ("build_slots", C.c_int32),
                ("build_budget", C.c_uint64), ("query_order", C.c_int32)]


class chl_server_stats(C.Structure):
    _fields_ = [("batches", C.c_uint64), ("pairs", C.c_uint64), ("max_batch_seen", C.c_uint64),
                ("builds_done", C.c_uint64), ("builds_failed", C.c_uint64),
                ("build_bytes_peak", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class chl_build_stats(C.Structure):
    _fields_ = [("trees", C.c_uint64), ("labels", C.c_uint64), ("expanded", C.c_uint64),
                ("arcs", C.c_uint64), ("trivial", C.c_uint64), ("build_ms", C.c_double),
                ("tree_ms", C.c_double), ("sort_ms", C.c_double), ("launches", C.c_uint64),
                ("rounds", C.c_uint64), ("buckets", C.c_uint64), ("pruned", C.c_uint64),
                ("table_ms", C.c_double), ("phases", C.c_uint64),
                ("label_table_phases", C.c_uint64), ("small_tree_phases", C.c_uint64),
                ("overlapped_trees", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libchl.so (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is not built; call paper_1907_00140_gb300.build()")
            L = C.CDLL(LIB_PATH)
            vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
            L.chl_build.argtypes = [C.POINTER(chl_csr), vp, C.POINTER(chl_build_opts), vp,
                                    C.POINTER(vp)]
            L.chl_build.restype = i32
            L.chl_tune.argtypes = [C.POINTER(chl_csr), vp, C.POINTER(chl_build_opts), vp,
                                   C.POINTER(chl_build_opts), C.POINTER(chl_tune_report)]
            L.chl_tune.restype = i32
            L.chl_labels_info.argtypes = [vp, C.POINTER(u32), C.POINTER(u64), C.POINTER(u64)]
            L.chl_labels_info.restype = i32
            L.chl_labels_stats.argtypes = [vp, C.POINTER(chl_build_stats)]
            L.chl_labels_stats.restype = i32
            L.chl_labels_view.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]
            L.chl_labels_view.restype = i32
            L.chl_labels_copy.argtypes = [vp, vp, vp, vp, i32, vp]
            L.chl_labels_copy.restype = i32
            L.chl_query.argtypes = [vp, vp, u64, vp, i32, vp]
            L.chl_query.restype = i32
            L.chl_query_noalloc.argtypes = [vp, vp, u64, vp, i32, vp]
            L.chl_query_noalloc.restype = i32
            L.chl_query_partitioned.argtypes = [C.POINTER(vp), u32, vp, u64, vp, i32, vp]
            L.chl_query_partitioned.restype = i32
            L.chl_query_grouped.argtypes = [vp, vp, u64, vp, i32, vp]
            L.chl_query_grouped.restype = i32
            L.chl_server_add_partitioned_set.argtypes = [vp, C.POINTER(vp), u32, C.POINTER(u32)]
            L.chl_server_add_partitioned_set.restype = i32
            L.chl_labels_free.argtypes = [vp]
            L.chl_labels_free.restype = None
            L.chl_last_error.argtypes = []
            L.chl_last_error.restype = C.c_char_p
            L.chl_version.argtypes = []
            L.chl_version.restype = C.c_char_p
            L.chl_labels_parents.argtypes = [vp, vp, i32, vp]
            L.chl_labels_parents.restype = i32
            L.chl_path.argtypes = [vp, vp, u64, u32, vp, vp, i32, vp]
            L.chl_path.restype = i32
            L.chl_server_create.argtypes = [C.POINTER(chl_server_opts), C.POINTER(vp)]
            L.chl_server_add_set.argtypes = [vp, vp, C.POINTER(u32)]
            L.chl_server_submit_query.argtypes = [vp, u32, vp, u64, vp, C.POINTER(u64)]
            L.chl_server_submit_build.argtypes = [vp, C.POINTER(chl_csr), vp,
                                                  C.POINTER(chl_build_opts), C.POINTER(u64)]
            L.chl_server_wait.argtypes = [vp, u64, C.c_double, C.POINTER(vp),
                                          C.POINTER(C.c_double)]
            L.chl_server_replay.argtypes = [vp, u64, vp, vp, vp, vp, vp, vp,
                                            C.POINTER(C.c_double)]
            L.chl_server_stats_get.argtypes = [vp, C.POINTER(chl_server_stats)]
            L.chl_server_destroy.argtypes = [vp]
            L.chl_server_destroy.restype = None
            for f in ("chl_server_create", "chl_server_add_set", "chl_server_submit_query",
                      "chl_server_submit_build", "chl_server_wait", "chl_server_replay",
                      "chl_server_stats_get"):
                getattr(L, f).restype = i32
            _lib = L
    return _lib


class ChlError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st: int):
    if st != CHL_OK:
        raise ChlError(st, lib().chl_last_error().decode())


# ------------------------------------------------------------------ raw ABI (same names)
def chl_build(g: chl_csr, rank_ptr: int, opts: chl_build_opts | None, stream: int) -> int:
    out = C.c_void_p()
    _check(lib().chl_build(C.byref(g), rank_ptr, C.byref(opts) if opts is not None else None,
                           stream, C.byref(out)))
    return out.value


def chl_tune(g: chl_csr, rank_ptr: int, base: chl_build_opts | None, stream: int):
    best, rep = chl_build_opts(), chl_tune_report()
    _check(lib().chl_tune(C.byref(g), rank_ptr, C.byref(base) if base is not None else None,
                          stream, C.byref(best), C.byref(rep)))
    return best, rep


def chl_labels_info(handle: int):
    n, t, b = C.c_uint32(), C.c_uint64(), C.c_uint64()
    _check(lib().chl_labels_info(handle, C.byref(n), C.byref(t), C.byref(b)))
    return n.value, t.value, b.value


def chl_labels_stats(handle: int) -> chl_build_stats:
    s = chl_build_stats()
    _check(lib().chl_labels_stats(handle, C.byref(s)))
    return s


def chl_labels_view(handle: int):
    o, h, d = C.c_void_p(), C.c_void_p(), C.c_void_p()
    _check(lib().chl_labels_view(handle, C.byref(o), C.byref(h), C.byref(d)))
    return o.value, h.value, d.value


def chl_labels_copy(handle: int, offsets: int, hub: int, dist: int, mem: int, stream: int):
    _check(lib().chl_labels_copy(handle, offsets, hub, dist, mem, stream))


def chl_query(handle: int, pairs: int, q: int, out: int, mem: int, stream: int):
    _check(lib().chl_query(handle, pairs, q, out, mem, stream))


def chl_query_noalloc(handle: int, pairs: int, q: int, out: int, mem: int, stream: int):
    """chl_query without any allocation: at most 2^20 pairs per call, staged
    in one fixed device array that all calls share (see include/chl.h)."""
    _check(lib().chl_query_noalloc(handle, pairs, q, out, mem, stream))


def chl_query_partitioned(handles, pairs: int, q: int, out: int, mem: int, stream: int):
    arr = (C.c_void_p * len(handles))(*handles)
    _check(lib().chl_query_partitioned(arr, len(handles), pairs, q, out, mem, stream))


def chl_query_grouped(handle: int, pairs: int, q: int, out: int, mem: int, stream: int):
    _check(lib().chl_query_grouped(handle, pairs, q, out, mem, stream))


def chl_labels_free(handle: int):
    lib().chl_labels_free(handle)


def chl_last_error() -> str:
    return lib().chl_last_error().decode()


def chl_version() -> str:
    return lib().chl_version().decode()


# ------------------------------------------------------------------ helpers
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr_mem(x, dtype):
    """(pointer, memory kind, keep-alive) for a numpy array or a torch CUDA tensor."""
    if _is_torch(x):
        import torch
        want = {np.uint32: torch.int32, np.uint64: torch.int64}[dtype]
        if not x.is_cuda:
            x = x.contiguous().numpy().view(dtype)
            return x.ctypes.data, CHL_MEM_HOST, x
        if x.dtype not in (want, {np.uint32: torch.uint32, np.uint64: torch.uint64}[dtype]):
            raise TypeError(f"tensor dtype {x.dtype} does not match {dtype.__name__}")
        x = x.contiguous()
        return x.data_ptr(), CHL_MEM_DEVICE, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, CHL_MEM_HOST, a


def _current_stream() -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


class Labels:
    """Owner of a chl_labels handle (device-resident labels)."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "handle", None):
            chl_labels_free(self.handle)
            self.handle = None

    @property
    def n(self) -> int:
        return chl_labels_info(self.handle)[0]

    @property
    def total(self) -> int:
        return chl_labels_info(self.handle)[1]

    @property
    def nbytes(self) -> int:
        return chl_labels_info(self.handle)[2]

    def stats(self) -> dict:
        return chl_labels_stats(self.handle).as_dict()

    def to_numpy(self, stream: int | None = None):
        """(offsets uint64[n+1], hub uint32[T], dist uint32[T]) copied to host."""
        n, T, _ = chl_labels_info(self.handle)
        off = np.empty(n + 1, np.uint64)
        hub = np.empty(T, np.uint32)
        dist = np.empty(T, np.uint32)
        chl_labels_copy(self.handle, off.ctypes.data, hub.ctypes.data if T else None,
                        dist.ctypes.data if T else None, CHL_MEM_HOST,
                        _current_stream() if stream is None else stream)
        return off, hub, dist

    def parents(self, stream: int | None = None) -> np.ndarray:
        """SPT parent of every label (host uint32[T], aligned with to_numpy()'s hub/dist)."""
        T = chl_labels_info(self.handle)[1]
        par = np.empty(max(T, 1), np.uint32)
        _check(lib().chl_labels_parents(self.handle, par.ctypes.data, CHL_MEM_HOST,
                                        _current_stream() if stream is None else stream))
        return par[:T]

    def paths(self, pairs, max_len: int = 64, stream: int | None = None):
        """Shortest paths of host pairs [q,2]: (paths uint32[q,max_len], lens uint32[q])."""
        p = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
        q = len(p)
        out = np.zeros((q, max_len), np.uint32)
        lens = np.zeros(q, np.uint32)
        _check(lib().chl_path(self.handle, p.ctypes.data, q, max_len, out.ctypes.data,
                              lens.ctypes.data, CHL_MEM_HOST,
                              _current_stream() if stream is None else stream))
        return out, lens

    def query(self, pairs, out=None, stream: int | None = None, grouped: bool = False):
        """Distances for pairs [q,2] (numpy -> numpy, CUDA tensor -> CUDA tensor);
        grouped=True answers the batch in grouped order (chl_query_grouped)."""
        p, mem, q, out, op = _query_args(pairs, out)
        fn = chl_query_grouped if grouped else chl_query
        fn(self.handle, p, q, op, mem, _current_stream() if stream is None else stream)
        return out


def _query_args(pairs, out):
    p, mem, keep = _ptr_mem(pairs, np.uint32)
    q = (keep.numel() if _is_torch(keep) else keep.size) // 2
    if out is None:
        if mem == CHL_MEM_DEVICE:
            import torch
            out = torch.empty(q, dtype=torch.int32, device=keep.device)
        else:
            out = np.empty(q, np.uint32)
    op = out.data_ptr() if _is_torch(out) else out.ctypes.data
    return p, mem, q, out, op


def query_partitioned(parts, pairs, out=None, stream: int | None = None):
    """Distances over labels held as hub partitions (a list of Labels built
    over disjoint root ranges): chl_query_partitioned."""
    p, mem, q, out, op = _query_args(pairs, out)
    chl_query_partitioned([L.handle for L in parts], p, q, op, mem,
                          _current_stream() if stream is None else stream)
    return out


def _csr_args(g, rank):
    rp, mem, k1 = _ptr_mem(g.row_ptr, np.uint64)
    cp, mem2, k2 = _ptr_mem(g.col, np.uint32)
    wp, mem3, k3 = _ptr_mem(g.w, np.uint32)
    rkp, mem4, k4 = _ptr_mem(rank, np.uint32)
    if len({mem, mem2, mem3, mem4}) != 1:
        raise ValueError("graph arrays and rank must all be host arrays or all CUDA tensors")
    narcs = (k2.numel() if _is_torch(k2) else k2.size)
    csr = chl_csr(int(g.n), int(narcs), rp, cp if narcs else None, wp if narcs else None, mem)
    return csr, rkp, (k1, k2, k3, k4)


def _build_opts(**kw) -> chl_build_opts:
    """chl_build_opts with the given fields (floats for float fields, else ints)."""
    o = chl_build_opts()
    kinds = dict(chl_build_opts._fields_)
    for k, v in kw.items():
        if k not in kinds:
            raise TypeError(f"unknown build option {k!r}")
        setattr(o, k, float(v) if kinds[k] is C.c_float else int(v))
    return o


def tune(g, rank, stream: int | None = None, **fixed):
    """Measured choice of threads_per_tree, bucket_delta and window_buckets
    for this graph, and for a whole build the phases' switch points
    switch_ratio and small_tree_expansions (chl_tune). Returns (build options
    for build_labels: the tuned fields, those set non-zero, and the fixed
    ones; tuning report)."""
    csr, rkp, keep = _csr_args(g, rank)
    base = _build_opts(**fixed)
    best, rep = chl_tune(csr, rkp, base, _current_stream() if stream is None else stream)
    out = {k: getattr(best, k) for k in ("threads_per_tree", "bucket_delta", "window_buckets")}
    for k in ("switch_ratio", "small_tree_expansions", "big_tree_bucket_delta", "common_hubs"):
        if getattr(best, k):
            out[k] = getattr(best, k)
    out.update(fixed)
    return out, rep.as_dict()


def build_labels(g, rank, stream: int | None = None, **opts) -> Labels:
    """Canonical hub labels of graph g (object with n, row_ptr, col, w; numpy
    arrays or CUDA tensors) under rank R (permutation, larger = more important).
    opts: fields of chl_build_opts (root_begin, root_end, threads_per_tree,
    bucket_delta, window_buckets, slots, mode)."""
    csr, rkp, keep = _csr_args(g, rank)
    o = _build_opts(**opts)
    h = chl_build(csr, rkp, o, _current_stream() if stream is None else stream)
    return Labels(h)


def query(labels: Labels, pairs, **kw):
    return labels.query(pairs, **kw)


# ------------------------------------------------------------------ serving loop
class Server:
    """Owner of a chl_server: resident label sets, continuous batching of
    queries, builds admitted by device memory (see include/chl.h)."""

    def __init__(self, **opts):
        o = chl_server_opts()
        for k, v in opts.items():
            setattr(o, k, v)
        h = C.c_void_p()
        _check(lib().chl_server_create(C.byref(o), C.byref(h)))
        self.handle = h.value
        self._keep = {}

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            lib().chl_server_destroy(self.handle)
            self.handle = None
            self._keep = {}

    def add_set(self, labels: "Labels") -> int:
        k = C.c_uint32()
        _check(lib().chl_server_add_set(self.handle, labels.handle, C.byref(k)))
        self._keep[("set", k.value)] = labels
        return k.value

    def add_partitioned_set(self, parts) -> int:
        """A label set held as hub partitions (Labels over disjoint root ranges)."""
        k = C.c_uint32()
        arr = (C.c_void_p * len(parts))(*[L.handle for L in parts])
        _check(lib().chl_server_add_partitioned_set(self.handle, arr, len(parts), C.byref(k)))
        self._keep[("set", k.value)] = list(parts)
        return k.value

    def submit_query(self, set_id: int, pairs) -> int:
        """Queue host pairs [q,2]; wait() returns the answers."""
        p = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
        out = np.empty(len(p), np.uint32)
        t = C.c_uint64()
        _check(lib().chl_server_submit_query(self.handle, set_id, p.ctypes.data, len(p),
                                             out.ctypes.data, C.byref(t)))
        self._keep[t.value] = (p, out)
        return t.value

    def submit_build(self, g, rank, **opts) -> int:
        """Queue a build from host arrays; wait() returns its Labels."""
        csr, rkp, keep = _csr_args(g, rank)
        o = chl_build_opts()
        for k, v in opts.items():
            setattr(o, k, v)
        t = C.c_uint64()
        _check(lib().chl_server_submit_build(self.handle, C.byref(csr), rkp, C.byref(o), C.byref(t)))
        self._keep[t.value] = (csr, keep, o)
        return t.value

    def wait(self, ticket: int, timeout: float = -1.0):
        """(answers or Labels, latency seconds) of a finished ticket."""
        built = C.c_void_p()
        lat = C.c_double()
        st = lib().chl_server_wait(self.handle, ticket, timeout, C.byref(built), C.byref(lat))
        kept = self._keep.pop(ticket, None) if st != CHL_ETIMEOUT else None
        _check(st)
        if built.value:
            return Labels(built.value), lat.value
        return kept[1], lat.value

    def replay(self, arrival_s, set_of, pair_off, pairs):
        """Open-loop replay; returns (answers, latency seconds per request, wall seconds)."""
        arr = np.ascontiguousarray(arrival_s, np.float64)
        so = np.ascontiguousarray(set_of, np.uint32)
        off = np.ascontiguousarray(pair_off, np.uint64)
        p = np.ascontiguousarray(pairs, np.uint32).reshape(-1, 2)
        out = np.empty(len(p), np.uint32)
        lat = np.empty(len(arr), np.float64)
        wall = C.c_double()
        _check(lib().chl_server_replay(self.handle, len(arr), arr.ctypes.data, so.ctypes.data,
                                       off.ctypes.data, p.ctypes.data, out.ctypes.data,
                                       lat.ctypes.data, C.byref(wall)))
        return out, lat, wall.value

    def stats(self) -> dict:
        st = chl_server_stats()
        _check(lib().chl_server_stats_get(self.handle, C.byref(st)))
        return st.as_dict()
