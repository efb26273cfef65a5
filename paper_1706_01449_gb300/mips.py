"""Python binding of libmips (include/mips.h): argument marshalling only.

Every step of the search runs in the CUDA library; this module passes
device pointers (from torch tensors), sizes and the current CUDA stream
through ctypes and turns status codes into exceptions.  There is no CPU
fallback: if the library is missing or CUDA is unavailable, calls raise.

Names follow the C ABI: build_index, topk, topk_maximus, select, select_arms,
topk_host, sync, get_stats, get_buffer, free_index, last_error.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmips.so")

MIPS_OK, MIPS_ERR_ARG, MIPS_ERR_NOMEM, MIPS_ERR_CUDA = 0, 1, 2, 3
MIPS_ERR_TIMEOUT, MIPS_ERR_OVERFLOW, MIPS_ERR_UNIMPLEMENTED, MIPS_ERR_NONFINITE = 4, 5, 6, 7
STATUS_NAMES = {0: "MIPS_OK", 1: "MIPS_ERR_ARG", 2: "MIPS_ERR_NOMEM", 3: "MIPS_ERR_CUDA",
                4: "MIPS_ERR_TIMEOUT", 5: "MIPS_ERR_OVERFLOW", 6: "MIPS_ERR_UNIMPLEMENTED",
                7: "MIPS_ERR_NONFINITE"}
DTYPES = {"fp32": 0, "bf16": 1, "fp8": 2}
METHODS = {"bmm": 0, "maximus": 1, "select": 2}

# every symbol include/mips.h declares
EXPORTS = ("mips_default_options", "mips_build_index", "mips_topk", "mips_topk_maximus",
           "mips_select", "mips_topk_host", "mips_sync", "mips_get_stats", "mips_get_buffer",
           "mips_free_index", "mips_last_error", "mips_version", "mips_topk_noalloc", "mips_topk_graph",
           "mips_autotune", "mips_server_create", "mips_server_submit", "mips_server_wait",
           "mips_server_destroy", "mips_fit_clusters", "mips_test_expire_next_wait", "mips_select_arms")


class MipsError(RuntimeError):
    """A non-OK status from the library; ``status`` is the mips_status code
    and the message is mips_last_error()."""
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Options(ctypes.Structure):
    """mips_options (include/mips.h)."""
    _fields_ = [("dtype", ctypes.c_int), ("kmeans_iters", ctypes.c_int), ("block_items", ctypes.c_int),
                ("sample_frac", ctypes.c_double), ("autotune", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("kmeans_spherical", ctypes.c_int)]


class SelectReport(ctypes.Structure):
    """mips_select_report: the Optimus decision and its estimates."""
    _fields_ = [("choice", ctypes.c_int), ("t_build", ctypes.c_double), ("q_user", ctypes.c_double),
                ("m_user", ctypes.c_double), ("sample_users", ctypes.c_int64),
                ("est_index", ctypes.c_double), ("est_bmm", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


MAX_ARMS = 16


class ArmReport(ctypes.Structure):
    """mips_arm_report: one (index dtype, method) arm of mips_select_arms."""
    _fields_ = [("index", ctypes.c_int), ("dtype", ctypes.c_int), ("method", ctypes.c_int), ("rounds", ctypes.c_int),
                ("est_mean", ctypes.c_double), ("est_ci", ctypes.c_double), ("dropped", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ArmsReport(ctypes.Structure):
    """mips_arms_report: the multi-arm selector's timings and choice."""
    _fields_ = [("n_arms", ctypes.c_int), ("arm", ArmReport * MAX_ARMS), ("choice", ctypes.c_int),
                ("separated", ctypes.c_int), ("rounds", ctypes.c_int), ("sample_users", ctypes.c_int64),
                ("t_sample", ctypes.c_double), ("t_total", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "arm"}
        d["arms"] = [self.arm[i].as_dict() for i in range(self.n_arms)]
        return d


class TuneReport(ctypes.Structure):
    """mips_tune_report: the autotuner's choice and the candidates it timed."""
    _fields_ = [("clusters", ctypes.c_int), ("block_items", ctypes.c_int), ("sample_users", ctypes.c_int64),
                ("n_tried", ctypes.c_int), ("tried_clusters", ctypes.c_int * 32), ("tried_block", ctypes.c_int * 32),
                ("tried_est", ctypes.c_double * 32), ("t_tune", ctypes.c_double)]


class ServerOptions(ctypes.Structure):
    """mips_server_options: method, stream slots, batch size cap, memory budget."""
    _fields_ = [("method", ctypes.c_int), ("slots", ctypes.c_int), ("max_batch_users", ctypes.c_int64),
                ("mem_budget", ctypes.c_int64)]


class RequestInfo(ctypes.Structure):
    """mips_request_info: a served request's timestamps and the batch it ran in."""
    _fields_ = [("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("batch", ctypes.c_int64), ("batch_users", ctypes.c_int64), ("batch_K", ctypes.c_int),
                ("slot", ctypes.c_int), ("batch_bytes", ctypes.c_int64), ("batch_ws_bytes", ctypes.c_int64),
                ("inflight_bytes", ctypes.c_int64)]


class Stats(ctypes.Structure):
    """mips_stats: counters and per-stage times of the index's last call."""
    _fields_ = [("cand_emitted", ctypes.c_uint64), ("cand_rescored", ctypes.c_uint64),
                ("users_overflow", ctypes.c_uint64), ("users_fp64", ctypes.c_uint64),
                ("pairs_scored", ctypes.c_uint64), ("blocks_walked", ctypes.c_uint64),
                ("n_users", ctypes.c_int64), ("clusters", ctypes.c_int), ("dtype", ctypes.c_int),
                ("launches", ctypes.c_int), ("pad_", ctypes.c_int),
                ("ms_prep", ctypes.c_double), ("ms_score", ctypes.c_double), ("ms_rescore", ctypes.c_double),
                ("ms_kmeans", ctypes.c_double), ("ms_bounds", ctypes.c_double), ("ms_sort", ctypes.c_double),
                ("ms_walk", ctypes.c_double), ("ms_total", ctypes.c_double), ("select_slow", ctypes.c_uint64),
                ("ms_kernel", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


_lib = None


def load():
    """Load the in-tree library (build it with __graft_entry__.build() or
    paper_1706_01449_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmips.so not built ({LIB_PATH}); run paper_1706_01449_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    st = ctypes.c_int
    lib.mips_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.mips_default_options.restype = None
    lib.mips_build_index.argtypes = [P, i64, i32, i32, ctypes.POINTER(Options), P, ctypes.POINTER(P)]
    lib.mips_build_index.restype = st
    for name in ("mips_topk", "mips_topk_maximus"):
        fn = getattr(lib, name)
        fn.argtypes = [P, P, i64, i32, P, P, P]
        fn.restype = st
    lib.mips_fit_clusters.argtypes = [P, P, i64, P]
    lib.mips_fit_clusters.restype = st
    lib.mips_select.argtypes = [P, P, i64, i32, P, P, P, ctypes.POINTER(SelectReport)]
    lib.mips_select.restype = st
    lib.mips_select_arms.argtypes = [ctypes.POINTER(P), i32, P, i64, i32, i32, P, P, P, ctypes.POINTER(ArmsReport)]
    lib.mips_select_arms.restype = st
    lib.mips_topk_host.argtypes = [P, P, i64, i32, i32, P, P, P]
    lib.mips_topk_host.restype = st
    lib.mips_topk_graph.argtypes = [P, P, i64, i32, i32, P, P, P]
    lib.mips_topk_graph.restype = st
    lib.mips_autotune.argtypes = [P, P, i64, i32, P, ctypes.POINTER(TuneReport)]
    lib.mips_autotune.restype = st
    lib.mips_server_create.argtypes = [P, ctypes.POINTER(ServerOptions), ctypes.POINTER(P)]
    lib.mips_server_create.restype = st
    lib.mips_server_submit.argtypes = [P, P, i64, i32, P, P, ctypes.POINTER(i64)]
    lib.mips_server_submit.restype = st
    lib.mips_server_wait.argtypes = [P, i64, ctypes.c_double, ctypes.POINTER(RequestInfo)]
    lib.mips_server_wait.restype = st
    lib.mips_server_destroy.argtypes = [P]
    lib.mips_server_destroy.restype = st
    lib.mips_sync.argtypes = [P, P]
    lib.mips_sync.restype = st
    lib.mips_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.mips_get_stats.restype = st
    lib.mips_get_buffer.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(P), ctypes.POINTER(i64)]
    lib.mips_get_buffer.restype = st
    lib.mips_free_index.argtypes = [P]
    lib.mips_free_index.restype = None
    lib.mips_last_error.argtypes = []
    lib.mips_last_error.restype = ctypes.c_char_p
    lib.mips_topk_noalloc.argtypes = [P, i64, P, i64, i32, i32, P, P, P]
    lib.mips_topk_noalloc.restype = st
    lib.mips_test_expire_next_wait.argtypes = [i64]
    lib.mips_test_expire_next_wait.restype = st
    lib.mips_version.argtypes = []
    lib.mips_version.restype = i32
    _lib = lib
    return lib


def last_error() -> str:
    """The calling thread's last error message from the library."""
    return load().mips_last_error().decode()


def _check(status: int):
    if status != MIPS_OK:
        raise MipsError(status, last_error())


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f32(x, name):
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float32 or x.dim() != 2:
        raise TypeError(f"{name} must be a 2-D float32 CUDA tensor")
    return x.contiguous()


class Index:
    """Owning handle of a libmips index (frees it on close/deletion)."""

    def __init__(self, handle, f, n_items, clusters, dtype):
        self._h = handle
        self.f, self.n_items, self.clusters, self.dtype = f, n_items, clusters, dtype

    @property
    def handle(self):
        """The mips_index_t pointer (raises once the index is freed)."""
        if self._h is None:
            raise ValueError("index already freed")
        return self._h

    def close(self):
        """mips_free_index (waits for the index's work first); idempotent."""
        if self._h is not None and _lib is not None:
            _lib.mips_free_index(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_index(items, clusters: int = 8, dtype: str = "bf16", kmeans_iters: int = 3,
                block_items: int = 0, sample_frac: float = 0.005, seed: int = 0, kmeans_spherical: bool = False,
                stream=None) -> Index:
    """mips_build_index over a 2-D float32 CUDA tensor of items [n_items, f]:
    ``clusters`` is |C| for Maximus, ``dtype`` the candidate pass ("bf16" or
    "fp32"), the rest are mips_options fields.  Returns an owning Index."""
    lib = load()
    items = _dev_f32(items, "items")
    opt = Options()
    lib.mips_default_options(ctypes.byref(opt))
    opt.dtype = DTYPES[dtype]
    opt.kmeans_iters = kmeans_iters
    opt.block_items = block_items
    opt.sample_frac = sample_frac
    opt.seed = seed
    opt.kmeans_spherical = 1 if kmeans_spherical else 0
    h = ctypes.c_void_p()
    _check(lib.mips_build_index(ctypes.c_void_p(items.data_ptr()), items.shape[0], items.shape[1], clusters,
                                ctypes.byref(opt), _stream_ptr(stream), ctypes.byref(h)))
    return Index(h, items.shape[1], items.shape[0], clusters, dtype)


def _outputs(n, K, out_idx, out_score, device):
    import torch
    if out_idx is None:
        out_idx = torch.empty((n, K), dtype=torch.int32, device=device)
    if out_score is None:
        out_score = torch.empty((n, K), dtype=torch.float64, device=device)
    if out_idx.dtype != torch.int32 or out_score.dtype != torch.float64 or not out_idx.is_contiguous() \
            or not out_score.is_contiguous() or out_idx.numel() < n * K or out_score.numel() < n * K:
        raise TypeError("out_idx must be int32 and out_score float64, contiguous, n*K elements")
    return out_idx, out_score


def _run(fn, index, users, K, out_idx, out_score, stream):
    users = _dev_f32(users, "users")
    if users.shape[1] != index.f:
        raise ValueError("users have a different f than the index")
    out_idx, out_score = _outputs(users.shape[0], K, out_idx, out_score, users.device)
    _check(fn(index.handle, ctypes.c_void_p(users.data_ptr()), users.shape[0], K,
              ctypes.c_void_p(out_idx.data_ptr()), ctypes.c_void_p(out_score.data_ptr()), _stream_ptr(stream)))
    return out_idx, out_score


def topk(index: Index, users, K: int, out_idx=None, out_score=None, stream=None):
    """Blocked multiply + fused top-K (mips_topk).  Asynchronous on the stream."""
    return _run(load().mips_topk, index, users, K, out_idx, out_score, stream)


def topk_maximus(index: Index, users, K: int, out_idx=None, out_score=None, stream=None):
    """Maximus (mips_topk_maximus).  Asynchronous on the stream."""
    return _run(load().mips_topk_maximus, index, users, K, out_idx, out_score, stream)


def fit_clusters(index: Index, users, stream=None):
    """mips_fit_clusters: k-means on these users; later Maximus calls on the
    index assign their users to the fitted centroids (Sec. III-E, dynamic
    users).  users=None drops the fitted centroids.  Asynchronous."""
    lib = load()
    if users is None:
        _check(lib.mips_fit_clusters(index.handle, None, 0, None))
        return
    users = _dev_f32(users, "users")
    _check(lib.mips_fit_clusters(index.handle, ctypes.c_void_p(users.data_ptr()), users.shape[0],
                                 _stream_ptr(stream)))


def topk_graph(index: Index, users, K: int, method: str = "bmm", out_idx=None, out_score=None, stream=None):
    """mips_topk_graph: the blocked multiply ("bmm") or Maximus ("maximus")
    captured into a CUDA graph on the first call with these buffers and
    replayed afterwards.  Asynchronous on the stream."""
    lib = load()
    users = _dev_f32(users, "users")
    out_idx, out_score = _outputs(users.shape[0], K, out_idx, out_score, users.device)
    m = {"bmm": 0, "maximus": 1}[method]
    _check(lib.mips_topk_graph(index.handle, ctypes.c_void_p(users.data_ptr()), users.shape[0], K, m,
                               ctypes.c_void_p(out_idx.data_ptr()), ctypes.c_void_p(out_score.data_ptr()),
                               _stream_ptr(stream)))
    return out_idx, out_score


def autotune(index: Index, users, K: int, stream=None) -> dict:
    """mips_autotune: choose |C| and B for Maximus on a user sample; the
    choice becomes the index's.  Returns the report as a dict."""
    lib = load()
    users = _dev_f32(users, "users")
    rep = TuneReport()
    _check(lib.mips_autotune(index.handle, ctypes.c_void_p(users.data_ptr()), users.shape[0], K,
                             _stream_ptr(stream), ctypes.byref(rep)))
    n = rep.n_tried
    return {"clusters": rep.clusters, "block_items": rep.block_items, "sample_users": rep.sample_users,
            "t_tune": rep.t_tune,
            "tried": [(rep.tried_clusters[i], rep.tried_block[i], rep.tried_est[i]) for i in range(n)]}


def select(index: Index, users, K: int, out_idx=None, out_score=None, stream=None):
    """Optimus selector (mips_select): returns (idx, score, report dict)."""
    lib = load()
    users = _dev_f32(users, "users")
    out_idx, out_score = _outputs(users.shape[0], K, out_idx, out_score, users.device)
    rep = SelectReport()
    _check(lib.mips_select(index.handle, ctypes.c_void_p(users.data_ptr()), users.shape[0], K,
                           ctypes.c_void_p(out_idx.data_ptr()), ctypes.c_void_p(out_score.data_ptr()),
                           _stream_ptr(stream), ctypes.byref(rep)))
    return out_idx, out_score, rep.as_dict()


def select_arms(indexes, users, K: int, max_rounds: int = 0, out_idx=None, out_score=None, stream=None):
    """Multi-arm selector (mips_select_arms) over indexes built on the same
    items: returns (idx, score, report dict)."""
    lib = load()
    users = _dev_f32(users, "users")
    out_idx, out_score = _outputs(users.shape[0], K, out_idx, out_score, users.device)
    handles = (ctypes.c_void_p * len(indexes))(*[ix.handle.value for ix in indexes])
    rep = ArmsReport()
    _check(lib.mips_select_arms(handles, len(indexes), ctypes.c_void_p(users.data_ptr()), users.shape[0], K,
                                max_rounds, ctypes.c_void_p(out_idx.data_ptr()), ctypes.c_void_p(out_score.data_ptr()),
                                _stream_ptr(stream), ctypes.byref(rep)))
    return out_idx, out_score, rep.as_dict()


def topk_host(index: Index, users_host, K: int, method: str = "bmm", out_idx=None, out_score=None,
              stream=None):
    """Host-buffer variant (mips_topk_host): numpy or pinned-torch CPU arrays
    in, host arrays out; synchronous."""
    import numpy as np
    import torch
    if isinstance(users_host, np.ndarray):
        users_host = torch.from_numpy(np.ascontiguousarray(users_host, dtype=np.float32))
    n = users_host.shape[0]
    if out_idx is None:
        out_idx = torch.empty((n, K), dtype=torch.int32, pin_memory=users_host.is_pinned())
    if out_score is None:
        out_score = torch.empty((n, K), dtype=torch.float64, pin_memory=users_host.is_pinned())
    _check(load().mips_topk_host(index.handle, ctypes.c_void_p(users_host.data_ptr()), n, K, METHODS[method],
                                 ctypes.c_void_p(out_idx.data_ptr()), ctypes.c_void_p(out_score.data_ptr()),
                                 _stream_ptr(stream)))
    return out_idx, out_score


def sync(index: Index, stream=None):
    """mips_sync: wait for the stream and raise on any device-side error."""
    _check(load().mips_sync(index.handle, _stream_ptr(stream)))


def get_stats(index: Index) -> dict:
    """mips_get_stats of the index's last call, as a dict."""
    st = Stats()
    _check(load().mips_get_stats(index.handle, ctypes.byref(st)))
    return st.as_dict()


def get_buffer(index: Index, name: str, dtype, shape):
    """Copy of an internal device array (see mips_get_buffer) as a torch tensor."""
    import torch
    p = ctypes.c_void_p()
    nbytes = ctypes.c_int64()
    _check(load().mips_get_buffer(index.handle, name.encode(), ctypes.byref(p), ctypes.byref(nbytes)))
    typestr = {torch.float32: "<f4", torch.int32: "<i4", torch.float64: "<f8", torch.int64: "<i8"}[dtype]
    esize = torch.empty((), dtype=dtype).element_size()
    count = 1
    for d in shape:
        count *= d
    if count * esize != nbytes.value:
        raise ValueError(f"buffer {name} holds {nbytes.value} bytes, shape asks for {count * esize}")

    class _View:
        __cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (p.value, False),
                                    "version": 3, "strides": None}

    return torch.as_tensor(_View(), device="cuda").clone()


def topk_noalloc(items, users, K: int, out_idx, out_score, stream=None):
    """mips_topk_noalloc: exact top-K on caller-owned device buffers with no
    device allocation inside the library (scratch is a static 32 MiB device
    array shared by all calls; serialise calls).  Synchronous."""
    items = _dev_f32(items, "items")
    users = _dev_f32(users, "users")
    if users.shape[1] != items.shape[1]:
        raise ValueError("users and items differ in f")
    out_idx, out_score = _outputs(users.shape[0], K, out_idx, out_score, users.device)
    _check(load().mips_topk_noalloc(ctypes.c_void_p(items.data_ptr()), items.shape[0],
                                    ctypes.c_void_p(users.data_ptr()), users.shape[0], users.shape[1], K,
                                    ctypes.c_void_p(out_idx.data_ptr()), ctypes.c_void_p(out_score.data_ptr()),
                                    _stream_ptr(stream)))
    return out_idx, out_score


def test_expire_next_wait(wait_ns: int):
    """Tests of the bounded device waits: the next tensor-core score launch
    publishes no work item, so its waits run out after wait_ns ns and the
    call's sync raises MIPS_ERR_TIMEOUT (one launch only)."""
    _check(load().mips_test_expire_next_wait(int(wait_ns)))


def free_index(index: Index):
    """Free the index now (same as index.close())."""
    index.close()


class Server:
    """Request loop with continuous batching (mips_server_*): submit host
    user rows with any K, wait for each request's results.  The index must
    outlive the server."""

    def __init__(self, index: Index, method: str = "bmm", slots: int = 2, max_batch_users: int = 8192,
                 mem_budget: int = 0):
        lib = load()
        opt = ServerOptions({"bmm": 0, "maximus": 1}[method], slots, max_batch_users, mem_budget)
        h = ctypes.c_void_p()
        _check(lib.mips_server_create(index.handle, ctypes.byref(opt), ctypes.byref(h)))
        self._h, self._index, self._live = h, index, {}

    def submit(self, users, K: int) -> int:
        """users: numpy float32 [n, f] (copied to a C-contiguous array kept
        alive until wait).  Returns the request id."""
        import numpy as np
        u = np.ascontiguousarray(users, dtype=np.float32)
        if u.ndim != 2 or u.shape[1] != self._index.f:
            raise TypeError(f"users must be [n, {self._index.f}] float32")
        oi = np.empty((u.shape[0], K), dtype=np.int32)
        osc = np.empty((u.shape[0], K), dtype=np.float64)
        rid = ctypes.c_int64()
        _check(load().mips_server_submit(self._h, u.ctypes.data, u.shape[0], K, oi.ctypes.data, osc.ctypes.data,
                                         ctypes.byref(rid)))
        self._live[rid.value] = (u, oi, osc)
        return rid.value

    def wait(self, rid: int, timeout: float = 60.0):
        """Returns (idx, score, info dict) of the request."""
        info = RequestInfo()
        st = load().mips_server_wait(self._h, rid, timeout, ctypes.byref(info))
        if st == MIPS_ERR_TIMEOUT:
            raise TimeoutError(last_error())
        _check(st)
        u, oi, osc = self._live.pop(rid)
        return oi, osc, {k: getattr(info, k) for k, _ in RequestInfo._fields_}

    def close(self):
        """mips_server_destroy: finish the queued requests and release the server."""
        if self._h is not None:
            _check(load().mips_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
