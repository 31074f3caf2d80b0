"""GB300 (sm_103a) DartMinHash: Python binding of libdartminhash.so.

Argument marshalling only: every step of the hot path runs in the library's CUDA kernels.
The functions carry the C ABI's names (include/dartminhash.h) and take torch tensors that
already live on the GPU (the ``*_host`` entry takes host tensors).  There is no CPU
fallback: if the library is missing or fails to load, every call raises.

    ctx = dm_create(device=0)
    keys = dm_sketch(ctx, indptr, indices, weights, k=256, seed=1)       # uint64 as int64
    words = dm_sketch_bbit(ctx, indptr, indices, weights, k=256, b=1, seed=1)
    dm_sync_status(ctx)   # raises DartMinHashError on a device-detected input error
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB, LIB_CHECKED, build

__all__ = ["DartMinHashError", "dm_create", "dm_destroy", "dm_sketch", "dm_sketch_bbit", "dm_lsh",
           "dm_sketch_host", "dm_bottomk", "dm_compare", "dm_compare_topk", "dm_lsh_scaled", "dm_weight_classes", "LshIndex", "estimate_jaccard", "dm_sync_status", "dm_strerror", "dm_set_option", "dm_t_of_k",
           "dm_poisson_thresholds", "dm_sketch_noalloc", "NOALLOC_MAX_SETS", "load", "build", "LIB", "LIB_CHECKED",
           "dm_build_flags", "ECHECK", "OPT_PHI0", "OPT_COUNTERS", "OPT_FORM",
           "OPT_WARPS_PER_BLOCK", "OPT_LSH_PHI0", "OPT_LARGE_NNZ", "OPT_GRAPH", "OPT_TUNED", "OPT_LARGE_WORK", "OPT_HOST_CHUNKS", "OPT_HOST_MODE", "OPT_SLOTS", "SLOTS_AUTO", "SLOTS_SHARED", "SLOTS_ROW", "HOST_STAGED", "HOST_IN_PLACE", "HOST_AUTO", "FORM_BATCHED",
           "FORM_PLAIN", "FORM_PERSISTENT", "dm_autotune", "Tuning", "Server", "EAGAIN"]

OPT_PHI0, OPT_COUNTERS, OPT_FORM, OPT_WARPS_PER_BLOCK, OPT_LSH_PHI0, OPT_LARGE_NNZ = 1, 2, 3, 4, 5, 6
OPT_GRAPH, OPT_TUNED, OPT_LARGE_WORK, OPT_HOST_CHUNKS, OPT_HOST_MODE, OPT_SLOTS = 7, 8, 9, 10, 11, 12
SLOTS_AUTO, SLOTS_SHARED, SLOTS_ROW = 0, 1, 2
HOST_STAGED, HOST_IN_PLACE, HOST_AUTO = 0, 1, 2
EAGAIN, ETIMEOUT, ECHECK = 7, 4, 8
FORM_BATCHED, FORM_PLAIN, FORM_PERSISTENT = 0, 1, 2
_lock = threading.Lock()
_lib = None


class DartMinHashError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = dm_strerror(code) if _lib is not None else str(code)
        super().__init__(f"{what}: DM status {code} ({msg})")
        self.code = code


def load(path: str | None = None):
    """Load libdartminhash.so (built in-tree by build()), or the library at `path` (e.g.
    LIB_CHECKED, the checked build), once per process.  Raises if it is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libdartminhash.so is not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
        sig = {
            "dm_create": ([ctypes.POINTER(P), ctypes.c_int, ctypes.c_size_t], ctypes.c_int),
            "dm_destroy": ([P], ctypes.c_int),
            "dm_sketch": ([P, P, P, P, i64, i32, u64, P, P], ctypes.c_int),
            "dm_sketch_bbit": ([P, P, P, P, i64, i32, i32, u64, P, P, P], ctypes.c_int),
            "dm_lsh": ([P, P, P, P, i64, i32, i32, u64, P, P], ctypes.c_int),
            "dm_bottomk": ([P, P, P, P, i64, i32, u64, P, P], ctypes.c_int),
            "dm_compare": ([P, P, P, i64, i64, i32, i32, i32, P, P], ctypes.c_int),
            "dm_estimate_jaccard": ([P, i64, i32, i32, P, P], ctypes.c_int),
            "dm_compare_topk": ([P, P, P, i64, i64, i32, i32, i32, P, P, P], ctypes.c_int),
            "dm_lsh_scaled": ([P, P, P, P, i64, i32, i32, u64, P, P, P], ctypes.c_int),
            "dm_lsh_index_create": ([ctypes.POINTER(P), ctypes.c_int, i32, i64], ctypes.c_int),
            "dm_lsh_index_insert": ([P, P, P, i64, P], ctypes.c_int),
            "dm_lsh_index_query": ([P, P, i64, i32, P, P, P], ctypes.c_int),
            "dm_lsh_index_size": ([P, P], ctypes.c_int),
            "dm_lsh_index_status": ([P, P], ctypes.c_int),
            "dm_lsh_index_destroy": ([P], ctypes.c_int),
            "dm_weight_classes": ([P, P, P, i64, P, P, i32, P], ctypes.c_int),
            "dm_sketch_host": ([P, P, P, P, i64, i32, i32, u64, P, P, P], ctypes.c_int),
            "dm_sketch_f64": ([P, P, P, P, i64, i32, u64, P, P], ctypes.c_int),
            "dm_sketch_f64_bbit": ([P, P, P, P, i64, i32, i32, u64, P, P, P], ctypes.c_int),
            "dm_mix64_burn": ([i64, i32, u64, P, P], ctypes.c_int),
            "dm_sync_status": ([P, P], ctypes.c_int),
            "dm_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "dm_build_flags": ([], ctypes.c_int32),
            "dm_set_option": ([P, ctypes.c_int, i64], ctypes.c_int),
            "dm_t_of_k": ([i32], i64),
            "dm_set_tuning": ([P, i32, i32, i32, P], ctypes.c_int),
            "dm_poisson_thresholds": ([P], None),
            "dm_sketch_noalloc": ([P, P, P, i64, i32, u64, P, P], ctypes.c_int),
            "dm_autotune": ([P, P, P, P, i64, i32, i32, i32, u64, i64, P, P], ctypes.c_int),
            "dm_server_create": ([ctypes.POINTER(P), P], ctypes.c_int),
            "dm_server_destroy": ([P], ctypes.c_int),
            "dm_server_submit": ([P, P, P, i64, i32, u64, P, P], ctypes.c_int),
            "dm_server_poll": ([P, i64, P], ctypes.c_int),
            "dm_server_wait": ([P, i64, i64, P], ctypes.c_int),
            "dm_server_replay": ([P, i64, P, P, P, P, P, P, P, P, P], ctypes.c_int),
            "dm_server_get_stats": ([P, P], ctypes.c_int),
            "dm_server_reset_stats": ([P], ctypes.c_int),
            "dm_server_fail_batches": ([P, i32], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int, what: str):
    if rc != 0:
        raise DartMinHashError(rc, what)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_ptr(t, dtype_name, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    want = {"int64": (torch.int64,), "int32": (torch.int32,), "uint32": (torch.int32, torch.uint32),
            "float32": (torch.float32,), "float64": (torch.float64,),
            "uint64": (torch.int64, torch.uint64)}[dtype_name]
    if t.dtype not in want:
        raise TypeError(f"{what} must be {dtype_name} (got {t.dtype})")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """Owns a dm_ctx*."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.dm_create(ctypes.byref(h), int(device), int(mem_budget_bytes)), "dm_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            load().dm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dm_create(device: int = 0, mem_budget_bytes: int = 0) -> Context:
    return Context(device, mem_budget_bytes)


def dm_destroy(ctx: Context) -> None:
    ctx.close()


def _need(t, numel: int, what: str):
    """A caller-provided output must hold exactly the values the call writes."""
    if t is not None and t.numel() != numel:
        raise ValueError(f"{what} must hold {numel} values (got {t.numel()})")


def _csr_ptrs(indptr, indices, weights):
    n = indptr.numel() - 1
    return (n, _dev_ptr(indptr, "int64", "indptr"), _dev_ptr(indices, "uint32", "indices"),
            _dev_ptr(weights, "float32", "weights"))


def dm_sketch(ctx: Context, indptr, indices, weights, k: int, seed: int, out=None, stream=None):
    """uint64[n_sets, k] minhash keys (returned as an int64 tensor holding the same bits)."""
    import torch
    n, ip, ix, w = _csr_ptrs(indptr, indices, weights)
    if out is None:
        out = torch.empty((n, k), dtype=torch.int64, device=indptr.device)
    elif out.numel() != n * k:
        raise ValueError("out has the wrong size")
    _check(load().dm_sketch(ctx.handle, ip, ix, w, n, int(k), int(seed) & (2**64 - 1),
                            _dev_ptr(out, "uint64", "out"), _stream(stream)), "dm_sketch")
    return out


def dm_sketch_f64(ctx: Context, indptr, indices, weights, k: int, seed: int, out=None, stream=None):
    """Wide-range minhash keys uint64[n_sets, k] (int64 tensor holding the same bits) of sets with
    64-bit ids (int64 or uint64 tensor) and binary64 weights (float64 tensor)."""
    import torch
    n = indptr.numel() - 1
    ip = _dev_ptr(indptr, "int64", "indptr")
    ix = _dev_ptr(indices, "uint64", "indices")
    w = _dev_ptr(weights, "float64", "weights")
    if out is None:
        out = torch.empty((n, k), dtype=torch.int64, device=indptr.device)
    elif out.numel() != n * k:
        raise ValueError("out has the wrong size")
    _check(load().dm_sketch_f64(ctx.handle, ip, ix, w, n, int(k), int(seed) & (2**64 - 1),
                                _dev_ptr(out, "uint64", "out"), _stream(stream)), "dm_sketch_f64")
    return out


def dm_sketch_f64_bbit(ctx: Context, indptr, indices, weights, k: int, b: int, seed: int, out_words=None,
                       out_keys=None, stream=None):
    """b-bit words uint64[n_sets, ceil(k b / 64)] (int64 tensor) of the wide-range keys; fills
    out_keys too when given."""
    import torch
    n = indptr.numel() - 1
    ip = _dev_ptr(indptr, "int64", "indptr")
    ix = _dev_ptr(indices, "uint64", "indices")
    w = _dev_ptr(weights, "float64", "weights")
    words = (k * b + 63) // 64
    if out_words is None:
        out_words = torch.empty((n, words), dtype=torch.int64, device=indptr.device)
    _need(out_words, n * words, "out_words")
    _need(out_keys, n * k, "out_keys")
    kp = _dev_ptr(out_keys, "uint64", "out_keys") if out_keys is not None else None
    _check(load().dm_sketch_f64_bbit(ctx.handle, ip, ix, w, n, int(k), int(b), int(seed) & (2**64 - 1),
                                     _dev_ptr(out_words, "uint64", "out_words"), kp, _stream(stream)),
           "dm_sketch_f64_bbit")
    return out_words


def dm_mix64_burn(blocks: int, iters: int, seed: int = 1, out=None, stream=None):
    """The hash's integer-issue ceiling: 4 * iters chained mixes per thread, blocks * 256 threads
    (see the C declaration).  Returns the output tensor (int64[blocks * 256])."""
    import torch
    if out is None:
        out = torch.empty(blocks * 256, dtype=torch.int64, device="cuda")
    _need(out, blocks * 256, "out")
    _check(load().dm_mix64_burn(int(blocks), int(iters), int(seed) & (2**64 - 1), _dev_ptr(out, "uint64", "out"),
                                _stream(stream)), "dm_mix64_burn")
    return out


def dm_sketch_bbit(ctx: Context, indptr, indices, weights, k: int, b: int, seed: int, out_words=None,
                   out_keys=None, stream=None):
    """b-bit packed sketches uint64[n_sets, ceil(k b / 64)] (int64 tensor); fills out_keys too
    when given."""
    import torch
    n, ip, ix, w = _csr_ptrs(indptr, indices, weights)
    words = (k * b + 63) // 64
    if out_words is None:
        out_words = torch.empty((n, words), dtype=torch.int64, device=indptr.device)
    _need(out_words, n * words, "out_words")
    _need(out_keys, n * k, "out_keys")
    kp = _dev_ptr(out_keys, "uint64", "out_keys") if out_keys is not None else None
    _check(load().dm_sketch_bbit(ctx.handle, ip, ix, w, n, int(k), int(b), int(seed) & (2**64 - 1),
                                 _dev_ptr(out_words, "uint64", "out_words"), kp, _stream(stream)),
           "dm_sketch_bbit")
    return out_words


def dm_lsh(ctx: Context, indptr, indices, weights, L: int, K: int, seed: int, out=None, stream=None):
    """uint32[n_sets, L] (L, K) LSH values (returned as an int32 tensor holding the same bits)."""
    import torch
    n, ip, ix, w = _csr_ptrs(indptr, indices, weights)
    if out is None:
        out = torch.empty((n, L), dtype=torch.int32, device=indptr.device)
    _need(out, n * L, "out")
    _check(load().dm_lsh(ctx.handle, ip, ix, w, n, int(L), int(K), int(seed) & (2**64 - 1),
                         _dev_ptr(out, "uint32", "out"), _stream(stream)), "dm_lsh")
    return out


def dm_lsh_scaled(ctx: Context, indptr, indices, weights, L: int, K: int, seed: int, scale_exp, out=None,
                  stream=None):
    """dm_lsh with set s's weights counted as x_i 2^scale_exp[s] (int32 CUDA tensor)."""
    import torch
    n, ip, ix, w = _csr_ptrs(indptr, indices, weights)
    if out is None:
        out = torch.empty((n, L), dtype=torch.int32, device=indptr.device)
    if scale_exp.numel() != n:
        raise ValueError("one scale per set")
    _need(out, n * L, "out")
    _check(load().dm_lsh_scaled(ctx.handle, ip, ix, w, n, int(L), int(K), int(seed) & (2**64 - 1),
                                _dev_ptr(scale_exp, "int32", "scale_exp"), _dev_ptr(out, "uint32", "out"),
                                _stream(stream)), "dm_lsh_scaled")
    return out


class LshIndex:
    """Owns a dm_lsh_index*: L hash tables of LSH values on a device."""

    def __init__(self, L: int, capacity: int, device: int = 0):
        h = ctypes.c_void_p()
        _check(load().dm_lsh_index_create(ctypes.byref(h), int(device), int(L), int(capacity)), "dm_lsh_index_create")
        self.handle, self.L = h, L

    def insert(self, values, ids=None, stream=None):
        n = values.shape[0]
        _need(values, n * self.L, "values")
        _need(ids, n, "ids")
        _check(load().dm_lsh_index_insert(self.handle, _dev_ptr(values, "uint32", "values"),
                                          _dev_ptr(ids, "int64", "ids") if ids is not None else None, n,
                                          _stream(stream)), "dm_lsh_index_insert")

    def query(self, values, max_candidates: int, stream=None):
        """(counts int32[m], ids int64[m, max_candidates]) as CUDA tensors."""
        import torch
        m = values.shape[0]
        _need(values, m * self.L, "values")
        counts = torch.empty(m, dtype=torch.int32, device=values.device)
        ids = torch.empty((m, max_candidates), dtype=torch.int64, device=values.device)
        _check(load().dm_lsh_index_query(self.handle, _dev_ptr(values, "uint32", "values"), m, int(max_candidates),
                                         _dev_ptr(counts, "int32", "counts"), _dev_ptr(ids, "int64", "ids"),
                                         _stream(stream)), "dm_lsh_index_query")
        return counts, ids

    def size(self) -> int:
        n = ctypes.c_int64()
        _check(load().dm_lsh_index_size(self.handle, ctypes.cast(ctypes.byref(n), ctypes.c_void_p)), "dm_lsh_index_size")
        return n.value

    def status(self, stream=None) -> int:
        return int(load().dm_lsh_index_status(self.handle, _stream(stream)))

    def close(self):
        if self.handle:
            load().dm_lsh_index_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dm_weight_classes(ctx: Context, indptr, weights, out=None, scale_out=None, norm_exp: int = 0, stream=None):
    """int32 weight class floor(log2 ||x||_1) of each set, from the exact sum of its positive
    finite weights (0 for a set without one); scale_out, when given, receives norm_exp - class,
    the scales that put every class's norms in [2^norm_exp, 2^(norm_exp+1))."""
    import torch
    n = indptr.numel() - 1
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=indptr.device)
    _need(out, n, "out")
    _need(scale_out, n, "scale_out")
    _check(load().dm_weight_classes(ctx.handle, _dev_ptr(indptr, "int64", "indptr"),
                                    _dev_ptr(weights, "float32", "weights"), n, _dev_ptr(out, "int32", "out"),
                                    _dev_ptr(scale_out, "int32", "scale_out") if scale_out is not None else None,
                                    int(norm_exp), _stream(stream)), "dm_weight_classes")
    return out


def dm_bottomk(ctx: Context, indptr, indices, weights, k: int, seed: int, out=None, stream=None):
    """uint64[n_sets, k] bottom-k sketches: each row the k smallest keys in increasing order
    (returned as an int64 tensor holding the same bits)."""
    import torch
    n, ip, ix, w = _csr_ptrs(indptr, indices, weights)
    if out is None:
        out = torch.empty((n, k), dtype=torch.int64, device=indptr.device)
    elif out.numel() != n * k:
        raise ValueError("out has the wrong size")
    _check(load().dm_bottomk(ctx.handle, ip, ix, w, n, int(k), int(seed) & (2**64 - 1),
                             _dev_ptr(out, "uint64", "out"), _stream(stream)), "dm_bottomk")
    return out


def dm_compare(ctx: Context, a, c, k: int, bits: int = 0, cross: bool = False, out=None, stream=None):
    """Agreeing slots per pair of sketch rows (uint32 as int32 tensor): rows of a with the same
    rows of c, or (cross=True) every row of a with every row of c.  a, c: int64 tensors holding
    uint64 keys [n, k] (bits = 0) or packed b-bit words [n, ceil(k b / 64)]."""
    import torch
    na, nc = a.shape[0], c.shape[0]
    if not cross and na != nc:
        raise ValueError("pairs need the same number of rows")
    if k >= 1 and bits in (0, 1, 2, 4, 8, 16, 32):        # other values: the library rejects them
        row = k if bits == 0 else (k * bits + 63) // 64
        _need(a, na * row, "a")
        _need(c, nc * row, "c")
    if out is None:
        out = torch.empty((na, nc) if cross else (na,), dtype=torch.int32, device=a.device)
    _need(out, na * nc if cross else na, "out")
    _check(load().dm_compare(ctx.handle, _dev_ptr(a, "uint64", "a"), _dev_ptr(c, "uint64", "c"), na, nc, int(k),
                             int(bits), 1 if cross else 0, _dev_ptr(out, "uint32", "out"), _stream(stream)),
           "dm_compare")
    return out


def dm_compare_topk(ctx: Context, a, c, k: int, topk: int, bits: int = 0, out_idx=None, out_count=None,
                    stream=None):
    """For each row of a, the `topk` rows of c with the most agreeing slots (ties: smaller row
    first), as (rows, counts): uint32 tensors (int32 holding the same bits) of shape
    (n_a, topk); rows past n_c are 0xFFFFFFFF with count 0.  Rows as for dm_compare."""
    import torch
    n_a, n_c = a.shape[0], c.shape[0]
    if k >= 1 and bits in (0, 1, 2, 4, 8, 16, 32):        # other values: the library rejects them
        row = k if bits == 0 else (k * bits + 63) // 64
        _need(a, n_a * row, "a")
        _need(c, n_c * row, "c")
    if out_idx is None:
        out_idx = torch.empty((n_a, topk), dtype=torch.int32, device=a.device)
    if out_count is None:
        out_count = torch.empty((n_a, topk), dtype=torch.int32, device=a.device)
    _need(out_idx, n_a * topk, "out_idx")
    _need(out_count, n_a * topk, "out_count")
    _check(load().dm_compare_topk(ctx.handle, _dev_ptr(a, "uint64", "a"), _dev_ptr(c, "uint64", "c"), n_a, n_c,
                                  int(k), int(bits), int(topk), _dev_ptr(out_idx, "uint32", "out_idx"),
                                  _dev_ptr(out_count, "uint32", "out_count"), _stream(stream)), "dm_compare_topk")
    return out_idx, out_count


def estimate_jaccard(matches, k: int, bits: int = 0, out=None, stream=None):
    """Weighted Jaccard estimates (float64 tensor) from dm_compare's agreeing-slot counts, computed
    by the library (dm_estimate_jaccard): m / k for keys, (m / k - 2^-b) / (1 - 2^-b) for b-bit
    fields.  matches: uint32 counts (int32 CUDA tensor), as dm_compare returns them."""
    import torch
    n = matches.numel()
    if out is None:
        out = torch.empty(matches.shape, dtype=torch.float64, device=matches.device)
    _need(out, n, "out")
    _check(load().dm_estimate_jaccard(_dev_ptr(matches, "uint32", "matches"), n, int(k), int(bits),
                                      _dev_ptr(out, "float64", "out"), _stream(stream)), "dm_estimate_jaccard")
    return out


def dm_sketch_host(ctx: Context, indptr, indices, weights, k: int, seed: int, out_keys=None, b: int = 0,
                   out_words=None, stream=None):
    """dm_sketch (b = 0) or dm_sketch_bbit (b > 0) on host tensors (pinned memory for full copy
    speed); synchronous.  Returns (out_keys, out_words)."""
    import torch
    n = indptr.numel() - 1
    words = (k * b + 63) // 64 if b else 0
    if out_keys is None and b == 0:
        out_keys = torch.empty((n, k), dtype=torch.int64)
    if out_words is None and b > 0:
        out_words = torch.empty((n, words), dtype=torch.int64)
    for t in (indptr, indices, weights, out_keys, out_words):
        if t is not None and (t.is_cuda or not t.is_contiguous()):
            raise ValueError("host entry takes contiguous CPU tensors")
    if out_keys is not None and out_keys.numel() != n * k:
        raise ValueError("out_keys must hold n_sets * k values")
    if out_words is not None and out_words.numel() != n * words:
        raise ValueError("out_words must hold n_sets * ceil(k b / 64) words")
    P = ctypes.c_void_p
    _check(load().dm_sketch_host(ctx.handle, P(indptr.data_ptr()), P(indices.data_ptr()),
                                 P(weights.data_ptr()), n, int(k), int(b), int(seed) & (2**64 - 1),
                                 P(out_keys.data_ptr()) if out_keys is not None else None,
                                 P(out_words.data_ptr()) if out_words is not None else None,
                                 _stream(stream)), "dm_sketch_host")
    return out_keys, out_words


def dm_sketch_noalloc(indptr, indices, weights, k: int, seed: int, out, stream=None):
    """dm_sketch for programs that forbid the library's own device allocations: no context, the
    scratch is a fixed array inside the library (at most DM_NOALLOC_MAX_SETS sets per call;
    overlapping calls race).  `out` must be given; all four tensors must be on one device, which
    the call makes current.  Synchronous (so never on a stream under graph capture); raises on
    any error."""
    import torch
    n, ip, ix, w = _csr_ptrs(indptr, indices, weights)
    if out.numel() != n * k:
        raise ValueError("out must hold n_sets * k keys")
    po = _dev_ptr(out, "uint64", "out")
    dev = indptr.device
    if any(t.device != dev for t in (indices, weights, out)):
        raise ValueError("indptr, indices, weights and out must be on one device")
    with torch.cuda.device(dev):                 # the library runs on the current device
        _check(load().dm_sketch_noalloc(ip, ix, w, n, int(k), int(seed) & (2**64 - 1), po, _stream(stream)),
               "dm_sketch_noalloc")
    return out


NOALLOC_MAX_SETS = 262144


class Tuning(ctypes.Structure):
    """dm_tuning: the settings dm_autotune chose."""
    _fields_ = [("form", ctypes.c_int32), ("warps_per_block", ctypes.c_int32), ("phi0_1024", ctypes.c_int32),
                ("large_nnz", ctypes.c_int32), ("large_work", ctypes.c_int32), ("sets_timed", ctypes.c_int64),
                ("ms_default", ctypes.c_float), ("ms_tuned", ctypes.c_float), ("slots", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def dm_autotune(ctx: Context, indptr, indices, weights, k: int, seed: int, b: int = 0, lsh_K: int = 0,
                max_sets: int = 0, stream=None, bottomk: bool = False) -> dict:
    """Time launch settings on a prefix of a device batch and store the fastest in the context
    for later calls of the same kind.  Sketches: k, b (0 = keys only); LSH: k = L and lsh_K = K;
    bottom-k sketches: k and bottomk=True."""
    n, ip, ix, w = _csr_ptrs(indptr, indices, weights)
    res = Tuning()
    lsh = 2 if bottomk else (1 if lsh_K > 0 else 0)
    _check(load().dm_autotune(ctx.handle, ip, ix, w, n, lsh, int(k), int(lsh_K if lsh else b),
                              int(seed) & (2**64 - 1), int(max_sets), ctypes.cast(ctypes.byref(res), ctypes.c_void_p),
                              _stream(stream)), "dm_autotune")
    return res.as_dict()


def dm_set_tuning(ctx: Context, k: int, tuning: dict, b: int = 0, lsh_K: int = 0, bottomk: bool = False) -> None:
    """Reinstall settings (a dict as dm_autotune returns) for later calls of that kind."""
    t = Tuning()
    for f in ("form", "warps_per_block", "phi0_1024", "large_nnz", "large_work"):
        setattr(t, f, int(tuning[f]))
    t.slots = int(tuning.get("slots", 0))
    lsh = 2 if bottomk else (1 if lsh_K > 0 else 0)
    _check(load().dm_set_tuning(ctx.handle, lsh, int(k), int(lsh_K if lsh else b),
                                ctypes.cast(ctypes.byref(t), ctypes.c_void_p)), "dm_set_tuning")


def save_tunings(path: str, entries) -> None:
    """Write dm_autotune results to a JSON file, keyed by the GPU model: entries is a list of
    {"k", "b", "lsh_K", "bottomk", "tuning"} dicts."""
    import json
    import torch
    data = {}
    if os.path.exists(path):
        data = json.load(open(path))
    data[torch.cuda.get_device_name()] = list(entries)
    with open(path, "w") as f:
        json.dump(data, f, indent=1)


def load_tunings(ctx: Context, path: str) -> int:
    """Install the saved settings of this GPU model into a context; returns how many."""
    import json
    import torch
    if not os.path.exists(path):
        return 0
    entries = json.load(open(path)).get(torch.cuda.get_device_name(), [])
    for e in entries:
        dm_set_tuning(ctx, e["k"], e["tuning"], b=e.get("b", 0), lsh_K=e.get("lsh_K", 0),
                      bottomk=e.get("bottomk", False))
    return len(entries)


def dm_sync_status(ctx: Context, stream=None, raise_on_error: bool = True) -> int:
    rc = load().dm_sync_status(ctx.handle, _stream(stream))
    if rc and raise_on_error:
        raise DartMinHashError(rc, "device status")
    return rc


def dm_strerror(code: int) -> str:
    return load().dm_strerror(int(code)).decode()


def dm_build_flags() -> int:
    """Build flags of the loaded library: bit 0 = the checked build (index checks in every kernel,
    failures reported as DM_ECHECK by dm_sync_status)."""
    return int(load().dm_build_flags())


def dm_set_option(ctx: Context, option: int, value: int) -> None:
    _check(load().dm_set_option(ctx.handle, int(option), int(value)), "dm_set_option")


def dm_t_of_k(k: int) -> int:
    return int(load().dm_t_of_k(int(k)))


def dm_poisson_thresholds():
    arr = (ctypes.c_uint32 * 12)()
    load().dm_poisson_thresholds(ctypes.cast(arr, ctypes.c_void_p))
    return [int(v) for v in arr]


class ServerConfig(ctypes.Structure):
    """dm_server_config."""
    _fields_ = [("device", ctypes.c_int32), ("lanes", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_size_t),
                ("lane_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int32), ("max_wait_us", ctypes.c_int32),
                ("per_request", ctypes.c_int32), ("large_nnz", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    """dm_server_stats."""
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("batches", ctypes.c_int64), ("admitted_bytes", ctypes.c_int64),
                ("mean_batch", ctypes.c_double), ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("groups", ctypes.c_int64), ("kernel_launches", ctypes.c_int64)]


def _host_ptr(a, dtype, what):
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.dtype(dtype) or not a.flags.c_contiguous:
        raise TypeError(f"{what} must be a contiguous numpy {dtype} array")
    return ctypes.c_void_p(a.ctypes.data)


class Server:
    """Owns a dm_server*: continuous batching of single-set requests (host arrays)."""

    def __init__(self, device: int = 0, lanes: int = 0, mem_budget_bytes: int = 0, lane_bytes: int = 0,
                 max_batch: int = 0, max_wait_us: int = 0, per_request: bool = False, large_nnz: int = 0):
        cfg = ServerConfig(device, lanes, mem_budget_bytes, lane_bytes, max_batch, max_wait_us,
                           1 if per_request else 0, large_nnz)
        h = ctypes.c_void_p()
        _check(load().dm_server_create(ctypes.byref(h), ctypes.cast(ctypes.byref(cfg), ctypes.c_void_p)),
               "dm_server_create")
        self.handle = h
        self._keep = {}          # ticket -> output array kept alive until the request is released

    def close(self):
        if self.handle:
            load().dm_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, indices, weights, k: int, seed: int, out=None):
        """Returns (status, ticket, out): status 0 or EAGAIN (ticket None then); raises on other
        errors.  out: numpy uint64[k] receiving the keys (allocated when None)."""
        import numpy as np
        if out is None:
            out = np.empty(k, dtype=np.uint64)
        t = ctypes.c_int64()
        nnz = len(indices)
        rc = load().dm_server_submit(self.handle, _host_ptr(indices, np.uint32, "indices"),
                                     _host_ptr(weights, np.float32, "weights"), nnz, int(k),
                                     int(seed) & (2**64 - 1), _host_ptr(out, np.uint64, "out"), ctypes.byref(t))
        if rc == EAGAIN:
            return rc, None, out
        _check(rc, "dm_server_submit")
        self._keep[t.value] = out
        return 0, t.value, out

    def poll(self, ticket: int):
        """None while pending, else the request's status (and the ticket is released)."""
        st = ctypes.c_int32()
        _check(load().dm_server_poll(self.handle, int(ticket), ctypes.byref(st)), "dm_server_poll")
        if st.value == -1:
            return None
        self._keep.pop(ticket, None)
        return st.value

    def wait(self, ticket: int, timeout_us: int = -1):
        """The request's status; None if the timeout passed first."""
        st = ctypes.c_int32()
        rc = load().dm_server_wait(self.handle, int(ticket), int(timeout_us), ctypes.byref(st))
        if rc == ETIMEOUT:
            return None
        _check(rc, "dm_server_wait")
        self._keep.pop(ticket, None)
        return st.value

    def replay(self, indptr, indices, weights, ks, seeds, arrival_ns, deliver: bool = True):
        """Plays a trace in real time; returns (keys or None, latency_ns, status)."""
        import numpy as np
        n = len(indptr) - 1
        ks = np.ascontiguousarray(ks, dtype=np.int32)
        seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        arrival_ns = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        out = np.empty(int(ks.astype(np.int64).sum()), dtype=np.uint64) if deliver else None
        lat = np.empty(n, dtype=np.int64)
        st = np.empty(n, dtype=np.int32)
        _check(load().dm_server_replay(self.handle, n, _host_ptr(indptr, np.int64, "indptr"),
                                       _host_ptr(indices, np.uint32, "indices"), _host_ptr(weights, np.float32, "weights"),
                                       _host_ptr(ks, np.int32, "k"), _host_ptr(seeds, np.uint64, "seed"),
                                       _host_ptr(arrival_ns, np.int64, "arrival_ns"),
                                       _host_ptr(out, np.uint64, "out") if deliver else None,
                                       _host_ptr(lat, np.int64, "latency"), _host_ptr(st, np.int32, "status")),
               "dm_server_replay")
        return out, lat, st

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().dm_server_get_stats(self.handle, ctypes.cast(ctypes.byref(s), ctypes.c_void_p)),
               "dm_server_get_stats")
        return {f: getattr(s, f) for f, _ in s._fields_}

    def reset_stats(self):
        _check(load().dm_server_reset_stats(self.handle), "dm_server_reset_stats")

    def fail_batches(self, n: int):
        _check(load().dm_server_fail_batches(self.handle, int(n)), "dm_server_fail_batches")
