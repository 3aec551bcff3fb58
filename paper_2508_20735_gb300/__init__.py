"""Python binding of libdfa_gb300.so (the C ABI declared in include/dfa.h).

Argument marshalling only: every step of the refinement runs in the library's
CUDA kernels.  The functions named ``dfa_*`` mirror the C calls one to one;
:func:`minimise`, :func:`equivalent` and :func:`minimise_batch` are thin
conveniences that accept torch tensors or numpy arrays, allocate the workspace
with PyTorch's caching allocator and pass torch's current CUDA stream.

There is no CPU fallback: if the shared library is missing or cannot be loaded
the import of any entry point raises :class:`LibraryMissing`.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_size_t, c_uint32, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdfa_gb300.so")

DFA_OK, DFA_EINVAL, DFA_ENOMEM, DFA_ECUDA, DFA_ETIMEOUT, DFA_EMAXROUNDS, DFA_EBUSY, DFA_ECANCELLED = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "DFA_OK", -1: "DFA_EINVAL", -2: "DFA_ENOMEM", -3: "DFA_ECUDA", -4: "DFA_ETIMEOUT",
                -5: "DFA_EMAXROUNDS", -6: "DFA_EBUSY", -7: "DFA_ECANCELLED"}
ALGOS = {"moore": 0, "naive": 1, "trans": 2, "closure_moore": 3, "sort": 4}
DFA_FLAG_EARLY_EXIT = 0x1
DFA_FLAG_TABLE_ONLY = 0x2
DFA_FLAG_STOP_DISCRETE = 0x4
DFA_FLAG_BUCKETED = 0x8
DFA_FLAG_GATHER = 0x10
DFA_FLAG_ONE_BLOCK = 0x20
DFA_FLAG_CLUSTER = 0x40
DFA_REQ_MINIMISE, DFA_REQ_EQUIVALENT = 0, 1


class LibraryMissing(RuntimeError):
    pass


class DfaError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class DfaT(ctypes.Structure):
    _fields_ = [("n", c_uint32), ("k", c_uint32), ("delta", c_void_p), ("accept", c_void_p), ("start", c_uint32)]


class DfaOpts(ctypes.Structure):
    _fields_ = [("algo", c_int32), ("max_rounds", c_uint32), ("timeout_ns", c_uint64), ("schedule", c_int32),
                ("flags", c_uint32)]


class DfaResult(ctypes.Structure):
    _fields_ = [("num_blocks", c_uint32), ("rounds_changed", c_uint32), ("rounds_executed", c_uint32),
                ("status", c_int32), ("device_ns", c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None

# (name, restype, argtypes) of every C entry point
_SIGS = [
    ("dfa_workspace_size", c_size_t, [POINTER(DfaT), POINTER(DfaOpts)]),
    ("dfa_minimise", c_int, [POINTER(DfaT), POINTER(DfaOpts), c_void_p, POINTER(DfaResult), c_void_p, c_size_t, c_void_p]),
    ("dfa_batch_workspace_size", c_size_t, [POINTER(DfaT), c_uint32, POINTER(DfaOpts)]),
    ("dfa_minimise_batch", c_int, [POINTER(DfaT), c_uint32, POINTER(DfaOpts), c_void_p, POINTER(DfaResult), c_void_p,
                                   c_size_t, c_void_p]),
    ("dfa_batch_packed_workspace_size", c_size_t, [c_uint32, c_void_p, c_void_p, c_void_p, c_void_p,
                                                   POINTER(DfaOpts)]),
    ("dfa_minimise_batch_packed", c_int, [c_uint32, c_void_p, c_void_p, c_void_p, c_void_p, POINTER(DfaOpts),
                                          c_void_p, POINTER(DfaResult), c_void_p, c_size_t, c_void_p]),
    ("dfa_batch_graph_stats", c_int, [POINTER(c_uint64), POINTER(c_uint64)]),
    ("dfa_equivalent_workspace_size", c_size_t, [POINTER(DfaT), POINTER(DfaT), POINTER(DfaOpts)]),
    ("dfa_equivalent", c_int, [POINTER(DfaT), POINTER(DfaT), POINTER(DfaOpts), POINTER(c_int), POINTER(DfaResult),
                               c_void_p, c_size_t, c_void_p]),
    ("dfa_serve_create", c_int, [POINTER(c_void_p), c_size_t, c_uint32, c_int]),
    ("dfa_serve_submit", c_int, [c_void_p, c_int, POINTER(DfaT), POINTER(DfaT), POINTER(DfaOpts), POINTER(c_uint64)]),
    ("dfa_serve_poll", c_int, [c_void_p, c_uint64, POINTER(DfaResult), POINTER(c_int), c_void_p]),
    ("dfa_serve_wait", c_int, [c_void_p, c_uint64, c_uint64, POINTER(DfaResult), POINTER(c_int), c_void_p]),
    ("dfa_serve_stats", c_int, [c_void_p, POINTER(c_double), POINTER(c_double), POINTER(c_double)]),
    ("dfa_serve_counters", c_int, [c_void_p, POINTER(c_uint64), POINTER(c_uint64), POINTER(c_uint64),
                                   POINTER(c_uint64 * 3), POINTER(c_double)]),
    ("dfa_serve_destroy", c_int, [c_void_p]),
    ("dfa_minimise_noalloc", c_int, [POINTER(DfaT), POINTER(DfaOpts), c_void_p, POINTER(DfaResult), c_void_p]),
    ("dfa_product_workspace_size", c_size_t, [POINTER(DfaT), POINTER(DfaT), c_uint64]),
    ("dfa_product_check", c_int, [POINTER(DfaT), POINTER(DfaT), c_int, c_uint64, POINTER(c_int), POINTER(c_uint64),
                                  POINTER(ctypes.c_int64), c_void_p, c_size_t, c_void_p]),
    ("dfa_quotient_workspace_size", c_size_t, [POINTER(DfaT), c_void_p, c_void_p, c_void_p]),
    ("dfa_quotient", c_int, [POINTER(DfaT), c_void_p, c_void_p, c_void_p, POINTER(c_uint32), POINTER(c_uint32),
                             c_void_p, c_size_t, c_void_p]),
    ("dfa_minimise_async", c_int, [POINTER(DfaT), POINTER(DfaOpts), c_void_p, c_void_p, c_size_t, c_void_p]),
    ("dfa_minimise_result", c_int, [c_void_p, POINTER(DfaResult), c_void_p]),
    ("dfa_trans_workspace_size", c_size_t, [POINTER(DfaT), c_void_p]),
    ("dfa_trans", c_int, [POINTER(DfaT), c_void_p, POINTER(c_uint32), c_void_p, c_size_t, c_void_p]),
    ("dfa_last_error", ctypes.c_char_p, []),
    ("dfa_version", ctypes.c_char_p, []),
]


def lib():
    """The loaded shared library (raises LibraryMissing if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LibraryMissing(f"{LIB_PATH} not found; build it with __graft_entry__.build() "
                                 "or python paper_2508_20735_gb300/_build.py")
        try:
            L = ctypes.CDLL(LIB_PATH)
        except OSError as e:
            raise LibraryMissing(f"cannot load {LIB_PATH}: {e}") from e
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def last_error() -> str:
    return lib().dfa_last_error().decode()


def _check(status: int):
    if status not in (DFA_OK,):
        raise DfaError(status, last_error())


# ----------------------------------------------------------------- marshalling

def _ptr(x):
    """Address of a torch tensor or numpy array (kept alive by the caller)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"unsupported array type {type(x)}")


def _is_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


def _contig(x, np_dtype):
    """Contiguous 32-bit (np_dtype uint32) or 8-bit (uint8) view of x."""
    if hasattr(x, "data_ptr"):
        import torch
        if np_dtype == np.uint32:
            ok = (torch.int32, getattr(torch, "uint32", torch.int32))   # same bits
            if x.dtype not in ok:
                x = x.to(torch.int32)
        elif x.dtype != torch.uint8:
            x = x.to(torch.uint8)
        return x.contiguous()
    return np.ascontiguousarray(x, dtype=np_dtype)


def make_dfa(delta, accept, start: int = 0) -> tuple[DfaT, tuple]:
    """A dfa_t for arrays delta (k, n) of 32-bit targets and accept (n,) bytes;
    returns the struct and the arrays it points into (keep them alive)."""
    delta = _contig(delta, np.uint32)
    accept = _contig(accept, np.uint8)
    k, n = int(delta.shape[0]), int(delta.shape[1])
    if int(accept.shape[0]) != n:
        raise ValueError("delta must have shape (k, n) matching accept (n,)")
    d = DfaT(n, k, _ptr(delta) if k > 0 and n > 0 else None, _ptr(accept), int(start))
    return d, (delta, accept)


def make_opts(algo="moore", max_rounds=0, timeout_ns=0, schedule=-1, flags=0) -> DfaOpts:
    a = ALGOS[algo] if isinstance(algo, str) else int(algo)
    return DfaOpts(a, int(max_rounds), int(timeout_ns), int(schedule), int(flags))


def _stream(stream):
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    import torch
    return torch.cuda.current_stream().cuda_stream


def _workspace(nbytes: int, device=None):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


# ----------------------------------------------------------------- C entry points

def dfa_workspace_size(dfa: DfaT, opts: DfaOpts | None = None) -> int:
    return int(lib().dfa_workspace_size(ctypes.byref(dfa), ctypes.byref(opts) if opts else None))


def dfa_minimise(dfa: DfaT, opts: DfaOpts | None, block_out_ptr: int, workspace_ptr: int, ws_bytes: int,
                 stream: int | None) -> tuple[int, DfaResult]:
    res = DfaResult()
    st = lib().dfa_minimise(ctypes.byref(dfa), ctypes.byref(opts) if opts else None, block_out_ptr,
                            ctypes.byref(res), workspace_ptr, ws_bytes, stream)
    return st, res


def dfa_minimise_noalloc(dfa: DfaT, opts: DfaOpts | None, block_out_ptr: int,
                         stream: int | None) -> tuple[int, DfaResult]:
    """dfa_minimise without a caller workspace (fixed scratch inside the library;
    device pointers only, n <= 65,536; see include/dfa.h)."""
    res = DfaResult()
    st = lib().dfa_minimise_noalloc(ctypes.byref(dfa), ctypes.byref(opts) if opts else None, block_out_ptr,
                                    ctypes.byref(res), stream)
    return st, res


def batch_graph_stats() -> tuple[int, int]:
    """(instantiations, updates) of the batch calls' CUDA graph in this process."""
    i, u = c_uint64(0), c_uint64(0)
    lib().dfa_batch_graph_stats(ctypes.byref(i), ctypes.byref(u))
    return int(i.value), int(u.value)


def dfa_equivalent_workspace_size(a: DfaT, b: DfaT, opts: DfaOpts | None = None) -> int:
    return int(lib().dfa_equivalent_workspace_size(ctypes.byref(a), ctypes.byref(b),
                                                   ctypes.byref(opts) if opts else None))


def dfa_equivalent(a: DfaT, b: DfaT, opts: DfaOpts | None, workspace_ptr: int, ws_bytes: int,
                   stream: int | None) -> tuple[int, bool, DfaResult]:
    res = DfaResult()
    eq = c_int(-1)
    st = lib().dfa_equivalent(ctypes.byref(a), ctypes.byref(b), ctypes.byref(opts) if opts else None,
                              ctypes.byref(eq), ctypes.byref(res), workspace_ptr, ws_bytes, stream)
    return st, bool(eq.value == 1), res


def _dfa_array(dfas):
    return dfas if isinstance(dfas, ctypes.Array) else (DfaT * len(dfas))(*dfas)


def dfa_batch_workspace_size(dfas, opts: DfaOpts | None = None) -> int:
    arr = _dfa_array(dfas)
    return int(lib().dfa_batch_workspace_size(arr, len(arr), ctypes.byref(opts) if opts else None))


def dfa_minimise_batch(dfas, opts: DfaOpts | None, block_out_ptr: int, workspace_ptr: int, ws_bytes: int,
                       stream: int | None):
    arr = _dfa_array(dfas)
    res = (DfaResult * len(arr))()
    st = lib().dfa_minimise_batch(arr, len(arr), ctypes.byref(opts) if opts else None, block_out_ptr, res,
                                  workspace_ptr, ws_bytes, stream)
    return st, res   # the ctypes array: indexable and iterable, elements built on access


def dfa_batch_packed_workspace_size(count: int, n_ptr: int, k_ptr: int, delta_ptr, accept_ptr: int,
                                    opts: DfaOpts | None = None) -> int:
    return int(lib().dfa_batch_packed_workspace_size(count, n_ptr, k_ptr, delta_ptr, accept_ptr,
                                                     ctypes.byref(opts) if opts else None))


def dfa_minimise_batch_packed(count: int, n_ptr: int, k_ptr: int, delta_ptr, accept_ptr: int,
                              opts: DfaOpts | None, block_out_ptr: int, workspace_ptr: int, ws_bytes: int,
                              stream: int | None):
    res = (DfaResult * count)()
    st = lib().dfa_minimise_batch_packed(count, n_ptr, k_ptr, delta_ptr, accept_ptr,
                                         ctypes.byref(opts) if opts else None, block_out_ptr, res, workspace_ptr,
                                         ws_bytes, stream)
    return st, res   # the ctypes array: indexable and iterable, elements built on access


# ----------------------------------------------------------------- conveniences

def minimise(delta, accept, algo="moore", max_rounds=0, timeout_ns=0, out=None, workspace=None, stream=None,
             check=True, schedule=-1, flags=0):
    """Coarsest partition of the DFA given by delta (k, n) and accept (n,).

    Arrays may be CUDA tensors, CPU tensors or numpy arrays.  The output has the
    input's kind (CUDA tensor in -> CUDA tensor out; otherwise numpy).
    Returns (block, DfaResult)."""
    d, keep = make_dfa(delta, accept)
    o = make_opts(algo, max_rounds, timeout_ns, schedule, flags)
    on_dev = _is_cuda(keep[1])
    if out is None:
        if on_dev:
            import torch
            out = torch.empty(d.n, dtype=torch.int32, device=keep[1].device)
        else:
            out = np.empty(d.n, dtype=np.uint32)
    need = dfa_workspace_size(d, o)
    if need == 0:
        raise DfaError(DFA_EINVAL, last_error())
    if workspace is None:
        workspace = _workspace(need)
    st, res = dfa_minimise(d, o, _ptr(out), _ptr(workspace), int(workspace.numel()), _stream(stream))
    if check and st not in (DFA_OK,):
        raise DfaError(st, last_error())
    res.call_status = st
    return out, res


def equivalent(A, B, early_exit=False, timeout_ns=0, workspace=None, stream=None, check=True, flags=0, schedule=-1):
    """L(A) = L(B)?  A and B are (delta, accept, start) triples.  Returns (bool, DfaResult)."""
    a, ka = make_dfa(A[0], A[1], A[2])
    b, kb = make_dfa(B[0], B[1], B[2])
    o = make_opts("moore", 0, timeout_ns, schedule, flags=(DFA_FLAG_EARLY_EXIT if early_exit else 0) | int(flags))
    need = dfa_equivalent_workspace_size(a, b, o)
    if need == 0:
        raise DfaError(DFA_EINVAL, last_error() or "bad arguments")
    if workspace is None:
        workspace = _workspace(need)
    st, eq, res = dfa_equivalent(a, b, o, _ptr(workspace), int(workspace.numel()), _stream(stream))
    if check and st != DFA_OK:
        raise DfaError(st, last_error())
    res.call_status = st
    return eq, res


def minimise_batch(dfas, algo="moore", max_rounds=0, timeout_ns=0, schedule=-1, out=None, workspace=None,
                   stream=None, check=True, flags=0):
    """Refine a list of (delta, accept) pairs in one launch.  Returns (blocks, [DfaResult])."""
    structs, keep = [], []
    for item in dfas:
        d, kk = make_dfa(item[0], item[1])
        structs.append(d)
        keep.append(kk)
    structs = _dfa_array(structs)
    o = make_opts(algo, max_rounds, timeout_ns, schedule, flags)
    total = sum(s.n for s in structs)
    if out is None:
        import torch
        out = torch.empty(total, dtype=torch.int32, device="cuda")
    need = dfa_batch_workspace_size(structs, o)
    if need == 0:
        raise DfaError(DFA_EINVAL, last_error() or "bad arguments")
    if workspace is None:
        workspace = _workspace(need)
    st, res = dfa_minimise_batch(structs, o, _ptr(out), _ptr(workspace), int(workspace.numel()), _stream(stream))
    if check and st != DFA_OK:
        raise DfaError(st, last_error())
    return out, res


def pack_batch(dfas, device="cuda"):
    """The segment-offset form of a list of (delta (k, n), accept (n,)) pairs:
    (n, k, delta, accept) with n, k numpy uint32 arrays and delta, accept the
    concatenated arrays (each DFA's letter-major table in turn), as torch tensors
    on `device` (numpy arrays if device is None)."""
    ns = np.array([int(np.asarray(a).shape[0]) for _, a in dfas], dtype=np.uint32)
    ks = np.array([int(np.asarray(d).shape[0]) for d, _ in dfas], dtype=np.uint32)
    delta = np.concatenate([np.ascontiguousarray(d, dtype=np.uint32).reshape(-1) for d, _ in dfas])
    accept = np.concatenate([np.ascontiguousarray(a, dtype=np.uint8).reshape(-1) for _, a in dfas])
    if device is None:
        return ns, ks, delta, accept
    import torch
    return ns, ks, torch.from_numpy(delta.view(np.int32)).to(device), torch.from_numpy(accept).to(device)


def minimise_batch_packed(n, k, delta, accept, algo="moore", max_rounds=0, timeout_ns=0, schedule=-1, out=None,
                          workspace=None, stream=None, check=True, flags=0):
    """dfa_minimise_batch_packed over the segment-offset form (see pack_batch).
    Returns (blocks, [DfaResult])."""
    n = np.ascontiguousarray(n, dtype=np.uint32)
    k = np.ascontiguousarray(k, dtype=np.uint32)
    if n.shape != k.shape or n.ndim != 1:
        raise ValueError("n and k must be 1-D arrays of the same length")
    delta = _contig(delta, np.uint32)
    accept = _contig(accept, np.uint8)
    o = make_opts(algo, max_rounds, timeout_ns, schedule, flags)
    count = int(n.shape[0])
    dptr = _ptr(delta) if int(np.prod(delta.shape)) > 0 else None
    args = (count, n.ctypes.data, k.ctypes.data, dptr, _ptr(accept))
    if out is None:
        import torch
        out = torch.empty(int(n.sum(dtype=np.uint64)), dtype=torch.int32, device="cuda")
    need = dfa_batch_packed_workspace_size(*args, o)
    if need == 0:
        raise DfaError(DFA_EINVAL, last_error() or "bad arguments")
    if workspace is None:
        workspace = _workspace(need)
    st, res = dfa_minimise_batch_packed(*args, o, _ptr(out), _ptr(workspace), int(workspace.numel()),
                                        _stream(stream))
    if check and st != DFA_OK:
        raise DfaError(st, last_error())
    return out, res


DFA_CHECK_EQUIVALENCE = 0
DFA_CHECK_INCLUSION = 1


def product_check(A, B, inclusion=False, max_pairs=None, workspace=None, stream=None):
    """Equivalence (or inclusion L(A) ⊆ L(B)) by product exploration
    (dfa_product_check).  A and B are (delta, accept, start) triples.  Returns
    (holds, pairs explored, counterexample length or -1).  max_pairs bounds the
    explored pairs (default min(n_A n_B, 8 (n_A + n_B) + 65536)); a larger
    product raises DfaError(DFA_ENOMEM)."""
    a, ka = make_dfa(A[0], A[1], A[2])
    b, kb = make_dfa(B[0], B[1], B[2])
    if max_pairs is None:
        max_pairs = min(a.n * b.n, 8 * (a.n + b.n) + 65536)
    need = lib().dfa_product_workspace_size(ctypes.byref(a), ctypes.byref(b), int(max_pairs))
    if need == 0:
        raise DfaError(DFA_EINVAL, last_error() or "bad arguments")
    if workspace is None:
        workspace = _workspace(need)
    holds, pairs, cex = c_int(0), c_uint64(0), ctypes.c_int64(0)
    st = lib().dfa_product_check(ctypes.byref(a), ctypes.byref(b), DFA_CHECK_INCLUSION if inclusion else
                                 DFA_CHECK_EQUIVALENCE, int(max_pairs), ctypes.byref(holds), ctypes.byref(pairs),
                                 ctypes.byref(cex), _ptr(workspace), int(workspace.numel()), _stream(stream))
    if st != DFA_OK:
        raise DfaError(st, last_error())
    return bool(holds.value), int(pairs.value), int(cex.value)


def quotient(delta, accept, start, block, workspace=None, stream=None):
    """The minimal DFA from a partition (dfa_quotient).  Returns (delta', accept',
    start') as arrays of the inputs' kind (numpy in, numpy out; torch in, torch
    out), delta' of shape (k, n')."""
    d, keep = make_dfa(delta, accept, start)
    blk = _contig(block, np.uint32)
    torch_in = hasattr(keep[0], "data_ptr")
    n, k = d.n, d.k
    if torch_in:
        import torch
        dev = keep[1].device
        dout = torch.empty(max(k * n, 1), dtype=torch.int32, device=dev)
        aout = torch.empty(n, dtype=torch.uint8, device=dev)
    else:
        dout = np.empty(max(k * n, 1), dtype=np.uint32)
        aout = np.empty(n, dtype=np.uint8)
    need = lib().dfa_quotient_workspace_size(ctypes.byref(d), _ptr(blk), _ptr(dout), _ptr(aout))
    if need == 0:
        raise DfaError(DFA_EINVAL, last_error() or "bad arguments")
    if workspace is None:
        workspace = _workspace(need)
    nq, sq = c_uint32(0), c_uint32(0)
    st = lib().dfa_quotient(ctypes.byref(d), _ptr(blk), _ptr(dout), _ptr(aout), ctypes.byref(nq), ctypes.byref(sq),
                            _ptr(workspace), int(workspace.numel()), _stream(stream))
    if st != DFA_OK:
        raise DfaError(st, last_error())
    m = nq.value
    return dout[:k * m].reshape(k, m), aout[:m], sq.value


def minimise_async(d: DfaT, opts: DfaOpts | None, block_out_ptr: int, workspace_ptr: int, ws_bytes: int,
                   stream: int) -> int:
    """dfa_minimise_async on an already built dfa_t (see make_dfa): enqueue only."""
    return int(lib().dfa_minimise_async(ctypes.byref(d), ctypes.byref(opts) if opts else None, block_out_ptr,
                                        workspace_ptr, int(ws_bytes), stream))


def minimise_result(workspace_ptr: int, stream: int) -> tuple[int, DfaResult]:
    """dfa_minimise_result: wait for the stream; (status, DfaResult)."""
    res = DfaResult()
    st = lib().dfa_minimise_result(workspace_ptr, ctypes.byref(res), stream)
    return int(st), res


DFA_TRANS_MAX_STATES = 256


def trans(delta, accept, workspace=None, stream=None):
    """Algorithm 1 (dfa_trans): the partition by transitive closure of the pair
    graph, n <= DFA_TRANS_MAX_STATES.  Returns (block, iterations), block of the
    inputs' kind (numpy in, numpy out; torch in, torch out)."""
    d, keep = make_dfa(delta, accept, 0)
    if hasattr(keep[1], "data_ptr"):
        import torch
        out = torch.empty(d.n, dtype=torch.int32, device=keep[1].device)
    else:
        out = np.empty(d.n, dtype=np.uint32)
    need = lib().dfa_trans_workspace_size(ctypes.byref(d), _ptr(out))
    if need == 0:
        raise DfaError(DFA_EINVAL, last_error() or "bad arguments")
    if workspace is None:
        workspace = _workspace(need)
    it = c_uint32(0)
    st = lib().dfa_trans(ctypes.byref(d), _ptr(out), ctypes.byref(it), _ptr(workspace), int(workspace.numel()),
                         _stream(stream))
    if st != DFA_OK:
        raise DfaError(st, last_error())
    return out, it.value


def header_functions() -> list[str]:
    """Names of the functions include/dfa.h declares (used by the ABI tests)."""
    import re
    path = os.path.join(os.path.dirname(_HERE), "include", "dfa.h")
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dfa_[a-z_0-9]+)\s*\(", src)))


class Server:
    """Thin wrapper over dfa_serve_*: continuous batching of minimisation and
    equivalence requests on one device arena of `hbm_budget_bytes`."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 64, device: int = 0):
        h = c_void_p()
        st = lib().dfa_serve_create(ctypes.byref(h), int(hbm_budget_bytes), int(max_slots), int(device))
        if st != DFA_OK:
            raise DfaError(st, last_error())
        self._h = h

    def submit_minimise(self, delta, accept, max_rounds=0) -> int:
        d, keep = make_dfa(delta, accept)
        t = c_uint64()
        o = make_opts("moore", max_rounds)
        st = lib().dfa_serve_submit(self._h, DFA_REQ_MINIMISE, ctypes.byref(d), None, ctypes.byref(o),
                                    ctypes.byref(t))
        if st != DFA_OK:
            raise DfaError(st, last_error())
        return t.value

    def submit_equivalent(self, A, B, early_exit=False) -> int:
        a, ka = make_dfa(A[0], A[1], A[2])
        b, kb = make_dfa(B[0], B[1], B[2])
        t = c_uint64()
        o = make_opts("moore", flags=DFA_FLAG_EARLY_EXIT if early_exit else 0)
        st = lib().dfa_serve_submit(self._h, DFA_REQ_EQUIVALENT, ctypes.byref(a), ctypes.byref(b), ctypes.byref(o),
                                    ctypes.byref(t))
        if st != DFA_OK:
            raise DfaError(st, last_error())
        return t.value

    def poll(self, ticket: int, n: int = 0):
        """(status, DfaResult, equivalent, blocks-or-None); status DFA_EBUSY while running."""
        res = DfaResult()
        eq = c_int(-1)
        out = np.empty(n, dtype=np.uint32) if n else None
        st = lib().dfa_serve_poll(self._h, ticket, ctypes.byref(res), ctypes.byref(eq),
                                  out.ctypes.data if out is not None else None)
        return st, res, eq.value, out

    def wait(self, ticket: int, n: int = 0, timeout_ns: int = 0):
        res = DfaResult()
        eq = c_int(-1)
        out = np.empty(n, dtype=np.uint32) if n else None
        st = lib().dfa_serve_wait(self._h, ticket, int(timeout_ns), ctypes.byref(res), ctypes.byref(eq),
                                  out.ctypes.data if out is not None else None)
        return st, res, eq.value, out

    def stats(self):
        p50, p99, rps = c_double(), c_double(), c_double()
        st = lib().dfa_serve_stats(self._h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(rps))
        if st != DFA_OK:
            raise DfaError(st, last_error())
        return {"p50_us": p50.value, "p99_us": p99.value, "throughput_rps": rps.value}

    def counters(self):
        """Steps run, request-rounds and state-rounds advanced (also by round mode), host time in
        steps (dfa_serve_counters)."""
        st_, rr, sr, us = c_uint64(), c_uint64(), c_uint64(), c_double()
        modes = (c_uint64 * 3)()
        st = lib().dfa_serve_counters(self._h, ctypes.byref(st_), ctypes.byref(rr), ctypes.byref(sr),
                                      ctypes.byref(modes), ctypes.byref(us))
        if st != DFA_OK:
            raise DfaError(st, last_error())
        return {"steps": st_.value, "request_rounds": rr.value, "state_rounds": sr.value,
                "state_rounds_direct": modes[0], "state_rounds_filter": modes[1], "state_rounds_table": modes[2],
                "step_us": us.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().dfa_serve_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
