"""Thin Python binding of libsoar.so (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: it checks shapes and dtypes of torch CUDA tensors,
passes their device pointers and the current CUDA stream, and raises
``SoarError`` on a non-zero status.  There is no CPU fallback: if the shared
library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsoar.so")

SOAR_OK, SOAR_EINVAL, SOAR_ENOMEM, SOAR_ECUDA, SOAR_ETIMEOUT, SOAR_EUNSUPPORTED = range(6)
SOAR_F32, SOAR_BF16 = 0, 1
SOAR_SCORE_F32, SOAR_SCORE_FP8, SOAR_SCORE_PQ4 = 0, 2, 3
STATUS_NAMES = {0: "SOAR_OK", 1: "SOAR_EINVAL", 2: "SOAR_ENOMEM", 3: "SOAR_ECUDA",
                4: "SOAR_ETIMEOUT", 5: "SOAR_EUNSUPPORTED"}

_lib = None


class SoarError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ServerConfig(ct.Structure):
    _fields_ = [("max_batch", ct.c_int32), ("streams", ct.c_int32), ("memory_budget", ct.c_int64),
                ("max_k", ct.c_int32)]


class ServerStats(ct.Structure):
    _fields_ = [("batches", ct.c_uint64), ("completed", ct.c_uint64), ("queries_in_batches", ct.c_uint64),
                ("pending", ct.c_uint64), ("max_in_flight", ct.c_int32), ("p50_ms", ct.c_double),
                ("p99_ms", ct.c_double)]


class IndexInfo(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("d", ct.c_int32), ("c", ct.c_int32), ("spills", ct.c_int32),
                ("mode", ct.c_int32), ("dtype", ct.c_int32), ("row_stride", ct.c_int32),
                ("rows", ct.c_int64), ("max_partition", ct.c_int64), ("offsets", ct.c_void_p),
                ("ids", ct.c_void_p), ("vectors", ct.c_void_p), ("row_scales", ct.c_void_p),
                ("originals", ct.c_void_p), ("centroids", ct.c_void_p), ("device_bytes", ct.c_int64)]


_P, _I32, _I64, _F32 = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_float
_SIGS = {
    "soar_last_error": ([], ct.c_char_p),
    "soar_version": ([], ct.c_char_p),
    "soar_train_centroids": ([_P, _I32, _I64, _I32, _I32, _I32, _P, _P, _P], _I32),
    "soar_assign": ([_P, _I32, _I64, _I32, _P, _I32, _F32, _I32, _P, _P], _I32),
    "soar_index_build": ([_P, _I32, _I64, _I32, _P, _I32, _P, _I32, _I32, ct.POINTER(_P), _P], _I32),
    "soar_index_get_info": ([_P, ct.POINTER(IndexInfo)], _I32),
    "soar_index_free": ([_P], _I32),
    "soar_index_save": ([_P, ct.c_char_p, _P], _I32),
    "soar_index_load": ([ct.c_char_p, ct.POINTER(_P), _P], _I32),
    "soar_select_partitions": ([_P, _P, _I32, _I64, _I32, _P, _P, _P], _I32),
    "soar_search": ([_P, _P, _I32, _I64, _I32, _I32, _P, _I32, _P, _P, _P], _I32),
    "soar_exact_mips": ([_P, _I32, _I64, _I32, _P, _I32, _I64, _I32, _P, _P, _P], _I32),
    "soar_quantize_fp8": ([_P, _I32, _I64, _I32, _P, _I32, _P, _P], _I32),
    "soar_merge_topk": ([_P, _P, _I64, _I32, _I32, _P, _I32, _P, _P, _P], _I32),
    "soar_select_partitions_static": ([_P, _P, _I32, _I64, _I32, _P, _P, _P], _I32),
    "soar_index_build_coarse": ([_P, _I32, _I32, _P, _F32, _I32, ct.POINTER(_P), _P], _I32),
    "soar_pq_train": ([_P, _I32, _I64, _I32, _P, _I32, _P, _I32, _P, _P, _P], _I32),
    "soar_index_build_pq": ([_P, _I32, _I64, _I32, _P, _I32, _P, _I32, _P, ct.POINTER(_P), _P], _I32),
    "soar_select_partitions_multilevel": ([_P, _P, _I32, _I64, _I32, _I32, _P, _P, _P, _P], _I32),
    "soar_search_multilevel": ([_P, _P, _P, _I32, _I64, _I32, _I32, _I32, _I32, _P, _P, _P], _I32),
    "soar_check_device": ([], _I32),
    "soar_server_create": ([_P, ct.POINTER(ServerConfig), ct.POINTER(_P)], _I32),
    "soar_server_submit": ([_P, _P, _I32, _I32, ct.POINTER(ct.c_uint64)], _I32),
    "soar_server_wait": ([_P, ct.c_uint64, _P, _P, ct.POINTER(ct.c_double), _I32], _I32),
    "soar_server_submit_many": ([_P, _P, _I64, _P, _P, _P, _P], _I32),
    "soar_server_wait_many": ([_P, _P, _I64, _I32, _P, _P, _P, _I32], _I32),
    "soar_server_stats": ([_P, ct.POINTER(ServerStats)], _I32),
    "soar_server_destroy": ([_P], _I32),
    "soar_mlp_param_count": ([_I32, _I32], _I64),
    "soar_probe_features": ([_P, _P, _I32, _I64, _I32, _P, _P], _I32),
    "soar_probe_labels": ([_P, _P, _I32, _I64, _P, _I32, _F32, _P, _P], _I32),
    "soar_mlp_forward": ([_P, _I32, _I32, _P, _I32, _I32, _P, _P], _I32),
    "soar_mlp_backward": ([_P, _I32, _I32, _P, _P, _I32, _I32, _P, _P, _P], _I32),
    "soar_mlp_adam": ([_P, _P, _P, _P, _I64, _I32, _F32, _F32, _F32, _F32, _P], _I32),
    "soar_mlp_predict_probes": ([_P, _I32, _I32, _P, _I32, _I32, _F32, _I32, _P, _P], _I32),
    "soar_search_learned": ([_P, _P, _I32, _I64, _I32, _I32, _P, _I32, _I32, _F32, _I32, _I32, _P, _P, _P, _P],
                            _I32),
    "soar_kernel_launches": ([], ct.c_uint64),
    "soar_set_wait_limit": ([_I64], _I32),
    "soar_stage_timing": ([_I32], _I32),
    "soar_stage_times": ([ct.c_char_p, _I32, _P, _P, _I32], _I32),
}


def load():
    """Loads libsoar.so (built by ``paper_2404_00774_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2404_00774_gb300.build`"
                           " (there is no CPU fallback)")
    lib = ct.CDLL(LIB_PATH)
    for name, (args, res) in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status: int):
    if status != SOAR_OK:
        raise SoarError(status, load().soar_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ct.c_void_p(stream.cuda_stream)


def _dtype(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return SOAR_F32
    if t.dtype == torch.bfloat16:
        return SOAR_BF16
    raise TypeError(f"vectors must be float32 or bfloat16, got {t.dtype}")


def _dev(t: torch.Tensor, name: str, dtype=None, ndim=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimensions")
    return ct.c_void_p(t.data_ptr())


def version() -> str:
    return load().soar_version().decode()


def soar_train_centroids(X: torch.Tensor, c: int, iters: int, init_idx: torch.Tensor, out=None, stream=None):
    n, d = X.shape
    if out is None:
        out = torch.empty((c, d), dtype=torch.float32, device=X.device)
    _check(load().soar_train_centroids(_dev(X, "X", ndim=2), _dtype(X), n, d, c, iters,
                                       _dev(init_idx, "init_idx", torch.int32, 1),
                                       _dev(out, "out", torch.float32, 2), _stream(stream)))
    return out


def soar_assign(X: torch.Tensor, C: torch.Tensor, lam: float, spills: int, out=None, stream=None):
    n, d = X.shape
    c = C.shape[0]
    if C.shape[1] != d:
        raise ValueError("C and X disagree on d")
    if out is None:
        out = torch.empty((n, 1 + spills), dtype=torch.int32, device=X.device)
    _check(load().soar_assign(_dev(X, "X", ndim=2), _dtype(X), n, d, _dev(C, "C", torch.float32, 2), c,
                              float(lam), spills, _dev(out, "out", torch.int32, 2), _stream(stream)))
    return out


class Index:
    """Owner of a soar_index handle (freed on ``close`` or garbage collection)."""

    def __init__(self, handle: ct.c_void_p):
        self._h = handle
        self.info = IndexInfo()
        _check(load().soar_index_get_info(self._h, ct.byref(self.info)))

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("index is closed")
        return self._h

    def close(self):
        if self._h is not None:
            _check(load().soar_index_free(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # device arrays owned by the index, as torch views
    def _view(self, ptr, count, dtype):
        if count == 0:
            return torch.empty(0, dtype=dtype, device="cuda")
        return _wrap_device(ptr, count, dtype)

    def offsets(self) -> torch.Tensor:
        return self._view(self.info.offsets, self.info.c + 1, torch.int64).clone()

    def ids(self) -> torch.Tensor:
        return self._view(self.info.ids, self.info.rows, torch.int32).clone()

    def vectors(self) -> torch.Tensor:
        i = self.info
        if i.mode in (SOAR_SCORE_FP8, SOAR_SCORE_PQ4):      # byte codes, row_stride bytes per copy
            return self._view(i.vectors, i.rows * i.row_stride, torch.uint8).clone().view(i.rows, i.row_stride)
        dt = torch.float32 if i.dtype == SOAR_F32 else torch.bfloat16
        return self._view(i.vectors, i.rows * i.row_stride, dt).clone().view(i.rows, i.row_stride)

    def row_scales(self) -> torch.Tensor:
        return self._view(self.info.row_scales, self.info.rows, torch.float32).clone()

    def centroids(self) -> torch.Tensor:
        i = self.info
        return self._view(i.centroids, i.c * i.d, torch.float32).clone().view(i.c, i.d)


class _DeviceArray:
    """Minimal __cuda_array_interface__ provider for memory the library owns."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


_TYPESTR = {torch.float32: "<f4", torch.int32: "<i4", torch.int64: "<i8", torch.uint8: "|u1",
            torch.bfloat16: "<i2"}


def _wrap_device(ptr: int, count: int, dtype: torch.dtype) -> torch.Tensor:
    """A torch tensor aliasing `count` elements of device memory at `ptr`."""
    t = torch.as_tensor(_DeviceArray(ptr, count, _TYPESTR[dtype]), device="cuda")
    return t.view(torch.bfloat16) if dtype == torch.bfloat16 else t


def soar_index_build(X: torch.Tensor, C: torch.Tensor, assign: torch.Tensor, mode: int = SOAR_SCORE_F32,
                     stream=None) -> Index:
    n, d = X.shape
    c = C.shape[0]
    spills = assign.shape[1] - 1
    if assign.shape[0] != n:
        raise ValueError("assign must have one row per datapoint")
    h = ct.c_void_p()
    _check(load().soar_index_build(_dev(X, "X", ndim=2), _dtype(X), n, d, _dev(C, "C", torch.float32, 2), c,
                                   _dev(assign, "assign", torch.int32, 2), spills, mode, ct.byref(h),
                                   _stream(stream)))
    return Index(h)


def soar_pq_train(X: torch.Tensor, C: torch.Tensor, part: torch.Tensor, iters: int, init_idx: torch.Tensor,
                  stream=None) -> torch.Tensor:
    """PQ codebooks [d/2, 16, 2] of the residuals X[i] - C[part[i]]."""
    n, d = X.shape
    B = torch.empty((d // 2, 16, 2), dtype=torch.float32, device=X.device)
    _check(load().soar_pq_train(_dev(X, "X", ndim=2), _dtype(X), n, d, _dev(C, "C", torch.float32, 2), C.shape[0],
                                _dev(part, "part", torch.int32, 1), iters, _dev(init_idx, "init_idx", torch.int32, 1),
                                _dev(B, "B"), _stream(stream)))
    return B


def soar_index_build_pq(X: torch.Tensor, C: torch.Tensor, assign: torch.Tensor, B: torch.Tensor,
                        stream=None) -> Index:
    n, d = X.shape
    if assign.shape[0] != n:
        raise ValueError("assign must have one row per datapoint")
    h = ct.c_void_p()
    _check(load().soar_index_build_pq(_dev(X, "X", ndim=2), _dtype(X), n, d, _dev(C, "C", torch.float32, 2),
                                      C.shape[0], _dev(assign, "assign", torch.int32, 2), assign.shape[1] - 1,
                                      _dev(B, "B", torch.float32, 3), ct.byref(h), _stream(stream)))
    return Index(h)


def soar_index_save(index: Index, path: str, stream=None) -> None:
    _check(load().soar_index_save(index.handle, os.fsencode(path), _stream(stream)))


def soar_index_load(path: str, stream=None) -> Index:
    h = ct.c_void_p()
    _check(load().soar_index_load(os.fsencode(path), ct.byref(h), _stream(stream)))
    return Index(h)


def soar_select_partitions(index: Index, Q: torch.Tensor, t: int, with_scores: bool = False, stream=None):
    nq = Q.shape[0]
    top = torch.empty((nq, t), dtype=torch.int32, device=Q.device)
    sc = torch.empty((nq, t), dtype=torch.float32, device=Q.device) if with_scores else None
    _check(load().soar_select_partitions(index.handle, _dev(Q, "Q", ndim=2), _dtype(Q), nq, t,
                                         _dev(top, "top"), _dev(sc, "scores") if sc is not None else None,
                                         _stream(stream)))
    return (top, sc) if with_scores else top


def soar_select_partitions_static(index: Index, Q: torch.Tensor, t: int, top_out: torch.Tensor,
                                  scores_out: torch.Tensor | None = None, stream=None):
    """soar_select_partitions into caller-provided outputs, with no device allocation
    inside the call (scratch is the library's fixed static buffer; see include/soar.h)."""
    nq = Q.shape[0]
    if tuple(top_out.shape) != (nq, t):
        raise ValueError("top_out must be [nq, t]")
    if scores_out is not None and tuple(scores_out.shape) != (nq, t):
        raise ValueError("scores_out must be [nq, t]")
    _check(load().soar_select_partitions_static(index.handle, _dev(Q, "Q", ndim=2), _dtype(Q), nq, t,
                                                _dev(top_out, "top_out", torch.int32, 2),
                                                _dev(scores_out, "scores_out", torch.float32, 2)
                                                if scores_out is not None else None, _stream(stream)))
    return top_out, scores_out


def soar_search(index: Index, Q: torch.Tensor, k: int, t: int, t_per_query=None, rescore: int = 0,
                ids_out=None, scores_out=None, stream=None):
    nq = Q.shape[0]
    if ids_out is None:
        ids_out = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
    if scores_out is None:
        scores_out = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
    tpq = _dev(t_per_query, "t_per_query", torch.int32, 1) if t_per_query is not None else None
    _check(load().soar_search(index.handle, _dev(Q, "Q", ndim=2), _dtype(Q), nq, k, t, tpq, rescore,
                              _dev(ids_out, "ids_out", torch.int64, 2),
                              _dev(scores_out, "scores_out", torch.float32, 2), _stream(stream)))
    return ids_out, scores_out


def soar_index_build_coarse(index: Index, c2: int, iters: int, init_idx: torch.Tensor, lam: float = 1.0,
                            spills: int = 1, stream=None) -> Index:
    """The coarse index of `index`: its fine centroids quantized into c2 partitions."""
    h = ct.c_void_p()
    _check(load().soar_index_build_coarse(index.handle, c2, iters, _dev(init_idx, "init_idx", torch.int32, 1),
                                          lam, spills, ct.byref(h), _stream(stream)))
    return Index(h)


def soar_select_partitions_multilevel(coarse: Index, Q: torch.Tensor, t: int, t1: int, stream=None):
    """(top [nq, t] int32, scores [nq, t], count [nq] int32) of the two-level selection."""
    nq = Q.shape[0]
    top = torch.empty((nq, t), dtype=torch.int32, device=Q.device)
    sc = torch.empty((nq, t), dtype=torch.float32, device=Q.device)
    cnt = torch.empty((nq,), dtype=torch.int32, device=Q.device)
    _check(load().soar_select_partitions_multilevel(coarse.handle, _dev(Q, "Q", ndim=2), _dtype(Q), nq, t, t1,
                                                    _dev(top, "top"), _dev(sc, "scores"), _dev(cnt, "count"),
                                                    _stream(stream)))
    return top, sc, cnt


def soar_search_multilevel(index: Index, coarse: Index, Q: torch.Tensor, k: int, t: int, t1: int,
                           rescore: int = 0, ids_out=None, scores_out=None, stream=None):
    nq = Q.shape[0]
    if ids_out is None:
        ids_out = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
    if scores_out is None:
        scores_out = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
    _check(load().soar_search_multilevel(index.handle, coarse.handle, _dev(Q, "Q", ndim=2), _dtype(Q), nq, k, t,
                                         t1, rescore, _dev(ids_out, "ids_out", torch.int64, 2),
                                         _dev(scores_out, "scores_out", torch.float32, 2), _stream(stream)))
    return ids_out, scores_out


def soar_exact_mips(X: torch.Tensor, Q: torch.Tensor, k: int, stream=None):
    n, d = X.shape
    nq = Q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
    sc = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
    _check(load().soar_exact_mips(_dev(X, "X", ndim=2), _dtype(X), n, d, _dev(Q, "Q", ndim=2), _dtype(Q), nq, k,
                                  _dev(ids, "ids"), _dev(sc, "scores"), _stream(stream)))
    return ids, sc


def soar_merge_topk(ids: torch.Tensor, scores: torch.Tensor, k: int, id_offsets: torch.Tensor | None = None,
                    stream=None):
    """ids / scores [nq][m][len] (m lists per query, best first) -> the merged top k [nq][k]."""
    nq, m, ln = ids.shape
    if tuple(scores.shape) != (nq, m, ln):
        raise ValueError("ids and scores must have the same shape")
    if id_offsets is not None and tuple(id_offsets.shape) != (m,):
        raise ValueError("id_offsets must have one entry per list")
    out_i = torch.empty((nq, k), dtype=torch.int64, device=ids.device)
    out_s = torch.empty((nq, k), dtype=torch.float32, device=ids.device)
    _check(load().soar_merge_topk(_dev(ids, "ids", torch.int64, 3), _dev(scores, "scores", torch.float32, 3), nq, m,
                                  ln, _dev(id_offsets, "id_offsets", torch.int64, 1) if id_offsets is not None
                                  else None, k, _dev(out_i, "ids_out"), _dev(out_s, "scores_out"), _stream(stream)))
    return out_i, out_s


def soar_quantize_fp8(V: torch.Tensor, code_stride: int | None = None, stream=None):
    m, d = V.shape
    cs = d if code_stride is None else code_stride
    codes = torch.empty((m, cs), dtype=torch.uint8, device=V.device)
    scales = torch.empty((m,), dtype=torch.float32, device=V.device)
    _check(load().soar_quantize_fp8(_dev(V, "V", ndim=2), _dtype(V), m, d, _dev(codes, "codes"), cs,
                                    _dev(scales, "scales"), _stream(stream)))
    return codes, scales


def soar_check_device() -> None:
    """Synchronises and raises SoarError if a kernel gave up a bounded wait."""
    _check(load().soar_check_device())


def soar_kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().soar_kernel_launches())


def soar_set_wait_limit(cycles: int) -> None:
    """Longest scan pipeline wait in SM cycles before a CTA gives up (0: default)."""
    _check(load().soar_set_wait_limit(int(cycles)))


def soar_stage_timing(enable: bool) -> None:
    _check(load().soar_stage_timing(1 if enable else 0))


def soar_stage_times() -> dict:
    """{stage: (total_ms, launches)} recorded since the last read (then cleared)."""
    names = ct.create_string_buffer(1024)
    ms = (ct.c_float * 32)()
    cnt = (ct.c_int32 * 32)()
    m = load().soar_stage_times(names, 1024, ct.cast(ms, ct.c_void_p), ct.cast(cnt, ct.c_void_p), 32)
    keys = names.value.decode().split(",") if m else []
    return {keys[i]: (float(ms[i]), int(cnt[i])) for i in range(m)}


# ---------------------------------------------------------------- learned probe count

def soar_mlp_param_count(d_in: int, hidden: int) -> int:
    return int(load().soar_mlp_param_count(d_in, hidden))


def soar_probe_features(index: Index, Q: torch.Tensor, top: int = 64, stream=None) -> torch.Tensor:
    nq, d = Q.shape
    Z = torch.empty((nq, d + top), dtype=torch.float32, device=Q.device)
    _check(load().soar_probe_features(index.handle, _dev(Q, "Q", ndim=2), _dtype(Q), nq, top, _dev(Z, "Z"),
                                      _stream(stream)))
    return Z


def soar_probe_labels(index: Index, Q: torch.Tensor, truth: torch.Tensor, target: float = 0.9,
                      stream=None) -> torch.Tensor:
    nq = Q.shape[0]
    k = truth.shape[1]
    out = torch.empty((nq,), dtype=torch.int32, device=Q.device)
    _check(load().soar_probe_labels(index.handle, _dev(Q, "Q", ndim=2), _dtype(Q), nq,
                                    _dev(truth, "truth", torch.int64, 2), k, float(target), _dev(out, "labels"),
                                    _stream(stream)))
    return out


def soar_mlp_forward(params: torch.Tensor, d_in: int, hidden: int, Z: torch.Tensor, bf16: bool = False,
                     stream=None) -> torch.Tensor:
    B = Z.shape[0]
    y = torch.empty((B,), dtype=torch.float32, device=Z.device)
    _check(load().soar_mlp_forward(_dev(params, "params", torch.float32, 1), d_in, hidden,
                                   _dev(Z, "Z", torch.float32, 2), B, int(bf16), _dev(y, "y"), _stream(stream)))
    return y


def soar_mlp_backward(params: torch.Tensor, d_in: int, hidden: int, Z: torch.Tensor, target: torch.Tensor,
                      bf16: bool = False, grads: torch.Tensor | None = None, loss: torch.Tensor | None = None,
                      stream=None):
    B = Z.shape[0]
    if grads is None:
        grads = torch.empty_like(params)
    if loss is None:
        loss = torch.empty((1,), dtype=torch.float32, device=Z.device)
    _check(load().soar_mlp_backward(_dev(params, "params", torch.float32, 1), d_in, hidden,
                                    _dev(Z, "Z", torch.float32, 2), _dev(target, "target", torch.float32, 1), B,
                                    int(bf16), _dev(grads, "grads", torch.float32, 1),
                                    _dev(loss, "loss", torch.float32, 1), _stream(stream)))
    return grads, loss


def soar_mlp_adam(params: torch.Tensor, grads: torch.Tensor, m1: torch.Tensor, m2: torch.Tensor, step: int,
                  lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None) -> None:
    _check(load().soar_mlp_adam(_dev(params, "params", torch.float32, 1), _dev(grads, "grads", torch.float32, 1),
                                _dev(m1, "m1", torch.float32, 1), _dev(m2, "m2", torch.float32, 1),
                                params.numel(), step, lr, beta1, beta2, eps, _stream(stream)))


def soar_search_learned(index: Index, Q: torch.Tensor, k: int, top: int, params: torch.Tensor, hidden: int,
                        alpha: float, t_cap: int, bf16: bool = True, rescore: int = 0, stream=None):
    """Search with the learned per-query probe count in one call; returns (ids, scores, counts)."""
    nq = Q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
    scores = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
    t = torch.empty((nq,), dtype=torch.int32, device=Q.device)
    _check(load().soar_search_learned(index.handle, _dev(Q, "Q", ndim=2), _dtype(Q), nq, k, top,
                                      _dev(params, "params", torch.float32, 1), hidden, int(bf16), float(alpha),
                                      t_cap, rescore, _dev(ids, "ids"), _dev(scores, "scores"), _dev(t, "t"),
                                      _stream(stream)))
    return ids, scores, t


def soar_mlp_predict_probes(params: torch.Tensor, d_in: int, hidden: int, Z: torch.Tensor, alpha: float, c: int,
                            bf16: bool = False, stream=None) -> torch.Tensor:
    B = Z.shape[0]
    t = torch.empty((B,), dtype=torch.int32, device=Z.device)
    _check(load().soar_mlp_predict_probes(_dev(params, "params", torch.float32, 1), d_in, hidden,
                                          _dev(Z, "Z", torch.float32, 2), B, int(bf16), float(alpha), c,
                                          _dev(t, "t"), _stream(stream)))
    return t


# ---------------------------------------------------------------- serving loop

class Server:
    """Continuous-batching server over an index (soar_server_* of the C ABI)."""

    def __init__(self, index: Index, max_batch: int = 256, streams: int = 2, memory_budget: int = 1 << 30,
                 max_k: int = 100):
        self.index = index                      # keeps the index alive
        self.max_k = max_k
        self.d = index.info.d
        cfg = ServerConfig(max_batch, streams, memory_budget, max_k)
        h = ct.c_void_p()
        st = load().soar_server_create(index.handle, ct.byref(cfg), ct.byref(h))
        if st != SOAR_OK:
            raise SoarError(st, "soar_server_create failed")
        self._h = h

    def submit(self, q: np.ndarray, k: int, t: int) -> int:
        q = np.ascontiguousarray(q, dtype=np.float32)
        if q.shape != (self.d,):
            raise ValueError(f"query must have shape ({self.d},)")
        rid = ct.c_uint64()
        st = load().soar_server_submit(self._h, q.ctypes.data_as(ct.c_void_p), k, t, ct.byref(rid))
        if st != SOAR_OK:
            raise SoarError(st, "soar_server_submit rejected the request")
        return int(rid.value)

    def submit_many(self, Q: np.ndarray, ks, ts, arrival_s=None) -> np.ndarray:
        """Queues len(Q) requests; arrival_s (seconds after the call, or None
        for now) replays an arrival trace.  Returns the request ids."""
        Q = np.ascontiguousarray(Q, dtype=np.float32)
        n = Q.shape[0]
        if Q.ndim != 2 or Q.shape[1] != self.d:
            raise ValueError(f"queries must have shape (n, {self.d})")
        ks = np.ascontiguousarray(np.broadcast_to(ks, (n,)), dtype=np.int32)
        ts = np.ascontiguousarray(np.broadcast_to(ts, (n,)), dtype=np.int32)
        arr = None if arrival_s is None else np.ascontiguousarray(arrival_s, dtype=np.float64)
        if arr is not None and arr.shape != (n,):
            raise ValueError("arrival_s must have one entry per query")
        rids = np.empty(n, dtype=np.uint64)
        st = load().soar_server_submit_many(self._h, Q.ctypes.data_as(ct.c_void_p), n,
                                            ks.ctypes.data_as(ct.c_void_p), ts.ctypes.data_as(ct.c_void_p),
                                            None if arr is None else arr.ctypes.data_as(ct.c_void_p),
                                            rids.ctypes.data_as(ct.c_void_p))
        if st != SOAR_OK:
            raise SoarError(st, "soar_server_submit_many rejected the requests")
        return rids

    def wait_many(self, rids: np.ndarray, kstride: int, timeout_ms: int = 600000):
        """(ids [n][kstride], scores [n][kstride], latency_ms [n]) of the requests, in order."""
        rids = np.ascontiguousarray(rids, dtype=np.uint64)
        n = rids.shape[0]
        ids = np.empty((n, kstride), dtype=np.int64)
        sc = np.empty((n, kstride), dtype=np.float32)
        lat = np.empty(n, dtype=np.float64)
        st = load().soar_server_wait_many(self._h, rids.ctypes.data_as(ct.c_void_p), n, kstride,
                                          ids.ctypes.data_as(ct.c_void_p), sc.ctypes.data_as(ct.c_void_p),
                                          lat.ctypes.data_as(ct.c_void_p), timeout_ms)
        if st != SOAR_OK:
            raise SoarError(st, "soar_server_wait_many failed")
        return ids, sc, lat

    def wait(self, rid: int, k: int, timeout_ms: int = 60000):
        ids = np.empty(k, dtype=np.int64)
        sc = np.empty(k, dtype=np.float32)
        lat = ct.c_double()
        st = load().soar_server_wait(self._h, rid, ids.ctypes.data_as(ct.c_void_p), sc.ctypes.data_as(ct.c_void_p),
                                     ct.byref(lat), timeout_ms)
        if st != SOAR_OK:
            raise SoarError(st, f"request {rid} failed")
        return ids, sc, float(lat.value)

    def stats(self) -> dict:
        out = ServerStats()
        _check(load().soar_server_stats(self._h, ct.byref(out)))
        return {name: getattr(out, name) for name, _ in ServerStats._fields_}

    def close(self):
        if self._h is not None:
            load().soar_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
