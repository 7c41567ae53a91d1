"""Thin Python binding of libphe (include/phe.h): argument marshalling only.

Function names match the C ABI.  Device buffers are passed as torch CUDA
tensors (or raw integer device pointers), host buffers as numpy arrays.
Every call raises PheError when the library returns a status other than
PHE_OK.  There is no fallback: if libphe.so is missing, loading fails.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libphe.so")            # production library
TEST_LIB_PATH = os.path.join(PKG, "libphe_test.so")  # plus the client-side calls (-DPHE_TESTING)
# Calls only the test library exports (they take or make a secret key).
TEST_ONLY = ("phe_client_encrypt", "phe_test_keygen")

PHE_OK, PHE_EINVAL, PHE_ENOMEM, PHE_EBUSY, PHE_ETIMEOUT, PHE_ECUDA, PHE_EUNSUPPORTED = range(7)
PHE_FWD, PHE_BWD = 0, 1
PHE_DIR_FWD_BIT, PHE_DIR_BWD_BIT = 1, 2
PHE_OUT_SWITCHED, PHE_OUT_RAW = 0, 1
PHE_PACK_DENSE = 2   # packing calls: several tokens per output RLWE


class PheError(RuntimeError):
    def __init__(self, status: int, name: str, message: str):
        super().__init__(f"{name}: {message}")
        self.status = status
        self.name = name


class phe_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("log2_qout", ctypes.c_uint32), ("q", ctypes.c_uint64),
                ("rns_p1", ctypes.c_uint32), ("rns_p2", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


PHE_CTX_FORCE_U64 = 1


class phe_trace_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double)]


class phe_job(ctypes.Structure):
    _fields_ = [("w", ctypes.c_void_p), ("dir", ctypes.c_int32), ("T", ctypes.c_uint32),
                ("d_in_mask", ctypes.c_void_p), ("d_in_body", ctypes.c_void_p),
                ("d_out_mask", ctypes.c_void_p), ("d_out_body", ctypes.c_void_p), ("d_in_seeds", ctypes.c_void_p)]


class phe_tuning(ctypes.Structure):
    _fields_ = [("tok_chunk", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32)]


class phe_plan_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint32), ("lwedot_launches", ctypes.c_uint32), ("tiles", ctypes.c_uint64),
                ("scratch_bytes", ctypes.c_uint64), ("modmuls", ctypes.c_uint64), ("tune", phe_tuning)]


class phe_server_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("chunk_tokens", ctypes.c_uint32),
                ("tok_chunk", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32), ("max_active", ctypes.c_uint32),
                ("max_jobs_per_iteration", ctypes.c_uint32), ("max_queue", ctypes.c_uint32),
                ("wait_timeout_ms", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("simulate", ctypes.c_uint32),
                ("sim_ns_per_item", ctypes.c_double)]


class phe_request(ctypes.Structure):
    _fields_ = [("w", ctypes.c_void_p), ("dir", ctypes.c_int32), ("T", ctypes.c_uint32),
                ("d_in_mask", ctypes.c_void_p), ("d_in_body", ctypes.c_void_p),
                ("h_out_mask", ctypes.c_void_p), ("h_out_body", ctypes.c_void_p), ("sim_rows", ctypes.c_uint32),
                ("d_in_seeds", ctypes.c_void_p)]


class phe_serving_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "failed", "tokens_completed", "iterations",
                                               "waiting", "active", "reserved_bytes", "peak_reserved_bytes")] + \
               [(n, ctypes.c_double) for n in ("p50_ms", "p99_ms", "max_ms", "mean_ms", "busy_ms")]


_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_i32 = ctypes.c_int
_sz = ctypes.c_size_t

# name -> (restype, argtypes); the C-ABI surface declared in include/phe.h.
SIGNATURES = {
    "phe_status_string": (ctypes.c_char_p, [_i32]),
    "phe_last_error": (ctypes.c_char_p, []),
    "phe_ctx_create": (_i32, [ctypes.POINTER(phe_params), _i32, ctypes.POINTER(_vp)]),
    "phe_ctx_destroy": (None, [_vp]),
    "phe_weights_upload": (_i32, [_vp, _vp, _u32, _u32, _u32, _vp, ctypes.POINTER(_vp)]),
    "phe_weights_free": (None, [_vp]),
    "phe_weights_shape": (_i32, [_vp, _i32, ctypes.POINTER(_u32), ctypes.POINTER(_u32), ctypes.POINTER(_u32)]),
    "phe_weights_device_bytes": (_u64, [_vp]),
    "phe_matmul": (_i32, [_vp, _vp, _i32, _u32, _vp, _vp, _vp, _vp, _u32, _vp]),
    "phe_modswitch": (_i32, [_vp, _vp, _vp, _sz, _vp]),
    "phe_client_encrypt": (_i32, [_vp, _u32, _u32, _vp, _vp, _vp, _vp, _u64, _vp, _vp]),
    "phe_test_keygen": (_i32, [_vp, _u64, _u32, _vp]),
    "phe_matmul_host": (_i32, [_vp, _vp, _i32, _u32, _vp, _vp, _vp, _vp, _u32, _u64, _vp]),
    "phe_trace_enable": (_i32, [_vp, _i32]),
    "phe_trace_read": (_i32, [_vp, ctypes.POINTER(phe_trace_entry), _u32, ctypes.POINTER(_u32)]),
    "phe_matmul_noalloc": (_i32, [_vp, _vp, _i32, _u32, _vp, _vp, _vp, _vp, _u32, _vp]),
    "phe_plan_create": (_i32, [_vp, ctypes.POINTER(phe_job), _u32, _u32, ctypes.POINTER(phe_tuning),
                               ctypes.POINTER(_vp)]),
    "phe_plan_run": (_i32, [_vp, _vp]),
    "phe_plan_graph": (_i32, [_vp, _vp]),
    "phe_plan_info": (_i32, [_vp, ctypes.POINTER(phe_plan_stats)]),
    "phe_plan_destroy": (None, [_vp]),
    "phe_autotune": (_i32, [_vp, ctypes.POINTER(phe_job), _u32, _u32, _u32, _vp, ctypes.POINTER(phe_tuning),
                            ctypes.POINTER(ctypes.c_double)]),
    "phe_server_create": (_i32, [_vp, ctypes.POINTER(phe_server_config), ctypes.POINTER(_vp)]),
    "phe_server_submit": (_i32, [_vp, ctypes.POINTER(phe_request), ctypes.POINTER(_u64)]),
    "phe_server_wait": (_i32, [_vp, _u64, _u32, ctypes.POINTER(ctypes.c_double)]),
    "phe_server_poll": (_i32, [_vp, _u64, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double)]),
    "phe_server_stats": (_i32, [_vp, ctypes.POINTER(phe_serving_stats)]),
    "phe_server_destroy": (None, [_vp]),
    "phe_matmul_seeded": (_i32, [_vp, _vp, _i32, _u32, _vp, _vp, _vp, _vp, _u32, _vp]),
    "phe_expand_masks": (_i32, [_vp, _vp, _u32, _vp, _vp]),
    "phe_ksk_upload": (_i32, [_vp, _vp, _vp, _u32, _u32, _u32, ctypes.POINTER(_vp)]),
    "phe_ksk_free": (None, [_vp]),
    "phe_ksk_device_bytes": (_u64, [_vp]),
    "phe_pack": (_i32, [_vp, _vp, _u32, _u32, _vp, _vp, _vp, _vp, _u32, _vp]),
    "phe_matmul_packed": (_i32, [_vp, _vp, _vp, _i32, _u32, _vp, _vp, _vp, _vp, _u32, _vp]),
    "phe_matmul_packed_seeded": (_i32, [_vp, _vp, _vp, _i32, _u32, _vp, _vp, _vp, _vp, _u32, _vp]),
    "phe_matmul_packed_host": (_i32, [_vp, _vp, _vp, _i32, _u32, _vp, _vp, _vp, _vp, _u32, _u32, _vp]),
    "phe_wire_sizes": (_i32, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "phe_pack_layout": (_i32, [_u32, _u32, _u32, _u32, ctypes.POINTER(_u64), ctypes.POINTER(_u32)]),
    "phe_wire_pack": (_i32, [_vp, _vp, _u32, _vp, _u32, _u64, _vp, _vp]),
    "phe_wire_unpack_inputs": (_i32, [_vp, _vp, _u64, _vp, _vp, _vp]),
    "phe_matmul_wire": (_i32, [_vp, _vp, _vp, _i32, _u32, _vp, _vp, _vp]),
    "phe_ctx_status": (_i32, [_vp, ctypes.POINTER(_u32), _i32]),
    "phe_ctx_set_body_path": (_i32, [_vp, _u32]),
    "phe_probe_alu": (_i32, [_i32, _i32, _u32, ctypes.POINTER(ctypes.c_double)]),
    "phe_probe_tensor": (_i32, [_i32, _u32, ctypes.POINTER(ctypes.c_double)]),
}

_lib = None
_lib_path = None
_want_test = os.environ.get("PHE_LIBRARY", "") == "test"
_lock = threading.Lock()


def use_test_library() -> None:
    """Load libphe_test.so instead of libphe.so (call before the first call
    into the library; one process uses one of the two: handles of one are
    not valid in the other).  Tests and the benchmark use it to make their
    encrypted inputs with phe_client_encrypt."""
    global _want_test
    with _lock:
        if _lib is not None and _lib_path != TEST_LIB_PATH:
            raise RuntimeError("libphe.so is already loaded in this process")
        _want_test = True


def lib() -> ctypes.CDLL:
    """Load the library (raises if it has not been built)."""
    global _lib, _lib_path
    with _lock:
        if _lib is None:
            path = TEST_LIB_PATH if _want_test else LIB_PATH
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with "
                                   "`python -m paper_2505_07329_b300.build` (or __graft_entry__.build())")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                if name in TEST_ONLY and path != TEST_LIB_PATH:
                    continue
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib, _lib_path = L, path
    return _lib


def _check(status: int) -> None:
    if status != PHE_OK:
        L = lib()
        raise PheError(status, L.phe_status_string(status).decode(), L.phe_last_error().decode())


def _dptr(x):
    """Device pointer of a torch CUDA tensor (must be contiguous), an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError(f"cannot take a device pointer of {type(x)}")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def phe_status_string(status: int) -> str:
    return lib().phe_status_string(status).decode()


def phe_last_error() -> str:
    return lib().phe_last_error().decode()


def phe_ctx_create(N: int, q: int, log2_qout: int, device: int = 0, rns=None, flags: int = 0):
    """rns: (p1, p2) when q = p1 * p2 is an RNS modulus of two 30-bit NTT primes."""
    p1, p2 = rns if rns else (0, 0)
    prm = phe_params(N, log2_qout, q, p1, p2, flags)
    out = _vp()
    _check(lib().phe_ctx_create(ctypes.byref(prm), device, ctypes.byref(out)))
    return out


def phe_ctx_destroy(ctx) -> None:
    lib().phe_ctx_destroy(ctx)


def phe_weights_upload(ctx, W, dirs: int = PHE_DIR_FWD_BIT | PHE_DIR_BWD_BIT, stream=None):
    """W: host int8 array [d_out, d_in] (numpy or CPU torch tensor)."""
    import numpy as np
    Wn = np.ascontiguousarray(W.numpy() if hasattr(W, "numpy") else np.asarray(W), dtype=np.int8)
    d_out, d_in = Wn.shape
    out = _vp()
    _check(lib().phe_weights_upload(ctx, Wn.ctypes.data, d_out, d_in, dirs, _stream(stream), ctypes.byref(out)))
    return out


def phe_weights_free(w) -> None:
    lib().phe_weights_free(w)


def phe_weights_shape(w, direction: int):
    r, c, L = _u32(), _u32(), _u32()
    _check(lib().phe_weights_shape(w, direction, ctypes.byref(r), ctypes.byref(c), ctypes.byref(L)))
    return r.value, c.value, L.value


def phe_weights_device_bytes(w) -> int:
    return int(lib().phe_weights_device_bytes(w))


def phe_matmul(ctx, w, direction: int, T: int, in_mask, in_body, out_mask, out_body,
               flags: int = PHE_OUT_SWITCHED, stream=None) -> None:
    _check(lib().phe_matmul(ctx, w, direction, T, _dptr(in_mask), _dptr(in_body), _dptr(out_mask),
                            _dptr(out_body), flags, _stream(stream)))


def phe_modswitch(ctx, d_in, d_out, n: int, stream=None) -> None:
    _check(lib().phe_modswitch(ctx, _dptr(d_in), _dptr(d_out), n, _stream(stream)))


PHE_KEY_BINARY, PHE_KEY_TERNARY = 0, 1


def phe_test_keygen(ctx, N: int, seed: int, kind: int = PHE_KEY_TERNARY):
    """Test library only: a seeded secret key for a context of ring degree N, int8 numpy array [N]."""
    import numpy as np
    out = np.zeros(N, dtype=np.int8)
    _check(lib().phe_test_keygen(ctx, seed, kind, out.ctypes.data))
    return out


def phe_client_encrypt(ctx, T: int, d: int, A, S, E, x, delta: int, B, stream=None) -> None:
    _check(lib().phe_client_encrypt(ctx, T, d, _dptr(A), _dptr(S), _dptr(E), _dptr(x), delta, _dptr(B),
                                    _stream(stream)))


def _hptr(a):
    """Host pointer of a numpy array or a CPU torch tensor (contiguous)."""
    if hasattr(a, "data_ptr"):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("expected a contiguous host tensor")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a contiguous host array")
    return a.ctypes.data


def phe_matmul_host(ctx, w, direction: int, T: int, h_in_mask, h_in_body, h_out_mask, h_out_body,
                    flags: int = PHE_OUT_SWITCHED, max_chunk_bytes: int = 0, stream=None) -> None:
    _check(lib().phe_matmul_host(ctx, w, direction, T, _hptr(h_in_mask), _hptr(h_in_body), _hptr(h_out_mask),
                                 _hptr(h_out_body), flags, max_chunk_bytes, _stream(stream)))


def phe_trace_enable(ctx, on: bool = True) -> None:
    _check(lib().phe_trace_enable(ctx, 1 if on else 0))


def phe_trace_read(ctx) -> dict:
    """{kernel name: {launches, total_ms, p50_ms, p99_ms, max_ms}}; clears the record."""
    cap = 16
    arr = (phe_trace_entry * cap)()
    n = _u32()
    _check(lib().phe_trace_read(ctx, arr, cap, ctypes.byref(n)))
    return {arr[i].name.decode(): {"launches": int(arr[i].launches), "total_ms": arr[i].total_ms,
                                   "p50_ms": arr[i].p50_ms, "p99_ms": arr[i].p99_ms, "max_ms": arr[i].max_ms}
            for i in range(n.value)}


def phe_ctx_status(ctx, clear: bool = True) -> int:
    """Status word of the context's bounded-wait kernels (0 = every wait completed)."""
    v = _u32()
    _check(lib().phe_ctx_status(ctx, ctypes.byref(v), 1 if clear else 0))
    return v.value


PHE_BODY_AUTO, PHE_BODY_TENSOR, PHE_BODY_FUSED = 0, 1, 2


def phe_ctx_set_body_path(ctx, path: int) -> None:
    """Where the bodies run: PHE_BODY_AUTO (by size), PHE_BODY_TENSOR, PHE_BODY_FUSED."""
    _check(lib().phe_ctx_set_body_path(ctx, path))


def phe_probe_alu(device: int = 0, form: int = 0, iters: int = 0) -> float:
    """Register-only butterflies per second (form 0: 32-bit residues; 1: 64-bit words)."""
    v = ctypes.c_double()
    _check(lib().phe_probe_alu(device, form, iters, ctypes.byref(v)))
    return v.value


def phe_probe_tensor(device: int = 0, iters: int = 0) -> float:
    """tcgen05.mma kind::f16 (bf16, fp32 accumulate) flop/s, M 128 N 256 K 16."""
    v = ctypes.c_double()
    _check(lib().phe_probe_tensor(device, iters, ctypes.byref(v)))
    return v.value


PHE_NOALLOC_MAX_SCRATCH_BYTES = 16 << 20


def phe_matmul_noalloc(ctx, w, direction: int, T: int, in_mask, in_body, out_mask, out_body,
                       flags: int = PHE_OUT_SWITCHED, stream=None) -> None:
    """phe_matmul with its scratch in the library's fixed device array (no allocation)."""
    _check(lib().phe_matmul_noalloc(ctx, w, direction, T, _dptr(in_mask), _dptr(in_body), _dptr(out_mask),
                                    _dptr(out_body), flags, _stream(stream)))


def _jobs(jobs):
    """jobs: list of (weights, direction, T, in_mask, in_body, out_mask, out_body[, in_seeds])."""
    arr = (phe_job * max(len(jobs), 1))()
    for i, job in enumerate(jobs):
        w, d, T, im, ib, om, ob = job[:7]
        seeds = job[7] if len(job) > 7 else None
        arr[i] = phe_job(w, d, T, _dptr(im), _dptr(ib), _dptr(om), _dptr(ob), _dptr(seeds))
    return arr


def phe_plan_create(ctx, jobs, flags: int = PHE_OUT_SWITCHED, tune=None):
    arr = _jobs(jobs)
    out = _vp()
    t = phe_tuning(*tune) if tune is not None else None
    _check(lib().phe_plan_create(ctx, arr, len(jobs), flags, ctypes.byref(t) if t is not None else None,
                                 ctypes.byref(out)))
    return out


def phe_plan_run(plan, stream=None) -> None:
    _check(lib().phe_plan_run(plan, _stream(stream)))


def phe_plan_graph(plan, stream=None) -> None:
    _check(lib().phe_plan_graph(plan, _stream(stream)))


def phe_plan_info(plan) -> dict:
    st = phe_plan_stats()
    _check(lib().phe_plan_info(plan, ctypes.byref(st)))
    return {"launches": st.launches, "lwedot_launches": st.lwedot_launches, "tiles": st.tiles,
            "scratch_bytes": st.scratch_bytes, "modmuls": st.modmuls,
            "tune": (st.tune.tok_chunk, st.tune.blocks_per_sm)}


def phe_plan_destroy(plan) -> None:
    lib().phe_plan_destroy(plan)


def phe_autotune(ctx, jobs, flags: int = PHE_OUT_SWITCHED, sample_tokens: int = 64, stream=None, timed=True):
    arr = _jobs(jobs)
    best = phe_tuning()
    ms = ctypes.c_double(0.0)
    _check(lib().phe_autotune(ctx, arr, len(jobs), flags, sample_tokens, _stream(stream), ctypes.byref(best),
                              ctypes.byref(ms) if timed else None))
    return (best.tok_chunk, best.blocks_per_sm), (ms.value if timed else None)


def phe_server_create(ctx, mem_budget_bytes: int, chunk_tokens: int = 32, tok_chunk: int = 8, blocks_per_sm: int = 0,
                      max_active: int = 64, max_jobs_per_iteration: int = 64, max_queue: int = 4096,
                      wait_timeout_ms: int = 60000, flags: int = PHE_OUT_SWITCHED, simulate: bool = False,
                      sim_ns_per_item: float = 0.0):
    cfg = phe_server_config(mem_budget_bytes, chunk_tokens, tok_chunk, blocks_per_sm, max_active,
                            max_jobs_per_iteration, max_queue, wait_timeout_ms, flags, 1 if simulate else 0,
                            sim_ns_per_item)
    out = _vp()
    _check(lib().phe_server_create(ctx, ctypes.byref(cfg), ctypes.byref(out)))
    return out


def phe_server_submit(srv, w, direction: int, T: int, in_mask=None, in_body=None, h_out_mask=None, h_out_body=None,
                      sim_rows: int = 0, in_seeds=None) -> int:
    req = phe_request(w, direction, T, _dptr(in_mask), _dptr(in_body),
                      _hptr(h_out_mask) if h_out_mask is not None else None,
                      _hptr(h_out_body) if h_out_body is not None else None, sim_rows, _dptr(in_seeds))
    rid = _u64()
    _check(lib().phe_server_submit(srv, ctypes.byref(req), ctypes.byref(rid)))
    return rid.value


def phe_server_wait(srv, rid: int, timeout_ms: int = 60000) -> float:
    lat = ctypes.c_double()
    _check(lib().phe_server_wait(srv, rid, timeout_ms, ctypes.byref(lat)))
    return lat.value


def phe_server_poll(srv, rid: int):
    done = _i32()
    lat = ctypes.c_double()
    _check(lib().phe_server_poll(srv, rid, ctypes.byref(done), ctypes.byref(lat)))
    return done.value, lat.value


def phe_server_stats(srv) -> dict:
    st = phe_serving_stats()
    _check(lib().phe_server_stats(srv, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in phe_serving_stats._fields_}


def phe_server_destroy(srv) -> None:
    lib().phe_server_destroy(srv)


def phe_matmul_seeded(ctx, w, direction: int, T: int, in_seeds, in_body, out_mask, out_body,
                      flags: int = PHE_OUT_SWITCHED, stream=None) -> None:
    """phe_matmul with per-ciphertext 64-bit seeds [T][L] in place of the masks."""
    _check(lib().phe_matmul_seeded(ctx, w, direction, T, _dptr(in_seeds), _dptr(in_body), _dptr(out_mask),
                                   _dptr(out_body), flags, _stream(stream)))


def phe_expand_masks(ctx, seeds, n: int, masks, stream=None) -> None:
    _check(lib().phe_expand_masks(ctx, _dptr(seeds), n, _dptr(masks), _stream(stream)))


def phe_ksk_upload(ctx, KA, KB, base_log: int, ell: int):
    """KA, KB: host uint64 arrays [n][ell][N] (the key-switching key, words mod q)."""
    import numpy as np
    KA = np.ascontiguousarray(np.asarray(KA, dtype=np.uint64))
    KB = np.ascontiguousarray(np.asarray(KB, dtype=np.uint64))
    if KA.shape != KB.shape or KA.ndim != 3 or KA.shape[1] != ell:
        raise ValueError(f"KA/KB must both be [n][{ell}][N], got {KA.shape} and {KB.shape}")
    out = _vp()
    _check(lib().phe_ksk_upload(ctx, KA.ctypes.data, KB.ctypes.data, KA.shape[0], base_log, ell,
                                ctypes.byref(out)))
    return out


def phe_ksk_free(k) -> None:
    lib().phe_ksk_free(k)


def phe_ksk_device_bytes(k) -> int:
    return int(lib().phe_ksk_device_bytes(k))


def phe_pack(ctx, k, T: int, rows: int, lwe_mask, lwe_body, out_a, out_b, flags: int = PHE_OUT_SWITCHED,
             stream=None) -> None:
    _check(lib().phe_pack(ctx, k, T, rows, _dptr(lwe_mask), _dptr(lwe_body), _dptr(out_a), _dptr(out_b), flags,
                          _stream(stream)))


def phe_matmul_packed(ctx, w, k, direction: int, T: int, in_mask, in_body, out_a, out_b,
                      flags: int = PHE_OUT_SWITCHED, stream=None) -> None:
    _check(lib().phe_matmul_packed(ctx, w, k, direction, T, _dptr(in_mask), _dptr(in_body), _dptr(out_a),
                                   _dptr(out_b), flags, _stream(stream)))


def phe_matmul_packed_host(ctx, w, k, direction: int, T: int, h_in_mask, h_in_body, h_out_a, h_out_b,
                           flags: int = PHE_OUT_SWITCHED, tok_chunk: int = 8, stream=None) -> None:
    _check(lib().phe_matmul_packed_host(ctx, w, k, direction, T, _hptr(h_in_mask), _hptr(h_in_body),
                                        _hptr(h_out_a), _hptr(h_out_b), flags, tok_chunk, _stream(stream)))


def phe_pack_layout(N: int, rows: int, T: int, flags: int = PHE_OUT_SWITCHED) -> tuple:
    """(output RLWEs, tokens per RLWE) of a packing call."""
    u, t = _u64(), _u32()
    _check(lib().phe_pack_layout(N, rows, T, flags, ctypes.byref(u), ctypes.byref(t)))
    return u.value, t.value


def phe_wire_sizes(ctx) -> dict:
    """Record sizes in bytes: {"input", "lwe", "rlwe"}."""
    a, b, c = _u64(), _u64(), _u64()
    _check(lib().phe_wire_sizes(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"input": a.value, "lwe": b.value, "rlwe": c.value}


def phe_wire_pack(ctx, a, fa: int, b, fb: int, n_records: int, out, stream=None) -> None:
    _check(lib().phe_wire_pack(ctx, _dptr(a), fa, _dptr(b), fb, n_records, _dptr(out), _stream(stream)))


def phe_wire_unpack_inputs(ctx, records, n_records: int, seeds, bodies, stream=None) -> None:
    _check(lib().phe_wire_unpack_inputs(ctx, _dptr(records), n_records, _dptr(seeds), _dptr(bodies),
                                        _stream(stream)))


def phe_matmul_wire(ctx, w, k, direction: int, T: int, in_records, out_records, stream=None) -> None:
    _check(lib().phe_matmul_wire(ctx, w, k, direction, T, _dptr(in_records), _dptr(out_records), _stream(stream)))


def phe_matmul_packed_seeded(ctx, w, k, direction: int, T: int, in_seeds, in_body, out_a, out_b,
                             flags: int = PHE_OUT_SWITCHED, stream=None) -> None:
    _check(lib().phe_matmul_packed_seeded(ctx, w, k, direction, T, _dptr(in_seeds), _dptr(in_body), _dptr(out_a),
                                          _dptr(out_b), flags, _stream(stream)))
