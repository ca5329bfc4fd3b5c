"""Thin ctypes binding of libkrp (include/krp.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Tensors are torch
tensors (device memory of the context's GPU) or, where the C ABI allows host
memory, CPU torch tensors / numpy arrays.  Element types map as
torch.float32 -> KRP_F32, torch.bfloat16 -> KRP_BF16, torch.float64 -> KRP_F64.
No computation happens here; a missing or unloadable library raises
immediately (there is no fallback path).
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkrp.so")

KRP_OK, KRP_EINVAL, KRP_ENOMEM, KRP_ECUDA, KRP_EUNSUPPORTED, KRP_ETIMEOUT, KRP_ENUMERIC = range(7)
KRP_F32, KRP_BF16, KRP_FP8_E4M3, KRP_F64, KRP_BF16X2 = 0, 1, 2, 3, 4
KRP_MEMO, KRP_TRUNCATE, KRP_RESIDUAL, KRP_TIMINGS = 0x1, 0x2, 0x4, 0x8
KRP_MAXD = 8
KRP_DRAW_MEMO, KRP_DRAW_FRESH_BASE, KRP_DRAW_STHOSVD_BASE = 0, 1, 64
KRP_TAG_OMEGA, KRP_TAG_PSI = 0, 1

EXPORTED = [
    "krp_create", "krp_destroy", "krp_set_stream", "krp_last_error", "krp_status_string",
    "krp_abi_version", "krp_launch_count", "krp_gen_factors", "krp_philox_words",
    "krp_sketch_mode", "krp_sketch_all_modes", "krp_qr", "krp_qr_noalloc", "krp_multi_ttm",
    "krp_tucker_rhosvd", "krp_tucker_sthosvd", "krp_block_hankel_lowrank",
    "krp_block_hankel_sketch", "krp_tucker_rhosvd_batched", "krp_tucker_batch_plan_info",
    "krp_block_hankel_batched", "krp_split_bf16x2", "krp_trace_begin", "krp_trace_end",
    "krp_core_truncate", "krp_residual", "krp_set_wait_limit", "krp_era_realize",
    "krp_block_hankel_nystrom", "krp_sensor_select", "krp_sensor_reconstruct",
    "krp_block_hankel2_lowrank", "krp_tucker_hadamard",
]


class KrpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


class PhaseTimes(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("rng_ms", "sketch_ms", "qr_ms", "core_ms", "truncate_ms", "residual_ms",
                 "total_ms")]


class TuckerOut(C.Structure):
    _fields_ = [
        ("core", C.c_void_p),
        ("factors", C.c_void_p * KRP_MAXD),
        ("d", C.c_int),
        ("core_dims", C.c_int64 * KRP_MAXD),
        ("rel_residual", C.c_double),
        ("x_norm", C.c_double),
        ("core_norm", C.c_double),
        ("times", PhaseTimes),
    ]


class TuckerItem(C.Structure):
    _fields_ = [
        ("X", C.c_void_p),
        ("dims", C.c_int64 * 3),
        ("ranks", C.c_int * 3),
        ("seed", C.c_uint64),
        ("core", C.c_void_p),
        ("factors", C.c_void_p * 3),
        ("rel_residual", C.c_double),
    ]


class HankelItem(C.Structure):
    _fields_ = [
        ("blocks", C.c_void_p),
        ("m", C.c_int), ("n", C.c_int), ("s", C.c_int), ("r", C.c_int),
        ("ell_r", C.c_int), ("ell_l", C.c_int),
        ("seed", C.c_uint64),
        ("U", C.c_void_p), ("S", C.c_void_p), ("V", C.c_void_p),
    ]


_lib = None


def load_library(path: Optional[str] = None):
    """Load libkrp.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"libkrp not built: {p} is missing (run __graft_entry__.build())")
    lib = C.CDLL(p)
    vp, i64p = C.c_void_p, C.POINTER(C.c_int64)
    sig = {
        "krp_create": (C.c_int, [C.POINTER(vp), C.c_int, vp]),
        "krp_destroy": (C.c_int, [vp]),
        "krp_set_stream": (C.c_int, [vp, vp]),
        "krp_set_wait_limit": (C.c_int, [vp, C.c_uint64]),
        "krp_era_realize": (C.c_int, [vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp,
                                      vp, vp, vp, vp, vp]),
        "krp_last_error": (C.c_char_p, [vp]),
        "krp_status_string": (C.c_char_p, [C.c_int]),
        "krp_abi_version": (C.c_int, []),
        "krp_launch_count": (C.c_uint64, [vp]),
        "krp_gen_factors": (C.c_int, [vp, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, i64p,
                                      C.c_int, C.c_int, C.POINTER(vp)]),
        "krp_philox_words": (C.c_int, [vp, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                       C.c_uint64, C.c_int64, vp]),
        "krp_sketch_mode": (C.c_int, [vp, vp, C.c_int, C.c_int, i64p, i64p, C.c_int,
                                      C.POINTER(vp), C.c_int, C.c_int, vp]),
        "krp_sketch_all_modes": (C.c_int, [vp, vp, C.c_int, C.c_int, i64p, i64p, C.POINTER(vp),
                                           C.c_int, C.c_int, C.POINTER(vp), C.c_int]),
        "krp_qr": (C.c_int, [vp, C.c_int, C.POINTER(vp), i64p, C.POINTER(C.c_int),
                             C.POINTER(vp), C.POINTER(vp)]),
        "krp_qr_noalloc": (C.c_int, [vp, C.c_int64, C.c_int, vp, vp, vp]),
        "krp_multi_ttm": (C.c_int, [vp, vp, C.c_int, C.c_int, i64p, i64p, C.POINTER(vp),
                                    C.POINTER(C.c_int), vp]),
        "krp_tucker_rhosvd": (C.c_int, [vp, vp, C.c_int, C.c_int, i64p, i64p,
                                        C.POINTER(C.c_int), C.c_int, C.c_uint64, C.c_uint,
                                        C.POINTER(TuckerOut)]),
        "krp_tucker_sthosvd": (C.c_int, [vp, vp, C.c_int, C.c_int, i64p, i64p,
                                         C.POINTER(C.c_int), C.c_int, C.c_uint64, C.c_uint,
                                         C.POINTER(TuckerOut)]),
        "krp_block_hankel_lowrank": (C.c_int, [vp, vp, C.c_int, C.c_int, C.c_int, C.c_int,
                                               C.c_int, C.c_int, C.c_int, C.c_uint64, vp, vp,
                                               vp]),
        "krp_tucker_hadamard": (C.c_int, [vp, C.c_int, i64p, C.POINTER(C.c_int), vp,
                                          C.POINTER(vp), C.POINTER(C.c_int), vp, C.POINTER(vp),
                                          C.c_int, C.c_uint64, vp, C.POINTER(vp),
                                          C.POINTER(C.c_double)]),
        "krp_sensor_select": (C.c_int, [vp, C.c_int, i64p, C.POINTER(C.c_int), C.POINTER(vp),
                                        C.POINTER(vp), C.POINTER(vp)]),
        "krp_sensor_reconstruct": (C.c_int, [vp, C.c_int, i64p, C.POINTER(C.c_int),
                                             C.POINTER(vp), vp, vp]),
        "krp_block_hankel_nystrom": (C.c_int, [vp, vp, C.c_int, C.c_int, C.c_int, C.c_int,
                                               C.c_int, C.c_double, C.c_uint64, vp, vp]),
        "krp_block_hankel2_lowrank": (C.c_int, [vp, vp, C.c_int, C.c_int, C.c_int, C.c_int,
                                                C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                                vp, vp, vp]),
        "krp_block_hankel_sketch": (C.c_int, [vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, vp,
                                              vp, C.c_int, vp, vp, C.c_int, vp, vp]),
        "krp_tucker_rhosvd_batched": (C.c_int, [vp, C.c_int, C.c_int, C.POINTER(TuckerItem),
                                                C.c_int, C.c_uint]),
        "krp_tucker_batch_plan_info": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                                 C.POINTER(C.c_int)]),
        "krp_block_hankel_batched": (C.c_int, [vp, C.c_int, C.c_int, C.POINTER(HankelItem)]),
        "krp_split_bf16x2": (C.c_int, [vp, vp, C.c_int64, vp]),
        "krp_trace_begin": (C.c_int, [vp]),
        "krp_trace_end": (C.c_int, [vp, C.c_char_p, C.c_size_t]),
        "krp_core_truncate": (C.c_int, [vp, C.c_int, i64p, C.POINTER(C.c_int),
                                        C.POINTER(C.c_int), vp, C.POINTER(vp), vp,
                                        C.POINTER(vp)]),
        "krp_residual": (C.c_int, [vp, vp, C.c_int, C.c_int, i64p, i64p, C.POINTER(C.c_int), vp,
                                   C.POINTER(vp), C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _status_name(s: int) -> str:
    names = ["KRP_OK", "KRP_EINVAL", "KRP_ENOMEM", "KRP_ECUDA", "KRP_EUNSUPPORTED",
             "KRP_ETIMEOUT", "KRP_ENUMERIC"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


# ---------------------------------------------------------------- marshalling --

class BF16x2:
    """A KRP_BF16X2 input: `tensor` holds 2N BF16 values (hi plane, lo plane)."""

    def __init__(self, tensor):
        self.tensor = tensor

    def is_contiguous(self):
        return self.tensor.is_contiguous()

    def data_ptr(self):
        return self.tensor.data_ptr()

    def element_size(self):
        return 4  # bytes per element of X (two BF16 planes)


def _dtype_code(t) -> int:
    import torch
    if isinstance(t, BF16x2):
        return KRP_BF16X2
    if isinstance(t, np.ndarray):
        m = {np.dtype(np.float32): KRP_F32, np.dtype(np.float64): KRP_F64}
        return m[t.dtype]
    m = {torch.float32: KRP_F32, torch.bfloat16: KRP_BF16, torch.float64: KRP_F64}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not (t.flags["C_CONTIGUOUS"] or t.flags["F_CONTIGUOUS"]):
            raise ValueError("array must be contiguous")
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _i64(vals) -> C.Array:
    return (C.c_int64 * len(vals))(*[int(v) for v in vals])


def _i32(vals) -> C.Array:
    return (C.c_int * len(vals))(*[int(v) for v in vals])


def _ptrs(ts) -> C.Array:
    return (C.c_void_p * len(ts))(*[_ptr(t) for t in ts])


def _current_stream(device: int) -> int:
    import torch
    return torch.cuda.current_stream(device).cuda_stream


class Context:
    """Owns a krp_ctx (workspace + stream binding) on one CUDA device."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        self.lib = load_library()
        self.device = device
        h = C.c_void_p()
        s = _current_stream(device) if stream is None else stream
        st = self.lib.krp_create(C.byref(h), device, C.c_void_p(s))
        if st != KRP_OK:
            raise KrpError(st, "krp_create failed")
        self.handle = h

    def check(self, st: int):
        if st != KRP_OK:
            raise KrpError(st, self.last_error())

    def last_error(self) -> str:
        return self.lib.krp_last_error(self.handle).decode()

    def set_stream(self, stream: int):
        self.check(self.lib.krp_set_stream(self.handle, C.c_void_p(stream)))

    def set_wait_limit(self, ns: int):
        """krp_set_wait_limit: limit of the tensor-core kernels' bounded waits (0 = 1 s)."""
        self.check(self.lib.krp_set_wait_limit(self.handle, C.c_uint64(ns)))

    def launch_count(self) -> int:
        return int(self.lib.krp_launch_count(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.krp_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- entry points --

def krp_abi_version() -> int:
    return int(load_library().krp_abi_version())


def krp_gen_factors(ctx: Context, seed: int, draw_id: int, tag: int, rows: Sequence[int],
                    ell: int, omega: Sequence):
    """Fill each non-None tensor omega[j] (rows[j] x ell, column-major) with N(0,1)."""
    t = next(o for o in omega if o is not None)
    ctx.check(ctx.lib.krp_gen_factors(ctx.handle, seed, draw_id, tag, len(rows), _i64(rows), ell,
                                      _dtype_code(t), _ptrs(omega)))


def krp_philox_words(ctx: Context, seed: int, c1: int, c2: int, c3: int, first_block: int,
                     nblocks: int, out):
    ctx.check(ctx.lib.krp_philox_words(ctx.handle, seed, c1, c2, c3, first_block, nblocks,
                                       _ptr(out)))


def _ld(ld):
    return None if ld is None else _i64(ld)


def krp_sketch_mode(ctx: Context, X, dims: Sequence[int], n: int, omega: Sequence, ell: int, Y,
                    ld: Optional[Sequence[int]] = None):
    om_t = next(o for o in omega if o is not None)
    ctx.check(ctx.lib.krp_sketch_mode(ctx.handle, _ptr(X), _dtype_code(X), len(dims), _i64(dims),
                                      _ld(ld), n, _ptrs(omega), _dtype_code(om_t), ell, _ptr(Y)))


def krp_sketch_all_modes(ctx: Context, X, dims: Sequence[int], omega: Sequence, ell: int,
                         Ys: Sequence, ld: Optional[Sequence[int]] = None, tree_split: int = -1):
    ctx.check(ctx.lib.krp_sketch_all_modes(ctx.handle, _ptr(X), _dtype_code(X), len(dims),
                                           _i64(dims), _ld(ld), _ptrs(omega),
                                           _dtype_code(omega[0]), ell, _ptrs(Ys), tree_split))


def krp_qr(ctx: Context, Ys: Sequence, ms: Sequence[int], ls: Sequence[int], Qs: Sequence,
           Rs: Optional[Sequence] = None):
    ctx.check(ctx.lib.krp_qr(ctx.handle, len(Ys), _ptrs(Ys), _i64(ms), _i32(ls), _ptrs(Qs),
                             _ptrs(Rs) if Rs is not None else None))


KRP_QR_NOALLOC_MAX_DOUBLES = 524288


def krp_qr_noalloc(Y, m: int, l: int, Q, R=None, stream: Optional[int] = None) -> int:
    """Thin QR of one FP32 matrix without device allocation (no context).

    For callers that may not allocate while running; the library keeps one
    fixed 4 MiB scratch array per GPU for it, shared by all calls (overlapping
    calls race).  Returns the krp_status code (0 = KRP_OK).
    """
    lib = load_library()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    return int(lib.krp_qr_noalloc(_ptr(Y), m, l, _ptr(Q), _ptr(R), C.c_void_p(stream)))


def krp_multi_ttm(ctx: Context, X, dims: Sequence[int], Qs: Sequence, cols: Sequence[int], G,
                  ld: Optional[Sequence[int]] = None):
    ctx.check(ctx.lib.krp_multi_ttm(ctx.handle, _ptr(X), _dtype_code(X), len(dims), _i64(dims),
                                    _ld(ld), _ptrs(Qs), _i32(cols), _ptr(G)))


def krp_core_truncate(ctx: Context, dims: Sequence[int], ell: Sequence[int], ranks: Sequence[int],
                      core, factors: Sequence, core_out, factors_out: Sequence):
    ctx.check(ctx.lib.krp_core_truncate(ctx.handle, len(dims), _i64(dims), _i32(ell), _i32(ranks),
                                        _ptr(core), _ptrs(factors), _ptr(core_out),
                                        _ptrs(factors_out)))


def krp_residual(ctx: Context, X, dims: Sequence[int], core_dims: Sequence[int], core,
                 factors: Sequence, ld: Optional[Sequence[int]] = None):
    """Returns (||X - X_hat||_F^2, ||X||_F^2) as Python floats."""
    sums = (C.c_double * 2)()
    ctx.check(ctx.lib.krp_residual(ctx.handle, _ptr(X), _dtype_code(X), len(dims), _i64(dims),
                                   _ld(ld), _i32(core_dims), _ptr(core), _ptrs(factors), sums))
    return float(sums[0]), float(sums[1])


def _tucker(fn, ctx, X, dims, ranks, oversample, seed, flags, core, factors, ld=None):
    out = TuckerOut()
    out.core = _ptr(core)
    for i, f in enumerate(factors):
        out.factors[i] = _ptr(f)
    ctx.check(fn(ctx.handle, _ptr(X), _dtype_code(X), len(dims), _i64(dims), _ld(ld),
                 _i32(ranks), oversample, seed, flags, C.byref(out)))
    t = out.times
    return {
        "core_dims": [int(out.core_dims[i]) for i in range(out.d)],
        "rel_residual": out.rel_residual,
        "x_norm": out.x_norm,
        "core_norm": out.core_norm,
        "times": {k: getattr(t, k) for k, _ in PhaseTimes._fields_},
    }


def krp_tucker_rhosvd(ctx: Context, X, dims, ranks, oversample, seed, flags, core, factors,
                      ld=None):
    """RHOSVD-KRP (Alg. 7); core/factors are preallocated outputs."""
    return _tucker(ctx.lib.krp_tucker_rhosvd, ctx, X, dims, ranks, oversample, seed, flags, core,
                   factors, ld)


def krp_tucker_sthosvd(ctx: Context, X, dims, ranks, oversample, seed, flags, core, factors,
                       ld=None):
    """RSTHOSVD-KRP (Alg. 8); core/factors are preallocated outputs."""
    return _tucker(ctx.lib.krp_tucker_sthosvd, ctx, X, dims, ranks, oversample, seed, flags,
                   core, factors, ld)


def krp_block_hankel_lowrank(ctx: Context, blocks, m, n, s, r, ell_r, ell_l, seed, U, S, V):
    ctx.check(ctx.lib.krp_block_hankel_lowrank(ctx.handle, _ptr(blocks), _dtype_code(blocks), m,
                                               n, s, r, ell_r, ell_l, seed, _ptr(U), _ptr(S),
                                               _ptr(V)))


def krp_tucker_hadamard(ctx: Context, dims, rg, G, Us, rh, H, Vs, ell, seed, core, factors):
    """RHOSVD-KRP-MEMO of the Hadamard product of two Tucker tensors; returns the relative error."""
    err = C.c_double(0.0)
    ctx.check(ctx.lib.krp_tucker_hadamard(ctx.handle, len(dims), _i64(dims), _i32(rg), _ptr(G),
                                          _ptrs(Us), _i32(rh), _ptr(H), _ptrs(Vs), ell, seed,
                                          _ptr(core), _ptrs(factors), C.byref(err)))
    return err.value


def krp_sensor_select(ctx: Context, dims, ells, Qs, idxs, As):
    """Sensor indices (int32, device) and interpolation factors of the factors Qs."""
    ctx.check(ctx.lib.krp_sensor_select(ctx.handle, len(dims), _i64(dims), _i32(ells), _ptrs(Qs),
                                        _ptrs(idxs), _ptrs(As)))


def krp_sensor_reconstruct(ctx: Context, dims, ells, As, T_hat, out):
    """out = T_hat x_1 A_1 ... x_d A_d (FP32 tensors, FP64 factors, device)."""
    ctx.check(ctx.lib.krp_sensor_reconstruct(ctx.handle, len(dims), _i64(dims), _i32(ells),
                                             _ptrs(As), _ptr(T_hat), _ptr(out)))


def krp_block_hankel_nystrom(ctx: Context, blocks, m, s, r, ell, seed, U, L, rcond=0.0):
    """Top r eigenpairs (U, L) of the Nystrom approximation of an SPSD block Hankel matrix."""
    ctx.check(ctx.lib.krp_block_hankel_nystrom(ctx.handle, _ptr(blocks), _dtype_code(blocks), m, s,
                                               r, ell, float(rcond), seed, _ptr(U), _ptr(L)))


def krp_block_hankel2_lowrank(ctx: Context, blocks, m, n, s1, s2, r, ell_r, ell_l, seed, U, S, V):
    """Alg. 6 on a two-level block Hankel matrix (blocks (k1, k2) at k1 + (2 s1 - 1) k2)."""
    ctx.check(ctx.lib.krp_block_hankel2_lowrank(ctx.handle, _ptr(blocks), _dtype_code(blocks), m,
                                                n, s1, s2, r, ell_r, ell_l, seed, _ptr(U),
                                                _ptr(S), _ptr(V)))


def krp_era_realize(ctx: Context, blocks, m, n, s, r, U, S, V, eig_re, eig_im, A=None):
    """Eigensystem realization from krp_block_hankel_lowrank's U, S, V (device)."""
    ctx.check(ctx.lib.krp_era_realize(ctx.handle, _ptr(blocks), _dtype_code(blocks), m, n, s, r,
                                      _ptr(U), _ptr(S), _ptr(V), _ptr(A), _ptr(eig_re),
                                      _ptr(eig_im)))


def krp_block_hankel_sketch(ctx: Context, blocks, m, n, s, omega1, omega2, ell_r, psi1, psi2,
                            ell_l, Y, Z):
    ctx.check(ctx.lib.krp_block_hankel_sketch(ctx.handle, _ptr(blocks), _dtype_code(blocks), m,
                                              n, s, _ptr(omega1), _ptr(omega2), ell_r, _ptr(psi1),
                                              _ptr(psi2), ell_l, _ptr(Y), _ptr(Z)))


def make_tucker_items(xs, dims, ranks, seeds, cores, factors):
    """Array of krp_tucker_item from per-tensor lists (kept by the caller so
    that a repeated call can pass the same descriptors)."""
    n = len(xs)
    arr = (TuckerItem * n)()
    for b in range(n):
        it = arr[b]
        it.X = _ptr(xs[b])
        for m in range(3):
            it.dims[m] = int(dims[b][m])
            it.ranks[m] = int(ranks[b][m])
            it.factors[m] = _ptr(factors[b][m])
        it.seed = int(seeds[b])
        it.core = _ptr(cores[b])
        it.rel_residual = 0.0
    return arr


def krp_tucker_rhosvd_batched(ctx: Context, xt: int, items, oversample: int, flags: int):
    """Batched RHOSVD-KRP-MEMO of 3-way tensors; fills items[b].rel_residual."""
    ctx.check(ctx.lib.krp_tucker_rhosvd_batched(ctx.handle, int(xt), len(items), items,
                                                int(oversample), int(flags)))
    return [items[b].rel_residual for b in range(len(items))]


def krp_tucker_batch_plan_info(ctx: Context):
    a, b, c = C.c_int(0), C.c_int(0), C.c_int(0)
    ctx.check(ctx.lib.krp_tucker_batch_plan_info(ctx.handle, C.byref(a), C.byref(b), C.byref(c)))
    return {"slabs_per_unit": a.value, "units": b.value, "grid": c.value}


def make_hankel_items(blocks, shapes, seeds, Us, Ss, Vs):
    """Array of krp_hankel_item; shapes[b] = (m, n, s, r, ell_r, ell_l)."""
    n = len(blocks)
    arr = (HankelItem * n)()
    for b in range(n):
        it = arr[b]
        it.blocks = _ptr(blocks[b])
        it.m, it.n, it.s, it.r, it.ell_r, it.ell_l = (int(v) for v in shapes[b])
        it.seed = int(seeds[b])
        it.U, it.S, it.V = _ptr(Us[b]), _ptr(Ss[b]), _ptr(Vs[b])
    return arr


def krp_block_hankel_batched(ctx: Context, bt: int, items):
    """Batched Alg. 6 over block Hankel matrices (outputs in the items' U, S, V)."""
    ctx.check(ctx.lib.krp_block_hankel_batched(ctx.handle, int(bt), len(items), items))


def krp_split_bf16x2(ctx: Context, X, out=None):
    """BF16 hi/lo pair of an FP32 device tensor (returns a BF16x2 input)."""
    import torch
    n = X.numel()
    if out is None:
        out = torch.empty(2 * n, dtype=torch.bfloat16, device=X.device)
    ctx.check(ctx.lib.krp_split_bf16x2(ctx.handle, _ptr(X), n, _ptr(out)))
    return BF16x2(out)


def krp_trace_begin(ctx: Context):
    ctx.check(ctx.lib.krp_trace_begin(ctx.handle))


def krp_trace_end(ctx: Context, cap: int = 1 << 20):
    """List of (launch name, ms) in launch order since krp_trace_begin."""
    import json
    buf = C.create_string_buffer(cap)
    ctx.check(ctx.lib.krp_trace_end(ctx.handle, buf, cap))
    return [(n, float(t)) for n, t in json.loads(buf.value.decode())]
