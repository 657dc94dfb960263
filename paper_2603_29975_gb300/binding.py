"""ctypes binding of libozk.so (include/ozk.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  Matrices are torch complex128
CUDA tensors in column-major layout (``t.stride(0) == 1``), as the C ABI expects; use
``colmajor_cuda(array)`` to move a numpy matrix to the GPU in that layout.  There is no
CPU fallback: if the library is missing or the device is not a CUDA GPU, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libozk.so")

OZK_OK = 0
OZK_ERR_TIMEOUT = 4
OZK_PAIRS_TRI = 0
OZK_PAIRS_FULL = 1
OZK_SEL_FEATURES = 16
OZK_SEL_OUTPUTS = 8
OZK_SEL_NPARAMS = 5768
OZK_SEL_SMIN, OZK_SEL_SMAX = 3, 10
OZK_SEL_NO_FALLBACK = 1
OZK_NB_MAX = 112
OZK_PANEL_MAX = 448
SELECTOR_WEIGHTS = os.path.join(HERE, "selector_weights.bin")


class SelectorInfo(ctypes.Structure):
    """ozk_selector_info (include/ozk.h)."""
    _fields_ = [("S_selected", ctypes.c_int), ("S_used", ctypes.c_int), ("fallback", ctypes.c_int),
                ("residual_ok", ctypes.c_int), ("residual", ctypes.c_double),
                ("residual_selected", ctypes.c_double),
                ("predicted_log10_err", ctypes.c_float * OZK_SEL_OUTPUTS), ("probe_seed", ctypes.c_uint64),
                ("gemms", ctypes.c_int), ("S_count", ctypes.c_int * OZK_SEL_OUTPUTS)]
STATUS_NAMES = {1: "ARG", 2: "NONFINITE", 3: "SINGULAR", 4: "TIMEOUT", 5: "CUDA", 6: "RANGE",
                7: "CAPTURE", 8: "RESIDUAL", 9: "NOFILE"}

EXPORTS = ["ozk_create", "ozk_destroy", "ozk_set_stream", "ozk_get_status", "ozk_reserve",
           "ozk_zgemm_workspace_size", "ozk_last_error", "ozk_launch_count", "ozaki_zgemm",
           "ozaki_zgemm_vbatched", "ozk_zgemm_dmma", "ozk_split_debug", "ozk_group_sums_debug",
           "kkr_build_m", "kkr_tau00", "kkr_tau00_batched", "ozk_profile_begin", "ozk_profile_end",
           "kkr_build_m_batched", "ozaki_zgemm_noalloc", "ozk_selector_init", "ozk_selector_set_params",
           "ozk_selector_get_params", "ozk_selector_load", "ozk_selector_save", "ozk_selector_configure",
           "ozk_selector_features", "ozk_selector_predict", "ozk_selector_train_step", "ozk_selector_gradient",
           "ozk_selector_last", "ozk_rel_diff", "kkr_build_m_shared", "kkr_tau00_autotune",
           "kkr_build_m_shared_sizes", "kkr_contour_trace", "ozaki2_zgemm", "ozaki_ztrsm", "kkr_tau00_lu",
           "ozk_profile_moved", "ozk_debug_stall_next_gemm", "kkr_tau00_batched_panels",
           "kkr_tau00_autotune_panels", "ozk_selector_log_begin", "ozk_selector_log_end"]
KIND_NAMES = ["split", "slice_gemm", "gj", "build_m", "dmma", "other"]

_lib = None


class OzkError(RuntimeError):
    pass


def lib():
    """Load libozk.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OzkError(f"{LIB_PATH} is missing: build it with paper_2603_29975_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp, c, i, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), \
            ctypes.c_char, ctypes.c_int, ctypes.c_size_t
        L.ozk_create.argtypes = [ctypes.POINTER(vp)]
        L.ozk_destroy.argtypes = [vp]
        L.ozk_set_stream.argtypes = [vp, vp]
        L.ozk_get_status.argtypes = [vp, ip]
        L.ozk_reserve.argtypes = [vp, sz]
        L.ozk_zgemm_workspace_size.argtypes = [i, i, i, i, i]
        L.ozk_zgemm_workspace_size.restype = sz
        L.ozk_last_error.restype = ctypes.c_char_p
        L.ozk_launch_count.restype = ctypes.c_uint64
        L.ozaki_zgemm.argtypes = [vp, c, c, i, i, i, dp, vp, i, vp, i, dp, vp, i, i, i]
        L.ozaki_zgemm_vbatched.argtypes = [vp, c, c, ip, ip, ip, dp, vp, ip, vp, ip, dp, vp, ip, i, i, i]
        L.ozk_zgemm_dmma.argtypes = [vp, c, c, i, i, i, dp, vp, i, vp, i, dp, vp, i]
        L.ozk_split_debug.argtypes = [vp, i, c, i, i, vp, i, i, vp, vp]
        L.ozk_group_sums_debug.argtypes = [vp, c, c, i, i, i, vp, i, vp, i, i, i, vp]
        L.kkr_build_m.argtypes = [vp, i, i, vp, vp, vp]
        L.kkr_tau00.argtypes = [vp, i, i, vp, vp, vp, i, i]
        L.kkr_tau00_batched.argtypes = [vp, i, ip, i, vp, vp, vp, i, i]
        L.kkr_tau00_batched_panels.argtypes = [vp, i, ip, i, vp, vp, vp, i, i, i]
        L.kkr_tau00_autotune_panels.argtypes = [vp, i, ip, i, i, ip, ip, ctypes.POINTER(ctypes.c_float), ip, i, ip]
        L.kkr_build_m_batched.argtypes = [vp, i, ip, i, vp, vp, vp]
        L.kkr_build_m_shared.argtypes = [vp, i, i, i, vp, vp, vp, i]
        L.kkr_tau00_autotune.argtypes = [vp, i, ip, i, i, ip, ctypes.POINTER(ctypes.c_float)]
        L.kkr_build_m_shared_sizes.argtypes = [vp, i, ip, i, vp, vp, i, vp, i]
        L.kkr_contour_trace.argtypes = [vp, i, i, vp, dp, dp, dp]
        L.ozaki2_zgemm.argtypes = [vp, c, c, i, i, i, dp, vp, i, vp, i, dp, vp, i, i]
        L.ozaki_ztrsm.argtypes = [vp, c, c, i, i, vp, i, vp, i, i]
        L.kkr_tau00_lu.argtypes = [vp, i, i, vp, vp, vp, i, i]
        L.ozaki_zgemm_noalloc.argtypes = [vp, c, c, i, i, i, dp, vp, i, vp, i, dp, vp, i, i, i, vp]
        fp, u64, f32 = ctypes.POINTER(ctypes.c_float), ctypes.c_uint64, ctypes.c_float
        L.ozk_selector_init.argtypes = [vp, u64]
        L.ozk_selector_set_params.argtypes = [vp, fp]
        L.ozk_selector_get_params.argtypes = [vp, fp]
        L.ozk_selector_load.argtypes = [vp, ctypes.c_char_p]
        L.ozk_selector_save.argtypes = [vp, ctypes.c_char_p]
        L.ozk_selector_configure.argtypes = [vp, ctypes.c_double, ctypes.c_double, i]
        L.ozk_selector_features.argtypes = [vp, c, c, i, i, i, vp, i, vp, i, u64, vp]
        L.ozk_selector_predict.argtypes = [vp, i, vp, vp]
        L.ozk_selector_train_step.argtypes = [vp, i, vp, vp, f32, dp]
        L.ozk_selector_gradient.argtypes = [vp, i, vp, vp, vp]
        L.ozk_selector_last.argtypes = [vp, ctypes.POINTER(SelectorInfo)]
        L.ozk_selector_log_begin.argtypes = [vp, vp, vp, i]
        L.ozk_selector_log_end.argtypes = [vp, ip]
        L.ozk_rel_diff.argtypes = [vp, i, i, vp, i, vp, i, dp]
        L.ozk_profile_begin.argtypes = [vp]
        L.ozk_profile_end.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), dp, dp, dp]
        L.ozk_profile_moved.argtypes = [vp, dp]
        L.ozk_debug_stall_next_gemm.argtypes = [vp, ctypes.c_longlong]
        for name in EXPORTS:
            if name not in ("ozk_zgemm_workspace_size", "ozk_last_error", "ozk_launch_count"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(st: int, what: str):
    if st != OZK_OK:
        msg = lib().ozk_last_error().decode(errors="replace")
        raise OzkError(f"{what} failed: status {st} ({STATUS_NAMES.get(st, '?')}): {msg}")


def _c2(z: complex):
    return (ctypes.c_double * 2)(float(complex(z).real), float(complex(z).imag))


def _ld(t, rows: int) -> int:
    """Leading dimension of a column-major complex tensor with `rows` rows."""
    if t.dim() != 2:
        raise OzkError("expected a 2-D tensor")
    if t.shape[0] > 1 and t.stride(0) != 1:
        raise OzkError("matrix must be column major (stride(0) == 1)")
    return max(1, rows, t.stride(1) if t.shape[1] > 1 else rows)


def _ptr(t) -> int:
    import torch
    if t.dtype != torch.complex128 or not t.is_cuda:
        raise OzkError("expected a complex128 CUDA tensor")
    return t.data_ptr()


def colmajor_cuda(a, device="cuda"):
    """numpy complex matrix -> complex128 CUDA tensor in column-major layout."""
    import torch
    a = np.asfortranarray(np.asarray(a, dtype=np.complex128))
    return torch.from_numpy(a).to(device)


def to_numpy(t) -> np.ndarray:
    return t.detach().cpu().numpy()


def launch_count() -> int:
    return int(lib().ozk_launch_count())


class Handle:
    """An ozk handle bound to the current torch CUDA stream (or the one given)."""

    def __init__(self, stream=None):
        import torch
        self._h = ctypes.c_void_p()
        _check(lib().ozk_create(ctypes.byref(self._h)), "ozk_create")
        self.set_stream(stream if stream is not None else torch.cuda.current_stream())

    def set_stream(self, stream):
        _check(lib().ozk_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)), "ozk_set_stream")

    @property
    def ptr(self):
        return self._h

    def status(self) -> int:
        v = ctypes.c_int(0)
        _check(lib().ozk_get_status(self._h, ctypes.byref(v)), "ozk_get_status")
        return v.value

    def reserve(self, nbytes: int):
        _check(lib().ozk_reserve(self._h, nbytes), "ozk_reserve")

    def debug_stall_next_gemm(self, cycles: int):
        """Test hook: the next slice-GEMM launch's bounded waits run out after `cycles` SM cycles."""
        _check(lib().ozk_debug_stall_next_gemm(self._h, int(cycles)), "ozk_debug_stall_next_gemm")

    def profile_begin(self):
        _check(lib().ozk_profile_begin(self._h), "ozk_profile_begin")

    def profile_end(self) -> dict:
        """Per kernel kind: launches, device ms, algorithmic flops and bytes (CUDA events)."""
        K = len(KIND_NAMES)
        n = (ctypes.c_uint64 * K)()
        ms, fl, by = (ctypes.c_double * K)(), (ctypes.c_double * K)(), (ctypes.c_double * K)()
        _check(lib().ozk_profile_end(self._h, n, ms, fl, by), "ozk_profile_end")
        mv = (ctypes.c_double * K)()
        _check(lib().ozk_profile_moved(self._h, mv), "ozk_profile_moved")
        return {KIND_NAMES[k]: {"launches": int(n[k]), "ms": float(ms[k]), "flops": float(fl[k]),
                                "bytes": float(by[k]), "bytes_moved": float(mv[k])} for k in range(K)}

    # ---- slice-count selector
    def selector_init(self, seed: int = 1):
        _check(lib().ozk_selector_init(self._h, seed), "ozk_selector_init")

    def selector_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != OZK_SEL_NPARAMS:
            raise OzkError(f"expected {OZK_SEL_NPARAMS} parameters")
        _check(lib().ozk_selector_set_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "ozk_selector_set_params")

    def selector_get_params(self) -> np.ndarray:
        p = np.zeros(OZK_SEL_NPARAMS, dtype=np.float32)
        _check(lib().ozk_selector_get_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "ozk_selector_get_params")
        return p

    def selector_load(self, path: str = SELECTOR_WEIGHTS):
        _check(lib().ozk_selector_load(self._h, os.fsencode(path)), "ozk_selector_load")

    def selector_save(self, path: str):
        _check(lib().ozk_selector_save(self._h, os.fsencode(path)), "ozk_selector_save")

    def selector_configure(self, tol: float = 1e-10, margin: float = 0.6, flags: int = 0):
        _check(lib().ozk_selector_configure(self._h, tol, margin, flags), "ozk_selector_configure")

    def selector_log_begin(self, features, targets):
        """Start logging selector training rows into float32 CUDA tensors (N x 16, N x 8)."""
        _check(lib().ozk_selector_log_begin(self._h, _f32(features, (features.shape[0], OZK_SEL_FEATURES)),
                                            _f32(targets, (features.shape[0], OZK_SEL_OUTPUTS)),
                                            int(features.shape[0])), "ozk_selector_log_begin")

    def selector_log_end(self) -> int:
        n = ctypes.c_int(0)
        _check(lib().ozk_selector_log_end(self._h, ctypes.byref(n)), "ozk_selector_log_end")
        return n.value

    def selector_last(self) -> dict:
        info = SelectorInfo()
        _check(lib().ozk_selector_last(self._h, ctypes.byref(info)), "ozk_selector_last")
        return {"S_selected": info.S_selected, "S_used": info.S_used, "fallback": bool(info.fallback),
                "residual_ok": bool(info.residual_ok), "residual": info.residual,
                "residual_selected": info.residual_selected,
                "predicted_log10_err": [float(v) for v in info.predicted_log10_err],
                "probe_seed": int(info.probe_seed), "gemms": info.gemms,
                "S_count": {3 + o: int(info.S_count[o]) for o in range(OZK_SEL_OUTPUTS) if info.S_count[o]}}

    def close(self):
        if self._h:
            lib().ozk_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _shapes(transa, transb, A, B):
    m, ka = (A.shape[0], A.shape[1]) if transa in "Nn" else (A.shape[1], A.shape[0])
    kb, n = (B.shape[0], B.shape[1]) if transb in "Nn" else (B.shape[1], B.shape[0])
    if ka != kb:
        raise OzkError(f"inner dimensions differ: {ka} vs {kb}")
    return m, n, ka


def ozaki_zgemm(h: Handle, A, B, C, S: int = 7, alpha=1.0, beta=0.0, transa="N", transb="N",
                pair_mode: int = OZK_PAIRS_TRI):
    """C = alpha op(A) op(B) + beta C (emulated, S slices) on column-major tensors."""
    m, n, k = _shapes(transa, transb, A, B)
    if tuple(C.shape) != (m, n):
        raise OzkError("C has the wrong shape")
    _check(lib().ozaki_zgemm(h.ptr, transa.encode(), transb.encode(), m, n, k, _c2(alpha), _ptr(A),
                             _ld(A, A.shape[0]), _ptr(B), _ld(B, B.shape[0]), _c2(beta), _ptr(C),
                             _ld(C, m), S, pair_mode), "ozaki_zgemm")
    return C


def ozaki2_zgemm(h: Handle, A, B, C, nmod: int = 16, alpha=1.0, beta=0.0, transa="N", transb="N"):
    """C = alpha op(A) op(B) + beta C by Ozaki-II (CRT) with nmod moduli, column-major tensors."""
    m, n, k = _shapes(transa, transb, A, B)
    if tuple(C.shape) != (m, n):
        raise OzkError("C has the wrong shape")
    _check(lib().ozaki2_zgemm(h.ptr, transa.encode(), transb.encode(), m, n, k, _c2(alpha), _ptr(A),
                              _ld(A, A.shape[0]), _ptr(B), _ld(B, B.shape[0]), _c2(beta), _ptr(C), _ld(C, m), nmod),
           "ozaki2_zgemm")
    return C


def ozaki_zgemm_noalloc(A, B, C, S: int = 7, alpha=1.0, beta=0.0, transa="N", transb="N",
                        pair_mode: int = OZK_PAIRS_TRI, stream=None, device_status=None):
    """Allocation-free emulated ZGEMM (static scratch inside the library, no handle)."""
    import torch
    m, n, k = _shapes(transa, transb, A, B)
    if tuple(C.shape) != (m, n):
        raise OzkError("C has the wrong shape")
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().ozaki_zgemm_noalloc(ctypes.c_void_p(s.cuda_stream), transa.encode(), transb.encode(), m, n, k,
                                     _c2(alpha), _ptr(A), _ld(A, A.shape[0]), _ptr(B), _ld(B, B.shape[0]), _c2(beta),
                                     _ptr(C), _ld(C, m), S, pair_mode,
                                     ctypes.c_void_p(device_status.data_ptr() if device_status is not None else 0)),
           "ozaki_zgemm_noalloc")
    return C


def ozk_zgemm_dmma(h: Handle, A, B, C, alpha=1.0, beta=0.0, transa="N", transb="N"):
    m, n, k = _shapes(transa, transb, A, B)
    if tuple(C.shape) != (m, n):
        raise OzkError("C has the wrong shape")
    _check(lib().ozk_zgemm_dmma(h.ptr, transa.encode(), transb.encode(), m, n, k, _c2(alpha), _ptr(A),
                                _ld(A, A.shape[0]), _ptr(B), _ld(B, B.shape[0]), _c2(beta), _ptr(C),
                                _ld(C, m)), "ozk_zgemm_dmma")
    return C


def ozaki_zgemm_vbatched(h: Handle, As, Bs, Cs, S: int = 7, alpha=1.0, beta=0.0, transa="N",
                         transb="N", pair_mode: int = OZK_PAIRS_TRI):
    """Variable-size batch: lists of column-major tensors."""
    import torch
    nb = len(As)
    dims = [_shapes(transa, transb, a, b) for a, b in zip(As, Bs)]
    I = ctypes.c_int * nb
    m = I(*[d[0] for d in dims]); n = I(*[d[1] for d in dims]); k = I(*[d[2] for d in dims])
    lda = I(*[_ld(a, a.shape[0]) for a in As]); ldb = I(*[_ld(b, b.shape[0]) for b in Bs])
    ldc = I(*[_ld(c, d[0]) for c, d in zip(Cs, dims)])
    dev = As[0].device
    pa = torch.tensor([_ptr(a) for a in As], dtype=torch.int64, device=dev)
    pb = torch.tensor([_ptr(b) for b in Bs], dtype=torch.int64, device=dev)
    pc = torch.tensor([_ptr(c) for c in Cs], dtype=torch.int64, device=dev)
    _check(lib().ozaki_zgemm_vbatched(h.ptr, transa.encode(), transb.encode(), m, n, k, _c2(alpha),
                                      pa.data_ptr(), lda, pb.data_ptr(), ldb, _c2(beta), pc.data_ptr(), ldc,
                                      nb, S, pair_mode), "ozaki_zgemm_vbatched")
    return Cs, (pa, pb, pc)


def ozk_split_debug(h: Handle, X, side: int, S: int, trans: str = "N"):
    """Exponents (int32) and digits (int16, [S][rows'][2k]) of op(X) as left/right operand."""
    import torch
    if side == 0:
        rows, k = (X.shape[0], X.shape[1]) if trans in "Nn" else (X.shape[1], X.shape[0])
    else:
        k, rows = (X.shape[0], X.shape[1]) if trans in "Nn" else (X.shape[1], X.shape[0])
    rows_out = rows if side == 0 else 2 * rows
    e = torch.zeros(rows, dtype=torch.int32, device=X.device)
    d = torch.zeros((S, rows_out, 2 * k), dtype=torch.int16, device=X.device)
    _check(lib().ozk_split_debug(h.ptr, side, trans.encode(), rows, k, _ptr(X), _ld(X, X.shape[0]), S,
                                 e.data_ptr(), d.data_ptr()), "ozk_split_debug")
    return e, d


def ozk_group_sums_debug(h: Handle, A, B, S: int, pair_mode: int = OZK_PAIRS_TRI, transa="N", transb="N"):
    """Exact group sums G_g (int64 [G][m][2n]) computed by the tensor-core kernel."""
    import torch
    m, n, k = _shapes(transa, transb, A, B)
    G = 2 * S - 1 if pair_mode == OZK_PAIRS_FULL else S
    out = torch.zeros((G, m, 2 * n), dtype=torch.int64, device=A.device)
    _check(lib().ozk_group_sums_debug(h.ptr, transa.encode(), transb.encode(), m, n, k, _ptr(A),
                                      _ld(A, A.shape[0]), _ptr(B), _ld(B, B.shape[0]), S, pair_mode,
                                      out.data_ptr()), "ozk_group_sums_debug")
    return out


def kkr_build_m(h: Handle, t, G, M):
    """M = I - blockdiag(t) G; t is (L, b, b) complex128 with column-major blocks."""
    L, b = t.shape[0], t.shape[1]
    if not t.is_contiguous():
        raise OzkError("t must be contiguous (L x b x b blocks, each column major)")
    _check(lib().kkr_build_m(h.ptr, L, b, _ptr(t), _ptr(G), _ptr(M)), "kkr_build_m")
    return M


def kkr_build_m_batched_ptrs(h: Handle, L_list, b: int, pt, pg, pm):
    """Batched M = I - t G with device pointer arrays (int64 CUDA tensors)."""
    nb_ = len(L_list)
    L = (ctypes.c_int * nb_)(*[int(v) for v in L_list])
    _check(lib().kkr_build_m_batched(h.ptr, nb_, L, b, pt.data_ptr(), pg.data_ptr(), pm.data_ptr()),
           "kkr_build_m_batched")


def kkr_build_m_shared_ptrs(h: Handle, natoms: int, L: int, b: int, pt, G, pm, S: int = 7):
    """M_a = I - blockdiag(t_a) G for atoms sharing G, emulated with S slices; pt, pm: int64
    CUDA tensors of device pointers (t blocks, M outputs), G a column-major CUDA tensor."""
    _check(lib().kkr_build_m_shared(h.ptr, natoms, L, b, pt.data_ptr(), _ptr(G), pm.data_ptr(), S),
           "kkr_build_m_shared")


def kkr_build_m_shared_sizes_ptrs(h: Handle, L_list, b: int, pt, G, pm, S: int = 7):
    """M_a = I - blockdiag(t_a) G[:L_a b, :L_a b] for atoms with LIZ sizes L_list sharing the
    largest LIZ's G (column-major CUDA tensor); pt, pm: int64 CUDA tensors of device pointers."""
    na = len(L_list)
    Ls = (ctypes.c_int * na)(*[int(v) for v in L_list])
    _check(lib().kkr_build_m_shared_sizes(h.ptr, na, Ls, b, pt.data_ptr(), _ptr(G), _ld(G, G.shape[0]),
                                          pm.data_ptr(), S), "kkr_build_m_shared_sizes")


def kkr_contour_trace(h: Handle, ptau, b: int, weights):
    """Tr tau_00(z_i) and sum_i w_i Tr tau_00(z_i) for the blocks behind the int64 CUDA tensor
    of device pointers `ptau`; returns (numpy complex traces, complex integral)."""
    ns = int(ptau.numel())
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.complex128))
    if w.size != ns:
        raise OzkError("one weight per block")
    tr = np.zeros(ns, dtype=np.complex128)
    out = np.zeros(1, dtype=np.complex128)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().kkr_contour_trace(h.ptr, ns, b, ptau.data_ptr(), w.ctypes.data_as(dp), tr.ctypes.data_as(dp),
                                   out.ctypes.data_as(dp)), "kkr_contour_trace")
    return tr, complex(out[0])


def kkr_tau00_autotune(h: Handle, n_list, b: int, S: int = 7):
    """Time every panel width for these sizes; returns (best nb, {nb: ms})."""
    ns = len(n_list)
    n = (ctypes.c_int * ns)(*[int(v) for v in n_list])
    cands = list(range(b, OZK_NB_MAX + 1, b))
    times = (ctypes.c_float * len(cands))()
    best = ctypes.c_int(0)
    _check(lib().kkr_tau00_autotune(h.ptr, ns, n, b, S, ctypes.byref(best), times), "kkr_tau00_autotune")
    return best.value, {nb: float(times[i]) for i, nb in enumerate(cands)}


def kkr_tau00_autotune_panels(h: Handle, n_list, b: int, S: int = 7):
    """Time every (panel, leaf) width pair for these sizes; returns ((W, w), {(W, w): ms})."""
    ns = len(n_list)
    n = (ctypes.c_int * ns)(*[int(v) for v in n_list])
    cap = 256
    times = (ctypes.c_float * cap)()
    cand = (ctypes.c_int * (2 * cap))()
    W, w, nc = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().kkr_tau00_autotune_panels(h.ptr, ns, n, b, S, ctypes.byref(W), ctypes.byref(w), times, cand, cap,
                                           ctypes.byref(nc)), "kkr_tau00_autotune_panels")
    return (W.value, w.value), {(cand[2 * c], cand[2 * c + 1]): float(times[c]) for c in range(nc.value)}


def kkr_tau00(h: Handle, M, t0, tau, S: int = 7, nb: int = 64):
    """tau_00 = [M^-1]_00 t_0 (M is overwritten)."""
    n = M.shape[0]
    b = t0.shape[0]
    _ld(M, n)
    _check(lib().kkr_tau00(h.ptr, n, b, _ptr(M), _ptr(t0), _ptr(tau), S, nb), "kkr_tau00")
    return tau


def ozaki_ztrsm(h: Handle, T, B, uplo: str = "U", diag: str = "N", S: int = 7):
    """X T = B for X, B overwritten (right side; T triangular, column-major tensors)."""
    m, n = B.shape
    if T.shape != (n, n):
        raise OzkError("T must be n x n for an m x n B")
    _check(lib().ozaki_ztrsm(h.ptr, uplo.encode(), diag.encode(), m, n, _ptr(T), _ld(T, n), _ptr(B), _ld(B, m), S),
           "ozaki_ztrsm")
    return B


def kkr_tau00_lu(h: Handle, M, t0, tau, S: int = 7, nb: int = 64):
    """tau_00 with LU-factored pivot blocks and emulated ZTRSMs (M is overwritten)."""
    n = M.shape[0]
    b = t0.shape[0]
    _ld(M, n)
    _check(lib().kkr_tau00_lu(h.ptr, n, b, _ptr(M), _ptr(t0), _ptr(tau), S, nb), "kkr_tau00_lu")
    return tau


def kkr_tau00_batched(h: Handle, Ms, t0s, taus, S: int = 7, nb: int = 64, leaf: int = None):
    """Batched tau_00 over lists of column-major tensors (the Ms are overwritten).  With `leaf`
    given, nb is the panel width and leaf the pivot-block width (kkr_tau00_batched_panels)."""
    import torch
    ns = len(Ms)
    b = t0s[0].shape[0]
    dev = Ms[0].device
    pm = torch.tensor([_ptr(M) for M in Ms], dtype=torch.int64, device=dev)
    pt = torch.tensor([_ptr(t) for t in t0s], dtype=torch.int64, device=dev)
    pu = torch.tensor([_ptr(u) for u in taus], dtype=torch.int64, device=dev)
    kkr_tau00_batched_ptrs(h, [int(M.shape[0]) for M in Ms], b, pm, pt, pu, S=S, nb=nb, leaf=leaf)
    return taus, (pm, pt, pu)


def kkr_tau00_batched_ptrs(h: Handle, n_list, b: int, pm, pt, pu, S: int = 7, nb: int = 64, leaf: int = None):
    """Batched tau_00 with device pointer arrays already built (int64 CUDA tensors).  With `leaf`
    given, nb is the panel width and leaf the pivot-block width (kkr_tau00_batched_panels)."""
    ns = len(n_list)
    n = (ctypes.c_int * ns)(*[int(v) for v in n_list])
    if leaf is None:
        _check(lib().kkr_tau00_batched(h.ptr, ns, n, b, pm.data_ptr(), pt.data_ptr(), pu.data_ptr(), S, nb),
               "kkr_tau00_batched")
    else:
        _check(lib().kkr_tau00_batched_panels(h.ptr, ns, n, b, pm.data_ptr(), pt.data_ptr(), pu.data_ptr(), S, nb,
                                              leaf), "kkr_tau00_batched_panels")


# ----------------------------------------------------------------------------- selector
def _f32(t, shape):
    import torch
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise OzkError(f"expected a contiguous float32 CUDA tensor of shape {shape}")
    return t.data_ptr()


def selector_features(h: Handle, A, B, transa="N", transb="N", seed: int = 0):
    """The 16 selector features of op(A) op(B) (float32 CUDA tensor)."""
    import torch
    m, n, k = _shapes(transa, transb, A, B)
    f = torch.empty(OZK_SEL_FEATURES, dtype=torch.float32, device=A.device)
    _check(lib().ozk_selector_features(h.ptr, transa.encode(), transb.encode(), m, n, k, _ptr(A),
                                       _ld(A, A.shape[0]), _ptr(B), _ld(B, B.shape[0]), seed, f.data_ptr()),
           "ozk_selector_features")
    return f


def selector_predict(h: Handle, X):
    """Perceptron outputs (N x 8) for features X (N x 16), float32 CUDA tensors."""
    import torch
    N = X.shape[0]
    Y = torch.empty((N, OZK_SEL_OUTPUTS), dtype=torch.float32, device=X.device)
    _check(lib().ozk_selector_predict(h.ptr, N, _f32(X, (N, OZK_SEL_FEATURES)), Y.data_ptr()),
           "ozk_selector_predict")
    return Y


def selector_train_step(h: Handle, X, T, lr: float, want_loss: bool = True):
    """One Adam step on the mean squared error of X (N x 16) against T (N x 8); returns the
    loss before the step (or None)."""
    N = X.shape[0]
    loss = ctypes.c_double(0.0)
    _check(lib().ozk_selector_train_step(h.ptr, N, _f32(X, (N, OZK_SEL_FEATURES)), _f32(T, (N, OZK_SEL_OUTPUTS)),
                                         float(lr), ctypes.byref(loss) if want_loss else None),
           "ozk_selector_train_step")
    return loss.value if want_loss else None


def selector_gradient(h: Handle, X, T):
    import torch
    N = X.shape[0]
    g = torch.empty(OZK_SEL_NPARAMS, dtype=torch.float32, device=X.device)
    _check(lib().ozk_selector_gradient(h.ptr, N, _f32(X, (N, OZK_SEL_FEATURES)), _f32(T, (N, OZK_SEL_OUTPUTS)),
                                       g.data_ptr()), "ozk_selector_gradient")
    return g


def rel_diff(h: Handle, X, Y) -> float:
    """||X - Y||_F / ||Y||_F of two column-major complex CUDA matrices of one shape."""
    if tuple(X.shape) != tuple(Y.shape):
        raise OzkError("shapes differ")
    m, n = X.shape
    out = ctypes.c_double(0.0)
    _check(lib().ozk_rel_diff(h.ptr, m, n, _ptr(X), _ld(X, m), _ptr(Y), _ld(Y, m), ctypes.byref(out)),
           "ozk_rel_diff")
    return out.value
