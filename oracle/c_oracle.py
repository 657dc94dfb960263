"""ctypes loader for the plain C oracle -- TEST INFRASTRUCTURE ONLY.

``build()`` compiles ``oracle/c/ozk_oracle.c`` with gcc (no -march flags, so the same
source builds on x86-64 and on Arm).  The wrappers take numpy arrays in the mathematical
orientation (row-major complex128) like oracle/ozaki.py and oracle/kkr.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "c", "ozk_oracle.c")
_LIB = os.path.join(_HERE, "c", "libozk_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        sp = ctypes.POINTER(ctypes.c_int16)
        lp = ctypes.POINTER(ctypes.c_int64)
        L.oz_row_exponents.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_long, ip]
        L.oz_split_left.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, sp]
        L.oz_split_right.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, sp]
        L.oz_group_sums.argtypes = [sp, sp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, lp]
        L.oz_group_sums.restype = None
        L.oz_round_scaled_hl.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_int]
        L.oz_round_scaled_hl.restype = ctypes.c_double
        L.oz_zgemm.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, dp]
        L.oz_zgemm_fp64.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.oz_zgemm_fp64.restype = None
        L.oz_gepp_inverse.argtypes = [dp, ctypes.c_int]
        L.oz_tau00_block.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, dp]
        L.oz_tau00_full.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp]
        L.oz_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"C oracle {what} failed with status {st}")


def num_threads() -> int:
    return int(lib().oz_num_threads())


def split_left(A, S):
    A = _c(A)
    m, k = A.shape
    e = np.zeros(m, dtype=np.int32)
    D = np.zeros((S, m, 2 * k), dtype=np.int16)
    _check(lib().oz_split_left(_dp(A), m, k, S, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               D.ctypes.data_as(ctypes.POINTER(ctypes.c_int16))), "split_left")
    return e.astype(np.int64), D.astype(np.int64)


def split_right(B, S):
    B = _c(B)
    k, n = B.shape
    f = np.zeros(n, dtype=np.int32)
    D = np.zeros((S, 2 * n, 2 * k), dtype=np.int16)
    _check(lib().oz_split_right(_dp(B), k, n, S, f.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                D.ctypes.data_as(ctypes.POINTER(ctypes.c_int16))), "split_right")
    return f.astype(np.int64), D.astype(np.int64)


def group_sums(DA, DB, S, full=False):
    DA = np.ascontiguousarray(DA, dtype=np.int16)
    DB = np.ascontiguousarray(DB, dtype=np.int16)
    rowsA, Kp = DA.shape[1], DA.shape[2]
    rowsB = DB.shape[1]
    gmax = 2 * S if full else S + 1
    G = np.zeros((gmax - 1, rowsA, rowsB), dtype=np.int64)
    lib().oz_group_sums(DA.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)),
                        DB.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)), S, rowsA, rowsB, Kp,
                        int(full), G.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return {g: G[g - 2] for g in range(2, gmax + 1)}


def round_scaled(T: int, E: int) -> float:
    T &= (1 << 128) - 1
    hi = T >> 64
    if hi >= 1 << 63:
        hi -= 1 << 64
    return float(lib().oz_round_scaled_hl(hi, T & ((1 << 64) - 1), E))


def zgemm(A, B, S, full=False):
    A, B = _c(A), _c(B)
    m, k = A.shape
    n = B.shape[1]
    C = np.zeros((m, n), dtype=np.complex128)
    _check(lib().oz_zgemm(_dp(A), _dp(B), m, n, k, S, int(full), 0, _dp(C)), "zgemm")
    return C


def zgemm_lu(C, A, B, S, full=False):
    A, B = _c(A), _c(B)
    C = np.array(C, dtype=np.complex128, order="C")
    m, k = A.shape
    n = B.shape[1]
    _check(lib().oz_zgemm(_dp(A), _dp(B), m, n, k, S, int(full), 1, _dp(C)), "zgemm_lu")
    return C


def zgemm_fp64(A, B):
    A, B = _c(A), _c(B)
    m, k = A.shape
    n = B.shape[1]
    C = np.zeros((m, n), dtype=np.complex128)
    lib().oz_zgemm_fp64(_dp(A), _dp(B), m, n, k, _dp(C))
    return C


def gepp_inverse(M):
    M = np.array(M, dtype=np.complex128, order="C")
    _check(lib().oz_gepp_inverse(_dp(M), M.shape[0]), "gepp_inverse")
    return M


def tau00_block(M, t0, nb, S=0, full=False, leaf=None):
    M, t0 = _c(M), _c(t0)
    n, b = M.shape[0], t0.shape[0]
    tau = np.zeros((b, b), dtype=np.complex128)
    _check(lib().oz_tau00_block(_dp(M), _dp(t0), n, b, nb, leaf or 0, S or 0, int(full), _dp(tau)),
           "tau00_block")
    return tau


def tau00_full(M, t0):
    M, t0 = _c(M), _c(t0)
    n, b = M.shape[0], t0.shape[0]
    tau = np.zeros((b, b), dtype=np.complex128)
    _check(lib().oz_tau00_full(_dp(M), _dp(t0), n, b, _dp(tau)), "tau00_full")
    return tau
