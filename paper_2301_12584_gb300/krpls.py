"""Thin ctypes binding over libkrpls (include/krpls.h).

Argument marshalling only: every step runs in the CUDA library.  Device
buffers are passed as torch tensors (their data_ptr()) or raw integers;
nothing here computes any part of the method.  If the library has not been
built, lib() raises — there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkrpls.so")

KRP_OK, KRP_EINVAL, KRP_ENOMEM, KRP_ECUDA, KRP_EZERO, KRP_ESINGULAR, KRP_ENUMERIC, KRP_ETIMEOUT, KRP_ESTATE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
KRP_PREC_FP32, KRP_PREC_BF16X3, KRP_PREC_EXACT, KRP_PREC_TF32X3 = 0, 1, 2, 3
KRP_PINV_FALLBACK = 1
KRP_DESCENT_AUTO, KRP_DESCENT_TEAM, KRP_DESCENT_NODE_MAJOR, KRP_DESCENT_NODE_MAJOR_TC = 0, 1, 2, 3

STATUS_NAMES = {0: "KRP_OK", -1: "KRP_EINVAL", -2: "KRP_ENOMEM", -3: "KRP_ECUDA", -4: "KRP_EZERO",
                -5: "KRP_ESINGULAR", -6: "KRP_ENUMERIC", -7: "KRP_ETIMEOUT", -8: "KRP_ESTATE"}

# (name, restype, argtypes) for every symbol declared in include/krpls.h
_P = C.c_void_p
_I64 = C.c_int64
_U64 = C.c_uint64
_INT = C.c_int
SIGNATURES = [
    ("krp_create", _INT, [C.POINTER(_P), _INT, C.POINTER(_I64), _INT, _INT, _INT, _P]),
    ("krp_destroy", None, [_P]),
    ("krp_set_factor", _INT, [_P, _INT, _P]),
    ("krp_set_factor_prec", _INT, [_P, _INT, _P, _INT]),
    ("krp_sample", _INT, [_P, _INT, _I64, _U64, _U64, _P, _P, _P, _P]),
    ("krp_sample_prepare", _INT, [_P, _INT]),
    ("krp_set_descent_form", _INT, [_P, _INT]),
    ("krp_sample_draw", _INT, [_P, _INT, _I64, _U64, _U64, _P, _P, _P, _P]),
    ("krp_launch_count", _I64, []),
    ("krp_exact_count", _INT, [_P, C.POINTER(_I64)]),
    ("krp_debug_wait_timeout", _INT, [_P, _INT]),
    ("krp_debug_sort_pairs", _INT, [_P, _P, _I64, _INT, _P]),
    ("krp_gather", _INT, [_P, _INT, _I64, _P, _P, _P]),
    ("krp_solve_dense", _INT, [_P, _I64, _P, _P, _P, _INT, _P, _INT]),
    ("krp_solve_dense_noalloc", _INT, [_I64, _INT, _P, _P, _P, _INT, _P, _INT, _P, _P]),
    ("krp_sptensor_create", _INT, [C.POINTER(_P), _INT, C.POINTER(_I64), _I64, C.POINTER(_P), _P, _P]),
    ("krp_sptensor_destroy", None, [_P]),
    ("krp_solve_sparse", _INT, [_P, _P, _INT, _I64, _P, _P, _P, _P, _INT]),
    ("krp_cp_als_sweep", _INT, [_P, _P, _I64, _U64, _U64, _P]),
    ("krp_cp_fit", _INT, [_P, _P, _P, C.POINTER(C.c_double)]),
    ("krp_debug_trace", _INT, [_P, _INT, _I64, _U64, _U64, _P, _P, _P, _I64]),
    ("krp_sync_status", _INT, [_P]),
    ("krp_last_error", C.c_char_p, [_P]),
    ("krp_tree_info", _INT, [_P, _INT, C.POINTER(_I64), C.POINTER(_INT), C.POINTER(_INT)]),
    ("krp_get_tree", _INT, [_P, _INT, _P, _I64]),
    ("krp_get_factor", _INT, [_P, _INT, _P, _I64]),
    ("krp_get_tree_exact", _INT, [_P, _INT, _P, _I64, _P, _I64]),
    ("krp_get_prep", _INT, [_P, _INT, _P, _P, _P, C.POINTER(_INT)]),
    ("krp_planted_rows", _INT, [_P, _INT, _I64, _P, _P, _INT, C.c_float, _U64, _P]),
    ("krp_update_entries", _INT, [_P, _INT, _I64, _P, _P, _P]),
    ("krp_kron_rows", _INT, [_P, _INT, _I64, _P, C.POINTER(_P), _P]),
    ("krp_sketch_distortion", _INT, [_P, _INT, _I64, _P, C.POINTER(C.c_double), C.POINTER(_INT)]),
    ("krp_capture_begin", _INT, [_P]),
    ("krp_capture_end", _INT, [_P, C.POINTER(_I64)]),
    ("krp_replay", _INT, [_P]),
    ("krp_batch_create", _INT, [C.POINTER(_P), C.POINTER(_P), _INT, _P]),
    ("krp_batch_destroy", None, [_P]),
    ("krp_batch_set_sources", _INT, [_P, C.POINTER(_P)]),
    ("krp_batch_build", _INT, [_P]),
    ("krp_batch_sample", _INT, [_P, _I64, _U64, _U64, _P, _P, _P]),
    ("krp_batch_planted_rows", _INT, [_P, _I64, _P, _P, _INT, C.c_float, _U64, _P]),
    ("krp_batch_solve_dense", _INT, [_P, _I64, _P, _P, _P, _INT, _P, _INT]),
    ("krp_batch_sync_status", _INT, [_P]),
    ("krp_batch_capture_begin", _INT, [_P]),
    ("krp_batch_capture_end", _INT, [_P, C.POINTER(_I64)]),
    ("krp_batch_replay", _INT, [_P]),
    ("krp_batch_set_tuning", _INT, [_P, _INT]),
    ("krp_batch_autotune", _INT, [_P, _I64, C.POINTER(_INT)]),
    ("krp_batch_last_error", C.c_char_p, [_P]),
]

_lib = None


def lib():
    """Load libkrpls.so (built by paper_2301_12584_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libkrpls.so not built ({LIB_PATH}); run paper_2301_12584_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class KrpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


class Sampler:
    """Owns a krp_sampler.  Mirrors krp_* calls one to one."""

    def __init__(self, I, R, F=0, precision=KRP_PREC_FP32, stream=None):
        L = lib()
        self._lib = L
        self.N = len(I)
        self.I = [int(x) for x in I]
        self.R = int(R)
        arr = (_I64 * self.N)(*self.I)
        h = _P()
        code = L.krp_create(C.byref(h), self.N, arr, self.R, int(F), int(precision), _P(_stream_ptr(stream)))
        if code != KRP_OK:
            raise KrpError(code, L.krp_last_error(None).decode())
        self.h = h

    def _check(self, code):
        if code != KRP_OK:
            raise KrpError(code, self._lib.krp_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self._lib.krp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- calls -----------------------------------------------------------
    def set_factor(self, j, U, precision=None):
        """U: device tensor or pinned/pageable host pointer (int) or CPU tensor."""
        if precision is None:
            self._check(self._lib.krp_set_factor(self.h, int(j), _P(_ptr(U))))
        else:
            self._check(self._lib.krp_set_factor_prec(self.h, int(j), _P(_ptr(U)), int(precision)))

    def sample(self, exclude_j, J, seed, draw_id, idx, weight, logq=None, SA=None):
        self._check(self._lib.krp_sample(self.h, int(exclude_j), int(J), int(seed), int(draw_id),
                                         _P(_ptr(idx)), _P(_ptr(weight)), _P(_ptr(logq)), _P(_ptr(SA))))

    def set_descent_form(self, form):
        """KRP_DESCENT_AUTO / _TEAM (team per sample), _NODE_MAJOR (batched node-major) or
        _NODE_MAJOR_TC (level-synchronous node-major, masses on the tensor cores), 32 < R <= 128."""
        self._check(self._lib.krp_set_descent_form(self.h, int(form)))

    def sample_prepare(self, exclude_j):
        self._check(self._lib.krp_sample_prepare(self.h, int(exclude_j)))

    def sample_draw(self, exclude_j, J, seed, draw_id, idx, weight, logq=None, SA=None):
        self._check(self._lib.krp_sample_draw(self.h, int(exclude_j), int(J), int(seed), int(draw_id),
                                              _P(_ptr(idx)), _P(_ptr(weight)), _P(_ptr(logq)), _P(_ptr(SA))))

    def debug_trace(self, exclude_j, J, seed, draw_id, idx, weight, trace, n_trace):
        self._check(self._lib.krp_debug_trace(self.h, int(exclude_j), int(J), int(seed), int(draw_id),
                                              _P(_ptr(idx)), _P(_ptr(weight)), _P(_ptr(trace)), int(n_trace)))

    def gather(self, exclude_j, J, idx, weight, SA):
        self._check(self._lib.krp_gather(self.h, int(exclude_j), int(J), _P(_ptr(idx)), _P(_ptr(weight)),
                                         _P(_ptr(SA))))

    def solve_dense(self, J, SA, weight, B_rows, nrhs, X, flags=0):
        self._check(self._lib.krp_solve_dense(self.h, int(J), _P(_ptr(SA)), _P(_ptr(weight)), _P(_ptr(B_rows)),
                                              int(nrhs), _P(_ptr(X)), int(flags)))

    def kron_rows(self, exclude_j, J, idx, cs, B_rows):
        """cs: list of N device vectors (None allowed for the excluded factor)."""
        arr = (_P * self.N)(*[_ptr(c) for c in cs])
        self._check(self._lib.krp_kron_rows(self.h, int(exclude_j), int(J), _P(_ptr(idx)), arr, _P(_ptr(B_rows))))

    def sketch_distortion(self, exclude_j, J, SA):
        """Returns (D, rank(A))."""
        D = C.c_double()
        r = _INT()
        self._check(self._lib.krp_sketch_distortion(self.h, int(exclude_j), int(J), _P(_ptr(SA)), C.byref(D),
                                                    C.byref(r)))
        return D.value, r.value

    def update_entries(self, j, rows, cols, values):
        """rows, cols: device int32 tensors; values: device float32 tensor (same length)."""
        n = int(rows.numel()) if hasattr(rows, "numel") else len(rows)
        self._check(self._lib.krp_update_entries(self.h, int(j), n, _P(_ptr(rows)), _P(_ptr(cols)),
                                                 _P(_ptr(values))))

    def capture_begin(self):
        self._check(self._lib.krp_capture_begin(self.h))

    def capture_end(self):
        n = _I64()
        self._check(self._lib.krp_capture_end(self.h, C.byref(n)))
        return n.value

    def replay(self):
        self._check(self._lib.krp_replay(self.h))

    def planted_rows(self, exclude_j, J, idx, X_true, nrhs, sigma, seed, B_rows):
        self._check(self._lib.krp_planted_rows(self.h, int(exclude_j), int(J), _P(_ptr(idx)), _P(_ptr(X_true)),
                                               int(nrhs), float(sigma), int(seed), _P(_ptr(B_rows))))

    def solve_sparse(self, tensor, j, J, idx, weight, SA, U_out, flags=KRP_PINV_FALLBACK):
        self._check(self._lib.krp_solve_sparse(self.h, tensor.h, int(j), int(J), _P(_ptr(idx)), _P(_ptr(weight)),
                                               _P(_ptr(SA)), _P(_ptr(U_out)), int(flags)))

    def cp_als_sweep(self, tensor, J, seed, draw_base, sigma):
        self._check(self._lib.krp_cp_als_sweep(self.h, tensor.h, int(J), int(seed), int(draw_base),
                                               _P(_ptr(sigma))))

    def cp_fit(self, tensor, sigma):
        out = C.c_double()
        self._check(self._lib.krp_cp_fit(self.h, tensor.h, _P(_ptr(sigma)), C.byref(out)))
        return out.value

    def debug_wait_timeout(self, tries):
        self._check(self._lib.krp_debug_wait_timeout(self.h, int(tries)))

    def sync_status(self):
        """Synchronise and return the device status code (0 = OK)."""
        return int(self._lib.krp_sync_status(self.h))

    def last_error(self):
        return self._lib.krp_last_error(self.h).decode()

    def tree_info(self, j):
        L, d, st = _I64(), _INT(), _INT()
        self._check(self._lib.krp_tree_info(self.h, int(j), C.byref(L), C.byref(d), C.byref(st)))
        return L.value, d.value, st.value

    def get_factor(self, j):
        """Host copy (numpy, I_j x R FP32) of the sampler's factor j."""
        import numpy as np
        out = np.zeros((self.I[j], self.R), dtype=np.float32)
        self._check(self._lib.krp_get_factor(self.h, int(j), out.ctypes.data_as(_P), out.size))
        return out

    def get_tree(self, j):
        import numpy as np
        L, _, st = self.tree_info(j)
        out = np.zeros(L * st, dtype=np.float32)
        self._check(self._lib.krp_get_tree(self.h, int(j), out.ctypes.data_as(_P), out.size))
        return out.reshape(L, st)

    def get_tree_exact(self, j):
        """Exact-decision samplers: (low parts shaped like get_tree, delta-encoded top)."""
        import numpy as np
        L, d, st = self.tree_info(j)
        ke = min(10, d)
        lo = np.zeros(L * st, dtype=np.float32)
        top = np.zeros((1 << ke) * st, dtype=np.float32)
        self._check(self._lib.krp_get_tree_exact(self.h, int(j), lo.ctypes.data_as(_P), lo.size,
                                                 top.ctypes.data_as(_P), top.size))
        return lo.reshape(L, st), top.reshape(1 << ke, st)

    def exact_count(self):
        """Row-stage descents switched to double-float masses so far (exact-decision samplers)."""
        n = _I64()
        self._check(self._lib.krp_exact_count(self.h, C.byref(n)))
        return n.value

    def get_prep(self, k):
        import numpy as np
        R = self.R
        lam = np.zeros(R)
        V = np.zeros((R, R))
        Gp = np.zeros((R, R))
        rank = _INT()
        self._check(self._lib.krp_get_prep(self.h, int(k), lam.ctypes.data_as(_P), V.ctypes.data_as(_P),
                                           Gp.ctypes.data_as(_P), C.byref(rank)))
        return lam, V, Gp, rank.value


def debug_sort_pairs(keys, vals, bits, stream=None):
    """krp_debug_sort_pairs on device uint32 tensors (given as int32 torch tensors)."""
    code = lib().krp_debug_sort_pairs(_P(_ptr(keys)), _P(_ptr(vals)), int(keys.numel()), int(bits),
                                      _P(_stream_ptr(stream)))
    if code != KRP_OK:
        raise KrpError(code, lib().krp_last_error(None).decode())


def launch_count():
    """Kernels launched by libkrpls in this process so far."""
    return int(lib().krp_launch_count())


def solve_dense_noalloc(J, R, SA, weight, B_rows, nrhs, X, status, flags=0, stream=None):
    """krp_solve_dense_noalloc: the dense solve with the library's fixed device
    scratch (R <= 32, nrhs <= 16); `status` is a device int32 the call clears
    and the kernels may raise.  Enqueues only; raises KrpError on a rejected call."""
    L = lib()
    rc = L.krp_solve_dense_noalloc(int(J), int(R), _P(_ptr(SA)), _P(_ptr(weight)), _P(_ptr(B_rows)), int(nrhs),
                                   _P(_ptr(X)), int(flags), _P(_ptr(status)), _P(_stream_ptr(stream)))
    if rc != 0:
        raise KrpError(rc, L.krp_last_error(None).decode())


class SparseTensor:
    """Owns a krp_sptensor built from host coordinates (N x nnz int32) and values."""

    def __init__(self, dims, coords, vals, stream=None):
        import numpy as np
        L = lib()
        self._lib = L
        coords = [np.ascontiguousarray(c, dtype=np.int32) for c in coords]
        vals = np.ascontiguousarray(vals, dtype=np.float32)
        self._keep = (coords, vals)
        N = len(dims)
        arr = (_I64 * N)(*[int(d) for d in dims])
        cptrs = (_P * N)(*[c.ctypes.data for c in coords])
        h = _P()
        code = L.krp_sptensor_create(C.byref(h), N, arr, int(vals.size), cptrs, _P(vals.ctypes.data),
                                     _P(_stream_ptr(stream)))
        if code != KRP_OK:
            raise KrpError(code, "krp_sptensor_create failed")
        self.h = h
        self._keep = None

    def close(self):
        if getattr(self, "h", None):
            self._lib.krp_sptensor_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns a krp_batch over existing Samplers (kept alive here).  Packed
    layouts as in include/krpls.h: problem p's SA rows and X start at row
    offset Roff[p] = sum of the earlier problems' R."""

    def __init__(self, samplers, stream):
        L = lib()
        self._lib = L
        self.samplers = list(samplers)
        self.P = len(self.samplers)
        self.N = self.samplers[0].N
        self.R = [s.R for s in self.samplers]
        self.row_off = [0]
        for r in self.R:
            self.row_off.append(self.row_off[-1] + r)
        arr = (_P * self.P)(*[s.h for s in self.samplers])
        h = _P()
        code = L.krp_batch_create(C.byref(h), arr, self.P, _P(_stream_ptr(stream)))
        if code != KRP_OK:
            raise KrpError(code, L.krp_last_error(None).decode())
        self.h = h

    def _check(self, code):
        if code != KRP_OK:
            raise KrpError(code, self._lib.krp_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self._lib.krp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_sources(self, U=None):
        """U: list of P*N device tensors/pointers (None entries: keep), or None."""
        if U is None:
            self._check(self._lib.krp_batch_set_sources(self.h, None))
            return
        arr = (_P * (self.P * self.N))(*[_ptr(u) for u in U])
        self._check(self._lib.krp_batch_set_sources(self.h, arr))

    def build(self):
        self._check(self._lib.krp_batch_build(self.h))

    def sample(self, J, seed, draw_id, idx, weight, SA=None):
        self._check(self._lib.krp_batch_sample(self.h, int(J), int(seed), int(draw_id), _P(_ptr(idx)),
                                               _P(_ptr(weight)), _P(_ptr(SA))))

    def planted_rows(self, J, idx, X_true, nrhs, sigma, seed, B_rows):
        self._check(self._lib.krp_batch_planted_rows(self.h, int(J), _P(_ptr(idx)), _P(_ptr(X_true)), int(nrhs),
                                                     float(sigma), int(seed), _P(_ptr(B_rows))))

    def solve_dense(self, J, SA, weight, B_rows, nrhs, X, flags=0):
        self._check(self._lib.krp_batch_solve_dense(self.h, int(J), _P(_ptr(SA)), _P(_ptr(weight)),
                                                    _P(_ptr(B_rows)), int(nrhs), _P(_ptr(X)), int(flags)))

    def sync_status(self):
        return int(self._lib.krp_batch_sync_status(self.h))

    def kron_rows(self, exclude_j, J, idx, cs, B_rows):
        """cs: list of N device vectors (None allowed for the excluded factor)."""
        arr = (_P * self.N)(*[_ptr(c) for c in cs])
        self._check(self._lib.krp_kron_rows(self.h, int(exclude_j), int(J), _P(_ptr(idx)), arr, _P(_ptr(B_rows))))

    def sketch_distortion(self, exclude_j, J, SA):
        """Returns (D, rank(A))."""
        D = C.c_double()
        r = _INT()
        self._check(self._lib.krp_sketch_distortion(self.h, int(exclude_j), int(J), _P(_ptr(SA)), C.byref(D),
                                                    C.byref(r)))
        return D.value, r.value

    def update_entries(self, j, rows, cols, values):
        """rows, cols: device int32 tensors; values: device float32 tensor (same length)."""
        n = int(rows.numel()) if hasattr(rows, "numel") else len(rows)
        self._check(self._lib.krp_update_entries(self.h, int(j), n, _P(_ptr(rows)), _P(_ptr(cols)),
                                                 _P(_ptr(values))))

    def capture_begin(self):
        self._check(self._lib.krp_batch_capture_begin(self.h))

    def capture_end(self):
        n = _I64()
        self._check(self._lib.krp_batch_capture_end(self.h, C.byref(n)))
        return n.value

    def replay(self):
        self._check(self._lib.krp_batch_replay(self.h))

    def set_tuning(self, descent_ctas_per_problem):
        self._check(self._lib.krp_batch_set_tuning(self.h, int(descent_ctas_per_problem)))

    def autotune(self, J):
        best = _INT()
        self._check(self._lib.krp_batch_autotune(self.h, int(J), C.byref(best)))
        return best.value
