"""Python binding of the C ABI in include/sp2.h (argument marshalling only).

Every step of the purification runs in libsp2.so's CUDA kernels; this module only
passes torch/numpy buffer addresses and CUDA stream handles through ctypes.  If the
library has not been built the first call raises: there is no CPU fallback.

The functions keep the C names (sp2_create, sp2_run, sp2_run_host, sp2_get_info,
sp2_destroy); `Purifier` wraps one handle for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# SP2_LIB=debug selects the build with device-side bounds checks (libsp2_debug.so)
LIB_PATH = os.path.join(HERE, "libsp2_debug.so" if os.environ.get("SP2_LIB") == "debug" else "libsp2.so")

SP2_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA runtime error", 3: "non-finite value in F",
          4: "device-side wait timed out", 5: "out of device memory", 6: "no gap (F = cI)",
          7: "unsupported option", 8: "device-side bounds check failed (debug library)"}
STOP_ORDER, STOP_TRACE_GUARD, STOP_EXACT, STOP_CAP, STOP_SCHEDULE = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": 0, "mixed": 1, "bf16x6": 1, "bf16x3": 2, "fp16x3": 3, "tf32x3": 4}
MAX_ITER = 512


class SP2Error(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, 'unknown')} (status {code})")
        self.code = code


class sp2_opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("guard", ctypes.c_int32), ("qtilde", ctypes.c_double),
                ("corrections", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("refine_fp64", ctypes.c_int32), ("launch_mode", ctypes.c_int32),
                ("history", ctypes.c_int32), ("tile", ctypes.c_int32), ("norm", ctypes.c_int32),
                ("bsr_cuda_cores", ctypes.c_int32)]


class sp2_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_iter", ctypes.c_int32), ("stop_reason", ctypes.c_int32),
                ("hist_len", ctypes.c_int32), ("lambda_min", ctypes.c_double),
                ("lambda_max", ctypes.c_double), ("loop_ms", ctypes.c_double), ("v", ctypes.POINTER(ctypes.c_double)),
                ("trace", ctypes.POINTER(ctypes.c_double)), ("p", ctypes.POINTER(ctypes.c_uint8)),
                ("tile", ctypes.c_int32)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libsp2.so (built in-tree by paper_1507_02087_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_1507_02087_gb300.build` "
                               "(the SP2 path has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.sp2_default_opts.argtypes = [ctypes.POINTER(sp2_opts)]
        L.sp2_default_opts.restype = None
        L.sp2_create.argtypes = [i64, i64, i32, ctypes.POINTER(sp2_opts), ctypes.POINTER(vp)]
        L.sp2_create.restype = i32
        L.sp2_run.argtypes = [vp, vp, vp, vp]
        L.sp2_run.restype = i32
        L.sp2_run_host.argtypes = [vp, vp, vp, vp]
        L.sp2_run_host.restype = i32
        L.sp2_get_info.argtypes = [vp, ctypes.POINTER(sp2_info)]
        L.sp2_get_info.restype = i32
        L.sp2_destroy.argtypes = [vp]
        L.sp2_destroy.restype = None
        L.sp2_status_string.argtypes = [i32]
        L.sp2_status_string.restype = ctypes.c_char_p
        L.sp2_test_tc_gemm.argtypes = [vp, i32, i32, i32, i32, i32, i32, vp, vp]
        L.sp2_test_tc_gemm.restype = i32
        L.sp2_test_tc_gemm_ex.argtypes = [vp, i32, i32, i32, i32, i32, i32, i32, i32, vp, vp]
        L.sp2_test_tc_gemm_ex.restype = i32
        L.sp2_test_tc_timeout.argtypes = [vp, i32, i32, vp, vp]
        L.sp2_test_tc_timeout.restype = i32
        L.sp2_build_device_checks.argtypes = []
        L.sp2_build_device_checks.restype = i32
        L.sp2_test_tc_bounds.argtypes = [vp, i32, i32, i32, vp, vp]
        L.sp2_test_tc_bounds.restype = i32
        L.sp2_run_fp64_noalloc.argtypes = [vp, vp, i64, i64, vp, vp]
        L.sp2_run_fp64_noalloc.restype = i32
        L.sp2_set_homo_lumo.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.sp2_set_homo_lumo.restype = i32
        L.sp2_set_homo_lumo_batch.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double)]
        L.sp2_set_mcweeny.argtypes = [vp, i32, ctypes.c_double, ctypes.c_double]
        L.sp2_set_mcweeny.restype = i32
        L.sp2_set_homo_lumo_batch.restype = i32
        L.sp2_create_batch.argtypes = [i32, ctypes.POINTER(i64), ctypes.POINTER(i64), i32,
                                       ctypes.POINTER(sp2_opts), ctypes.POINTER(vp)]
        L.sp2_create_batch.restype = i32
        L.sp2_run_batch.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
        L.sp2_run_batch.restype = i32
        L.sp2_get_info_batch.argtypes = [vp, i32, ctypes.POINTER(sp2_info)]
        L.sp2_get_info_batch.restype = i32
        L.sp2_destroy_batch.argtypes = [vp]
        L.sp2_destroy_batch.restype = None
        L.sp2_create_bsr.argtypes = [i64, i64, ctypes.c_double, ctypes.POINTER(sp2_opts), ctypes.POINTER(vp)]
        L.sp2_create_bsr.restype = i32
        L.sp2_create_bsr_ex.argtypes = [i64, i64, ctypes.c_double, i32, ctypes.POINTER(sp2_opts),
                                        ctypes.POINTER(vp)]
        L.sp2_create_bsr_ex.restype = i32
        L.sp2_run_bsr.argtypes = [vp, vp, vp, vp, i64, vp, vp]
        L.sp2_run_bsr.restype = i32
        L.sp2_get_info_bsr.argtypes = [vp, ctypes.POINTER(sp2_info), ctypes.POINTER(i64)]
        L.sp2_get_info_bsr.restype = i32
        L.sp2_get_work_bsr.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                       ctypes.POINTER(ctypes.c_double)]
        L.sp2_get_work_bsr.restype = i32
        L.sp2_destroy_bsr.argtypes = [vp]
        L.sp2_destroy_bsr.restype = None
        L.sp2_test_bsr_keep.argtypes = [vp, i64, ctypes.c_double, i32, vp, vp]
        L.sp2_test_bsr_keep.restype = i32
        L.sp2_test_bsr_square_pattern.argtypes = [vp, i32, vp]
        L.sp2_test_bsr_square_pattern.restype = i32
        L.sp2_set_bounds_bsr.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.sp2_set_bounds_bsr.restype = i32
        L.sp2_set_homo_lumo_bsr.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.sp2_set_homo_lumo_bsr.restype = i32
        L.sp2_set_bounds_batch.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double)]
        L.sp2_set_bounds_batch.restype = i32
        L.sp2_set_bounds.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.sp2_set_bounds.restype = i32
        L.sp2_test_set_perturbation.argtypes = [vp, vp, i64]
        L.sp2_test_set_perturbation.restype = i32
        _lib = L
    return _lib


def _check(code: int, where: str):
    if code != SP2_OK:
        raise SP2Error(code, where)


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


TILES = {"auto": 0, "128": 1, "pair": 2}
PRODUCT_UNITS = {"tensor": 0, "cuda": 1}     # block-sparse handles: tensor-core or FP32 CUDA-core block products
NORMS = {"fro": 0, "mixed": 1, "spectral": 2}
HISTORY = {"auto": 0, "full": 1, "recompute": 2}


def _opts(max_iter, guard, qtilde, corrections, refine_steps, refine_fp64, launch_mode, history="auto",
          tile="auto", norm="fro", products="tensor"):
    if launch_mode is None:
        launch_mode = int(os.environ.get("SP2_LAUNCH_MODE", "0"))
    return sp2_opts(max_iter, 1 if guard else 0, qtilde, corrections, refine_steps, int(refine_fp64),
                    launch_mode, HISTORY[history], TILES[tile], NORMS[norm], PRODUCT_UNITS[products])


def sp2_create(N: int, nocc: int, precision: str = "fp64", *, max_iter: int = 200, guard: bool = True,
               qtilde: float = 1.8, corrections: int = 1, refine_steps: int = 2,
               refine_fp64: int = 0, launch_mode: int | None = None, history: str = "auto",
               tile: str = "auto", norm: str = "fro") -> int:
    """launch_mode None reads SP2_LAUNCH_MODE from the environment (default 0, the graph).
    history: "auto", "full" (keep every iterate) or "recompute" (low memory).
    tile: tensor-core tiles of the mixed path, "auto", "128" or "pair" (256 x 256 per SM pair)."""
    o = _opts(max_iter, guard, qtilde, corrections, refine_steps, refine_fp64, launch_mode, history, tile, norm)
    h = ctypes.c_void_p()
    _check(lib().sp2_create(N, nocc, PRECISIONS[precision], ctypes.byref(o), ctypes.byref(h)), "sp2_create")
    return h.value


def sp2_run(h: int, F, D, stream=None) -> None:
    """Enqueue F -> D (torch CUDA float64 tensors, contiguous N x N) on `stream`."""
    _check(lib().sp2_run(h, F.data_ptr(), D.data_ptr(), _stream_ptr(stream)), "sp2_run")


def sp2_run_host(h: int, F: np.ndarray, D: np.ndarray, stream=None) -> None:
    """Host buffers in and out (copies inside the call); returns when D is written."""
    _check(lib().sp2_run_host(h, F.ctypes.data, D.ctypes.data, _stream_ptr(stream)), "sp2_run_host")


def _bounds4(bounds):
    if bounds is None:
        return None
    b = [float(x) for x in bounds]
    if len(b) != 4:
        raise ValueError("bounds = (homo_out, homo_in, lumo_in, lumo_out)")
    return (ctypes.c_double * 4)(*b)


def sp2_set_homo_lumo(h: int, bounds) -> None:
    """SP2-ACC (Alg. 4/5) with homo/lumo bounds (homo_out, homo_in, lumo_in, lumo_out) for
    the handle's following runs; None returns to the trace-based expansion."""
    _check(lib().sp2_set_homo_lumo(h, _bounds4(bounds)), "sp2_set_homo_lumo")


def sp2_get_info(h: int) -> dict:
    info = sp2_info()
    _check(lib().sp2_get_info(h, ctypes.byref(info)), "sp2_get_info")
    return _info_dict(info)


def sp2_create_batch(Ns, noccs, precision: str = "mixed", *, max_iter: int = 200, guard: bool = True,
                     qtilde: float = 1.8, corrections: int = 1, refine_steps: int = 2,
                     refine_fp64: int = 0, launch_mode: int | None = None, history: str = "auto",
                     tile: str = "auto", norm: str = "fro") -> int:
    count = len(Ns)
    o = _opts(max_iter, guard, qtilde, corrections, refine_steps, refine_fp64, launch_mode, history, tile, norm)
    n_arr = (ctypes.c_int64 * count)(*Ns)
    o_arr = (ctypes.c_int64 * count)(*noccs)
    h = ctypes.c_void_p()
    _check(lib().sp2_create_batch(count, n_arr, o_arr, PRECISIONS[precision], ctypes.byref(o), ctypes.byref(h)),
           "sp2_create_batch")
    return h.value


def sp2_run_batch(hb: int, Fs, Ds, stream=None) -> None:
    """Enqueue every F_i -> D_i of the batch (torch CUDA float64 tensors)."""
    count = len(Fs)
    f_arr = (ctypes.c_void_p * count)(*[F.data_ptr() for F in Fs])
    d_arr = (ctypes.c_void_p * count)(*[D.data_ptr() for D in Ds])
    _check(lib().sp2_run_batch(hb, f_arr, d_arr, _stream_ptr(stream)), "sp2_run_batch")


def sp2_get_info_batch(hb: int, i: int) -> dict:
    info = sp2_info()
    _check(lib().sp2_get_info_batch(hb, i, ctypes.byref(info)), "sp2_get_info_batch")
    return _info_dict(info)


def sp2_destroy_batch(hb: int) -> None:
    if hb:
        lib().sp2_destroy_batch(hb)


def _info_dict(info) -> dict:
    n, hl = info.n_iter, info.hist_len
    return {
        "status": info.status,
        "n_iter": n,
        "stop_reason": info.stop_reason,
        "hist_len": hl,
        "lambda_min": info.lambda_min,
        "lambda_max": info.lambda_max,
        "loop_ms": info.loop_ms,
        "v": np.ctypeslib.as_array(info.v, shape=(MAX_ITER + 2,))[:hl].copy(),
        "trace": np.ctypeslib.as_array(info.trace, shape=(MAX_ITER + 2,))[:hl + 1].copy(),
        "p": np.ctypeslib.as_array(info.p, shape=(MAX_ITER + 2,))[:hl + 1].copy(),
        "tile": {0: None, 1: "128", 2: "pair"}.get(info.tile),
    }


def sp2_test_tc_gemm(arena, ld: int, nslots: int, a_slot: int, b_slot: int, upper: bool, out,
                     stream=None, tile: str = "auto", fmt: str = "bf16", lowprec: bool = False) -> None:
    """Tensor-core product C = A B^T over a piece arena (see include/sp2_testing.h).
    tile: "128" (128 x 128 per SM), "pair" (256 x 256 per SM pair) or "auto"; fmt "bf16"
    (three bf16 planes per slot), "fp16" (two fp16 planes of 2^14 x) or "tf32" (two FP32 planes
    holding tf32 values); lowprec: the format's low-precision product."""
    _check(lib().sp2_test_tc_gemm_ex(arena.data_ptr(), ld, nslots, a_slot, b_slot, 1 if upper else 0,
                                     TILES[tile], {"bf16": 0, "fp16": 1, "tf32": 2}[fmt], 1 if lowprec else 0,
                                     out.data_ptr(), _stream_ptr(stream)), "sp2_test_tc_gemm_ex")


def sp2_destroy(h: int) -> None:
    if h:
        lib().sp2_destroy(h)


TRUNC_RULES = {"block": 0, "error": 1, "mixed": 2}


class BsrPurifier:
    """Block-sparse F (32 x 32 blocks, BSR) -> D with block truncation tau.
    rule: "block" (drop blocks with norm below tau), "error" (||E||_F <= tau) or "mixed"
    (||E||_M <= tau); norm: "fro" (stop on v_i) or "mixed" (m_i with the 32 x 32 blocks);
    products: "tensor" (tcgen05 block products, default) or "cuda" (FP32 CUDA cores)."""

    def __init__(self, N: int, nocc: int, tau: float, max_iter: int = 200, guard: bool = True,
                 qtilde: float = 1.8, launch_mode: int | None = None, rule: str = "block", norm: str = "fro",
                 products: str = "tensor"):
        o = _opts(max_iter, guard, qtilde, 1, 0, False, launch_mode, norm=norm, products=products)
        h = ctypes.c_void_p()
        _check(lib().sp2_create_bsr_ex(N, nocc, tau, TRUNC_RULES[rule], ctypes.byref(o), ctypes.byref(h)),
               "sp2_create_bsr_ex")
        self.N, self.nocc, self.tau, self.rule, self.h = N, nocc, tau, rule, h.value

    def run(self, row_ptr, col_idx, vals, D=None, dense=True, stream=None):
        """row_ptr/col_idx: CUDA int32 tensors, vals: CUDA float64 [nnzb, 32, 32]."""
        import torch
        if dense and D is None:
            D = torch.empty(self.N, self.N, dtype=torch.float64, device=vals.device)
        _check(lib().sp2_run_bsr(self.h, row_ptr.data_ptr(), col_idx.data_ptr(), vals.data_ptr(),
                                 vals.shape[0], D.data_ptr() if D is not None else None, _stream_ptr(stream)),
               "sp2_run_bsr")
        return D

    def set_homo_lumo(self, bounds) -> None:
        """SP2-ACC with homo/lumo bounds (homo_out, homo_in, lumo_in, lumo_out); None: Alg. 3."""
        _check(lib().sp2_set_homo_lumo_bsr(self.h, _bounds4(bounds)), "sp2_set_homo_lumo_bsr")

    def set_bounds(self, bounds) -> None:
        """Outer spectral bounds (lambda_min, lambda_max) in place of Gershgorin's; None: Gershgorin."""
        arr = None if bounds is None else (ctypes.c_double * 2)(*[float(x) for x in bounds])
        _check(lib().sp2_set_bounds_bsr(self.h, arr), "sp2_set_bounds_bsr")

    def info(self) -> dict:
        info = sp2_info()
        nz = ctypes.c_int64()
        _check(lib().sp2_get_info_bsr(self.h, ctypes.byref(info), ctypes.byref(nz)), "sp2_get_info_bsr")
        d = _info_dict(info)
        d["nnzb"] = nz.value
        bp, up, sb, nms = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().sp2_get_work_bsr(self.h, ctypes.byref(bp), ctypes.byref(up), ctypes.byref(sb),
                                      ctypes.byref(nms)), "sp2_get_work_bsr")
        d["block_products"], d["needed_products"] = bp.value, up.value
        d["square_blocks"], d["numeric_ms"] = sb.value, nms.value
        return d

    def close(self):
        if self.h:
            lib().sp2_destroy_bsr(self.h)
        self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            if self.h:
                self.close()
        except Exception:
            pass


class BatchPurifier:
    """One batch handle: F_i (N_i x N_i) -> D_i for problems of uneven size."""

    def __init__(self, Ns, noccs, precision: str = "mixed", **opts):
        self.Ns, self.noccs, self.precision = list(Ns), list(noccs), precision
        self.h = sp2_create_batch(self.Ns, self.noccs, precision, **opts)

    def run(self, Fs, Ds=None, stream=None):
        import torch
        if len(Fs) != len(self.Ns):
            raise ValueError("one F per problem")
        for F, N in zip(Fs, self.Ns):
            if F.dtype != torch.float64 or not F.is_cuda or not F.is_contiguous() or F.shape != (N, N):
                raise ValueError("each F must be a contiguous CUDA float64 tensor of its problem's shape")
        if Ds is None:
            Ds = [torch.empty_like(F) for F in Fs]
        sp2_run_batch(self.h, Fs, Ds, stream)
        return Ds

    def info(self, i: int) -> dict:
        return sp2_get_info_batch(self.h, i)

    def set_homo_lumo(self, i: int, bounds) -> None:
        _check(lib().sp2_set_homo_lumo_batch(self.h, i, _bounds4(bounds)), "sp2_set_homo_lumo_batch")

    def set_bounds(self, i: int, bounds) -> None:
        """Outer spectral bounds (lambda_min, lambda_max) of problem i; None: Gershgorin."""
        arr = None if bounds is None else (ctypes.c_double * 2)(*[float(x) for x in bounds])
        _check(lib().sp2_set_bounds_batch(self.h, i, arr), "sp2_set_bounds_batch")

    def close(self):
        sp2_destroy_batch(self.h)
        self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            if self.h:
                self.close()
        except Exception:
            pass


class Purifier:
    """One handle: F (N x N, symmetric, float64) -> density matrix D."""

    def __init__(self, N: int, nocc: int, precision: str = "fp64", **opts):
        self.N, self.nocc, self.precision = N, nocc, precision
        self.h = sp2_create(N, nocc, precision, **opts)

    def run(self, F, D=None, stream=None):
        import torch
        if F.dtype != torch.float64 or not F.is_cuda or not F.is_contiguous() or F.shape != (self.N, self.N):
            raise ValueError("F must be a contiguous CUDA float64 tensor of shape (N, N)")
        if D is None:
            D = torch.empty_like(F)
        sp2_run(self.h, F, D, stream)
        return D

    def run_host(self, F: np.ndarray, D: np.ndarray | None = None, stream=None) -> np.ndarray:
        F = np.ascontiguousarray(F, dtype=np.float64)
        if D is None:
            D = np.empty_like(F)
        sp2_run_host(self.h, F, D, stream)
        return D

    def info(self) -> dict:
        return sp2_get_info(self.h)

    def set_homo_lumo(self, bounds) -> None:
        sp2_set_homo_lumo(self.h, bounds)

    def set_bounds(self, bounds) -> None:
        """Outer spectral bounds (lambda_min, lambda_max) for the scaling in place of the
        Gershgorin bounds; None returns to Gershgorin."""
        arr = None if bounds is None else (ctypes.c_double * 2)(*[float(x) for x in bounds])
        _check(lib().sp2_set_bounds(self.h, arr), "sp2_set_bounds")

    def set_perturbation(self, E) -> None:
        """Testing hook (Alg. 1): E is a contiguous CUDA float64 tensor (count, N, N); later runs
        add E[i] to X_i as it is formed.  The tensor is kept alive here; None switches it off."""
        import torch
        if E is None:
            _check(lib().sp2_test_set_perturbation(self.h, None, 0), "sp2_test_set_perturbation")
            self._pert = None
            return
        if E.dtype != torch.float64 or not E.is_cuda or not E.is_contiguous() or E.shape[1:] != (self.N, self.N):
            raise ValueError("E must be a contiguous CUDA float64 tensor of shape (count, N, N)")
        _check(lib().sp2_test_set_perturbation(self.h, E.data_ptr(), E.shape[0]), "sp2_test_set_perturbation")
        self._pert = E

    def set_mcweeny(self, mode: str | None, mu: float = 0.0, xi: float = 0.0) -> None:
        """McWeeny expansion on an FP64 handle: mode "mcw", "mcw-acc" (gap estimate xi) or None
        (back to SP2); mu is the chemical potential."""
        m = {None: 0, "mcw": 1, "mcw-acc": 2}[mode]
        _check(lib().sp2_set_mcweeny(self.h, m, float(mu), float(xi)), "sp2_set_mcweeny")

    def close(self):
        sp2_destroy(self.h)
        self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            if self.h:
                self.close()
        except Exception:
            pass
