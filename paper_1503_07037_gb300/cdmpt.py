"""Thin ctypes binding of libcdmpt.so (include/cdmpt.h).

Argument marshalling only: every step of the computation runs in the CUDA
library. PyTorch provides device memory (output tensors) and the current
stream. The functions keep the C names without the ``cdmpt_`` prefix;
``Handle`` and ``solve`` wrap them for convenience.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcdmpt.so")

FP64, FP32, MIXED_TF32, MIXED_BF16 = 0, 1, 2, 3
GEMM_AUTO, GEMM_SIMT, GEMM_TC_TF32, GEMM_TC_3XTF32, GEMM_TC_BF16 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": FP64, "fp32": FP32, "mixed": MIXED_TF32, "mixed_tf32": MIXED_TF32,
              "mixed_bf16": MIXED_BF16}
ENGINES = {"auto": GEMM_AUTO, "simt": GEMM_SIMT, "tf32": GEMM_TC_TF32, "3xtf32": GEMM_TC_3XTF32,
           "bf16": GEMM_TC_BF16}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_RANGE", 3: "ERR_NO_CONVERGENCE", 4: "ERR_CG_MAXITER",
          5: "ERR_TIMEOUT", 6: "ERR_CUDA", 7: "ERR_OOM", 8: "ERR_UNSUPPORTED"}


class CdmptError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("gemm_engine", ctypes.c_int),
        ("cg_tol", ctypes.c_double),
        ("cg_maxit", ctypes.c_int),
        ("refine_rounds", ctypes.c_int),
        ("occ_tol", ctypes.c_double),
        ("mu_maxit", ctypes.c_int),
        ("have_mu_guess", ctypes.c_int),
        ("mu_guess", ctypes.c_double),
        ("profile", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("grand_canonical", ctypes.c_int),
        ("ckpt_stride", ctypes.c_int),
        ("fd_exact", ctypes.c_int),
        ("screen_tau", ctypes.c_double),
        ("fp64_residual", ctypes.c_int),
    ]


class SccModel(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_void_p),
        ("q0", ctypes.c_void_p),
        ("tol", ctypes.c_double),
        ("maxit", ctypes.c_int),
        ("history", ctypes.c_int),
        ("mix", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int), ("D", ctypes.c_int), ("n", ctypes.c_int),
        ("mu_iterations", ctypes.c_int),
        ("cg_iterations_sweeps", ctypes.c_int),
        ("cg_iterations_last_sweep", ctypes.c_int),
        ("cg_iterations_response", ctypes.c_int),
        ("cg_iterations_q", ctypes.c_int),
        ("cg_iterations_refine", ctypes.c_int),
        ("gemm_launches", ctypes.c_int),
        ("kernel_launches", ctypes.c_int),
        ("gemm_flops", ctypes.c_double),
        ("tensor_flops", ctypes.c_double),
        ("gemm_ms", ctypes.c_double),
        ("gemm_timed", ctypes.c_int),
        ("mu", ctypes.c_double), ("trace_P0", ctypes.c_double), ("trace_Q", ctypes.c_double),
        ("occupation_error", ctypes.c_double),
        ("seconds", ctypes.c_double),
        ("engine_ms", ctypes.c_double * 6),
        ("engine_launches", ctypes.c_int * 6),
        ("engine_flops", ctypes.c_double * 6),
        ("cg_iterations_recompute", ctypes.c_int),
        ("checkpoint_stride", ctypes.c_int),
        ("screen_slices_computed", ctypes.c_double),
        ("screen_slices_examined", ctypes.c_double),
        ("fp64_residual_passes", ctypes.c_int),
        ("fp64_residual_first_step", ctypes.c_int),
        ("refine_passes", ctypes.c_int),
        ("phase_ms", ctypes.c_double * 5),
    ]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if hasattr(v, "__len__") else v
        return d


_lib = None
EXPORTS = ["cdmpt_version", "cdmpt_default_opts", "cdmpt_create", "cdmpt_set_opts", "cdmpt_set_H",
           "cdmpt_solve", "cdmpt_polarizability", "cdmpt_get_stats", "cdmpt_last_error",
           "cdmpt_destroy", "cdmpt_gemm_f32", "cdmpt_gemm_f64", "cdmpt_spectral_bounds",
           "cdmpt_spectral_bounds_noalloc", "cdmpt_vjp_P0", "cdmpt_batch_create",
           "cdmpt_batch_set_H", "cdmpt_batch_solve", "cdmpt_batch_get_stats",
           "cdmpt_batch_last_error", "cdmpt_batch_destroy", "cdmpt_split_tf32",
           "cdmpt_gemm_f32_split", "cdmpt_response2", "cdmpt_batch_get_tuning",
           "cdmpt_response3", "cdmpt_free_energy", "cdmpt_set_overlap",
           "cdmpt_get_overlap_info", "cdmpt_scc_solve", "cdmpt_response1",
           "cdmpt_set_H_orders", "cdmpt_scc_solve2", "cdmpt_gemm_pair",
           "cdmpt_check_bounded_wait", "cdmpt_gemm_f64_tc"]


def lib() -> ctypes.CDLL:
    """Load libcdmpt.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_1503_07037_gb300.build` (nvcc, sm_103a)")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    sig = {
        "cdmpt_version": (I, []),
        "cdmpt_default_opts": (I, [ctypes.POINTER(Opts)]),
        "cdmpt_create": (I, [ctypes.POINTER(Opts), ctypes.POINTER(P)]),
        "cdmpt_set_opts": (I, [P, ctypes.POINTER(Opts)]),
        "cdmpt_set_H": (I, [P, I, P, I, P, I]),
        "cdmpt_solve": (I, [P, D, D, I, P, P, P, P, I]),
        "cdmpt_polarizability": (I, [P, P]),
        "cdmpt_get_stats": (I, [P, ctypes.POINTER(Stats)]),
        "cdmpt_last_error": (ctypes.c_char_p, [P]),
        "cdmpt_destroy": (V, [P]),
        "cdmpt_gemm_f32": (I, [I, I, I, I, P, I, P, I, P, I, D, D, P, I, D, I, I, P, P, I, P]),
        "cdmpt_gemm_f64": (I, [I, I, I, P, I, P, I, P, I, D, D, P, I, D, I, I, P, P, I, P]),
        "cdmpt_gemm_f64_tc": (I, [I, I, I, P, I, P, I, P, I, D, D, P, I, D, I, I, P, P, I, P]),
        "cdmpt_spectral_bounds": (I, [P, I, I, P, P]),
        "cdmpt_spectral_bounds_noalloc": (I, [P, I, I, P, P]),
        "cdmpt_vjp_P0": (I, [P, P, P, I]),
        "cdmpt_response2": (I, [P, P, P, P, P, P, I]),
        "cdmpt_response3": (I, [P, P, P, P, I]),
        "cdmpt_response1": (I, [P, I, P, P, P, P, P, I]),
        "cdmpt_set_H_orders": (I, [P, P, P, I]),
        "cdmpt_free_energy": (I, [P, P, P, I]),
        "cdmpt_set_overlap": (I, [P, I, P, I]),
        "cdmpt_get_overlap_info": (I, [P, P, P]),
        "cdmpt_scc_solve": (I, [P, ctypes.POINTER(SccModel), I, P, I, P, D, D, I, P, P, P, P, P, P,
                                P, I]),
        "cdmpt_scc_solve2": (I, [P, ctypes.POINTER(SccModel), I, P, I, P, D, D, I, P, P, P, P, P,
                                 P, P, P, P, P, I]),
        "cdmpt_batch_get_tuning": (I, [P, P, P, P]),
        "cdmpt_batch_create": (I, [ctypes.POINTER(Opts), I, P, I, ctypes.POINTER(P)]),
        "cdmpt_batch_set_H": (I, [P, P, P, I, I]),
        "cdmpt_batch_solve": (I, [P, P, P, I, P, P, P, P, P, I]),
        "cdmpt_batch_get_stats": (I, [P, ctypes.POINTER(Stats)]),
        "cdmpt_batch_last_error": (ctypes.c_char_p, [P]),
        "cdmpt_batch_destroy": (V, [P]),
        "cdmpt_split_tf32": (I, [P, ctypes.c_size_t, P, P, P]),
        "cdmpt_gemm_f32_split": (I, [I, I, I, I, P, P, I, P, P, I, P, I, D, D, P, I, D, I, I, P, P, I,
                                     P]),
        "cdmpt_gemm_pair": (I, [I, I, I, P, P, I, P, P, I, P, P, I, D, D, P, P, D, P, P, I, I, P]),
        "cdmpt_check_bounded_wait": (I, [D, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int, h=None):
    if status != 0:
        msg = lib().cdmpt_last_error(h)
        raise CdmptError(status, msg.decode() if msg else "")


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream_ptr(stream):
    import torch
    if stream is None:
        if not torch.cuda.is_available():
            return 0
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------- C-named wrappers

def version() -> int:
    return lib().cdmpt_version()


def default_opts() -> Opts:
    o = Opts()
    _check(lib().cdmpt_default_opts(ctypes.byref(o)))
    return o


def create(opts: Opts) -> int:
    h = ctypes.c_void_p()
    _check(lib().cdmpt_create(ctypes.byref(opts), ctypes.byref(h)))
    return h.value


def set_opts(h: int, opts: Opts):
    _check(lib().cdmpt_set_opts(h, ctypes.byref(opts)), h)


def set_H(h: int, N: int, H0_ptr: int, D: int, H1_ptr: Optional[int], on_device: int):
    _check(lib().cdmpt_set_H(h, N, H0_ptr, D, H1_ptr, on_device), h)


def solve_raw(h: int, beta, nocc, n, P0_ptr, P1_ptr, mu_ptr, mu1_ptr, out_on_device: int):
    _check(lib().cdmpt_solve(h, float(beta), float(nocc), int(n), P0_ptr, P1_ptr, mu_ptr,
                             mu1_ptr, out_on_device), h)


def polarizability(h: int, D: int) -> np.ndarray:
    a = np.zeros(max(D, 1))
    _check(lib().cdmpt_polarizability(h, a.ctypes.data), h)
    return a[:D]


def get_stats(h: int) -> dict:
    s = Stats()
    _check(lib().cdmpt_get_stats(h, ctypes.byref(s)), h)
    return s.as_dict()


def last_error(h: int) -> str:
    m = lib().cdmpt_last_error(h)
    return m.decode() if m else ""


def destroy(h: int):
    lib().cdmpt_destroy(h)


def gemm_f32(X, Y, D, alpha=1.0, beta=0.0, C=None, gamma=0.0, diag_block=0, trans_block=0,
             dot=None, E=None, engine="auto", M=None, Ncols=None, K=None, stream=None):
    """D = alpha X Y^T + beta C + gamma I on torch CUDA float32 tensors (row-major)."""
    M = X.shape[0] if M is None else M
    K = X.shape[1] if K is None else K
    Ncols = Y.shape[0] if Ncols is None else Ncols
    eng = ENGINES[engine] if isinstance(engine, str) else int(engine)
    _check(lib().cdmpt_gemm_f32(eng, M, Ncols, K, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0),
                                _ptr(D), D.stride(0), float(alpha), float(beta), _ptr(C),
                                C.stride(0) if C is not None else 0, float(gamma), diag_block,
                                trans_block, _ptr(dot), _ptr(E),
                                E.stride(0) if E is not None else 0, _stream_ptr(stream)))


def split_tf32(X, hi=None, lo=None, stream=None):
    """TF32 hi/lo split of a contiguous float32 CUDA tensor (returns (hi, lo))."""
    import torch
    hi = torch.empty_like(X) if hi is None else hi
    lo = torch.empty_like(X) if lo is None else lo
    _check(lib().cdmpt_split_tf32(_ptr(X), X.numel(), _ptr(hi), _ptr(lo), _stream_ptr(stream)))
    return hi, lo


def gemm_f32_split(Xs, Ys, D, alpha=1.0, beta=0.0, C=None, gamma=0.0, engine="3xtf32", M=None,
                   Ncols=None, K=None, dot=None, E=None, stream=None):
    """gemm_f32 on pre-split operands Xs = (hi, lo), Ys = (hi, lo); dot (a float64 CUDA
    tensor) receives += sum(D * E), or sum(D * D) without E."""
    Xh, Xl = Xs
    Yh, Yl = Ys
    M = Xh.shape[0] if M is None else M
    K = Xh.shape[1] if K is None else K
    Ncols = Yh.shape[0] if Ncols is None else Ncols
    eng = ENGINES[engine] if isinstance(engine, str) else int(engine)
    _check(lib().cdmpt_gemm_f32_split(eng, M, Ncols, K, _ptr(Xh), _ptr(Xl), Xh.stride(0),
                                      _ptr(Yh), _ptr(Yl), Yh.stride(0), _ptr(D), D.stride(0),
                                      float(alpha), float(beta), _ptr(C),
                                      C.stride(0) if C is not None else 0, float(gamma), 0, 0,
                                      _ptr(dot), _ptr(E), E.stride(0) if E is not None else 0,
                                      _stream_ptr(stream)))


def gemm_pair(Xh, Xl, Yh, Yl, D, Dl=None, alpha=1.0, b1=0.0, C1=(None, None), b2=0.0,
              C2=(None, None), K=None, sym=False, stream=None):
    """Ozaki-sliced product of pair-stored FP32 matrices (cdmpt_gemm_pair):
    D (+ Dl) = alpha (Xh + Xl)(Yh + Yl)^T + b1 C1 + b2 C2 with C1, C2 given as (hi, lo)
    pairs. All tensors are float32 CUDA tensors with row strides that are multiples of 8;
    any low part may be None. alpha, b1, b2 are powers of two or zero. sym: Y is X and the
    result symmetric, computed on the upper-triangle tiles and mirrored."""
    M, Ncols = Xh.shape[0], Yh.shape[0]
    K = Xh.shape[1] if K is None else K
    ldc = C1[0].stride(0) if C1[0] is not None else (C2[0].stride(0) if C2[0] is not None else D.stride(0))
    _check(lib().cdmpt_gemm_pair(M, Ncols, K, _ptr(Xh), _ptr(Xl), Xh.stride(0), _ptr(Yh), _ptr(Yl),
                                 Yh.stride(0), _ptr(D), _ptr(Dl), D.stride(0), float(alpha),
                                 float(b1), _ptr(C1[0]), _ptr(C1[1]), float(b2), _ptr(C2[0]),
                                 _ptr(C2[1]), ldc, 1 if sym else 0, _stream_ptr(stream)))


def check_bounded_wait(limit_ms=2.0, stream=None) -> int:
    """Runs cdmpt_check_bounded_wait and returns its status code (5 = ERR_TIMEOUT expected)."""
    return int(lib().cdmpt_check_bounded_wait(float(limit_ms), _stream_ptr(stream)))


def gemm_f64(X, Y, D, alpha=1.0, beta=0.0, C=None, gamma=0.0, diag_block=0, trans_block=0,
             dot=None, E=None, M=None, Ncols=None, K=None, stream=None, engine="simt"):
    """FP64 counterpart of gemm_f32: engine "simt" (cdmpt_gemm_f64, CUDA cores) or "tc"
    (cdmpt_gemm_f64_tc, the seven-digit Ozaki product on the tensor cores)."""
    M = X.shape[0] if M is None else M
    K = X.shape[1] if K is None else K
    Ncols = Y.shape[0] if Ncols is None else Ncols
    fn = lib().cdmpt_gemm_f64_tc if engine == "tc" else lib().cdmpt_gemm_f64
    _check(fn(M, Ncols, K, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0),
                                _ptr(D), D.stride(0), float(alpha), float(beta), _ptr(C),
                                C.stride(0) if C is not None else 0, float(gamma), diag_block,
                                trans_block, _ptr(dot), _ptr(E),
                                E.stride(0) if E is not None else 0, _stream_ptr(stream)))


def spectral_bounds(H, out=None, stream=None):
    """Gershgorin interval [lo, hi] of a symmetric torch CUDA float64 matrix H (2-element tensor)."""
    import torch
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=H.device)
    _check(lib().cdmpt_spectral_bounds(_ptr(H), H.shape[0], H.stride(0), _ptr(out),
                                       _stream_ptr(stream)))
    return out


def spectral_bounds_noalloc(H, out, stream=None):
    """spectral_bounds without any device allocation; `out` (2 float64 on the GPU) is required."""
    _check(lib().cdmpt_spectral_bounds_noalloc(_ptr(H), H.shape[0], H.stride(0), _ptr(out),
                                               _stream_ptr(stream)))
    return out


# ------------------------------------------------------------- convenience

class Handle:
    """Owns one cdmpt_handle. Inputs may be numpy arrays (host) or torch CUDA tensors."""

    def __init__(self, precision="fp32", engine="auto", cg_tol=0.0, cg_maxit=200,
                 refine_rounds=2, occ_tol=0.0, mu_maxit=60, mu_guess=None, profile=False,
                 stream=None, grand_canonical=False, ckpt_stride=0, fd_exact=False,
                 screen_tau=0.0, fp64_residual=0):
        """ckpt_stride: 0 stores the whole recursion trajectory; s > 0 keeps every s-th
        step and recomputes the rest segment by segment; "sqrt" (or -1) picks
        s = ceil(sqrt(n)). FP64 and FP32 precisions only. screen_tau > 0: block-sparse
        products that drop 128 x 32 tile terms with norm product <= screen_tau (FP32 and
        mixed TF32 only). fp64_residual (mixed only): 0 forms the final refinement pass's
        step residuals with Ozaki-sliced products on the late steps, 1 on every step, -1
        never."""
        o = default_opts()
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.gemm_engine = ENGINES[engine] if isinstance(engine, str) else int(engine)
        o.cg_tol = cg_tol
        o.cg_maxit = cg_maxit
        o.refine_rounds = refine_rounds
        o.occ_tol = occ_tol
        o.mu_maxit = mu_maxit
        o.have_mu_guess = 0 if mu_guess is None else 1
        o.mu_guess = 0.0 if mu_guess is None else float(mu_guess)
        o.profile = 1 if profile else 0
        o.stream = _stream_ptr(stream)
        o.grand_canonical = 1 if grand_canonical else 0
        o.ckpt_stride = -1 if ckpt_stride == "sqrt" else int(ckpt_stride)
        o.fd_exact = 1 if fd_exact else 0
        o.screen_tau = float(screen_tau)
        o.fp64_residual = int(fp64_residual)
        self.opts = o
        self.h = create(o)
        self.N = 0
        self.D = 0
        self._keep = None

    def set_overlap(self, S):
        """Non-orthogonal basis: S (N x N SPD; numpy or torch) or None for the orthogonal mode.
        Afterwards set_H takes F and h1, and the outputs are D = Z P_perp Z etc."""
        import torch
        if S is None:
            _check(lib().cdmpt_set_overlap(self.h, 0, None, 0), self.h)
            return
        if isinstance(S, torch.Tensor):
            Sc = S.detach().to(torch.float64).contiguous()
            _check(lib().cdmpt_set_overlap(self.h, Sc.shape[0], Sc.data_ptr(),
                                           1 if Sc.is_cuda else 0), self.h)
        else:
            Sc = np.ascontiguousarray(S, dtype=np.float64)
            _check(lib().cdmpt_set_overlap(self.h, Sc.shape[0], Sc.ctypes.data, 0), self.h)
        self.N = self.D = 0

    def overlap_info(self):
        """(Newton-Schulz iterations, final residual) of the last set_overlap."""
        it = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        _check(lib().cdmpt_get_overlap_info(self.h, ctypes.byref(it), ctypes.byref(res)), self.h)
        return it.value, res.value

    def set_H(self, H0, H1=None):
        import torch
        if H1 is None:
            D = 0
        else:
            D = 1 if H1.ndim == 2 else H1.shape[0]
        N = H0.shape[0]
        if isinstance(H0, torch.Tensor):
            H0c = H0.detach().to(torch.float64).contiguous()
            H1c = None if H1 is None else H1.detach().to(torch.float64).contiguous()
            on_dev = 1 if H0c.is_cuda else 0
            if on_dev and H1c is not None and not H1c.is_cuda:
                H1c = H1c.cuda()
            p0 = H0c.data_ptr()
            p1 = None if H1c is None else H1c.data_ptr()
            self._keep = (H0c, H1c)
        else:
            H0c = np.ascontiguousarray(H0, dtype=np.float64)
            H1c = None if H1 is None else np.ascontiguousarray(H1, dtype=np.float64)
            on_dev = 0
            p0 = H0c.ctypes.data
            p1 = None if H1c is None else H1c.ctypes.data
            self._keep = (H0c, H1c)
        set_H(self.h, N, p0, D, p1, on_dev)
        self._keep = None
        self.N, self.D = N, D

    def set_H_orders(self, H2=None, H3=None):
        """Higher perturbation terms H2, H3 ((D, N, N) numpy arrays, or None for zero) of
        H(lambda) = H0 + lambda H1 + lambda^2 H2 + lambda^3 H3, used by response2/3."""
        keep = []

        def ptr(A):
            if A is None:
                return None
            a = np.ascontiguousarray(A, dtype=np.float64)
            if a.ndim == 2:
                a = a[None]
            keep.append(a)
            return a.ctypes.data
        _check(lib().cdmpt_set_H_orders(self.h, ptr(H2), ptr(H3), 0), self.h)

    def solve(self, beta, nocc, n, want_P0=True, want_P1=True, device="cuda"):
        """Returns dict(P0, P1, mu, mu1) with P0/P1 float64 torch tensors on `device`."""
        import torch
        N, D = self.N, self.D
        dev = torch.device(device)
        on_dev = 1 if dev.type == "cuda" else 0
        P0 = torch.empty((N, N), dtype=torch.float64, device=dev) if want_P0 else None
        P1 = torch.empty((D, N, N), dtype=torch.float64, device=dev) if (want_P1 and D) else None
        mu = ctypes.c_double(0.0)
        mu1 = np.zeros(max(D, 1))
        solve_raw(self.h, beta, nocc, n, _ptr(P0), _ptr(P1), ctypes.addressof(mu),
                  mu1.ctypes.data, on_dev)
        return {"P0": P0, "P1": P1, "mu": mu.value, "mu1": mu1[:D].copy()}

    def polarizability(self):
        return polarizability(self.h, self.D)

    def vjp_P0(self, G0):
        """d Tr[G0 P0] / d H0 for the last solve (torch CUDA float64 in and out)."""
        import torch
        G = G0.detach().to(torch.float64).contiguous()
        out = torch.empty_like(G)
        _check(lib().cdmpt_vjp_P0(self.h, _ptr(G), _ptr(out), 1 if G.is_cuda else 0), self.h)
        return out

    def response1(self, H1, want_P1=True, device="cuda"):
        """First-order response of the last solve to new perturbations H1 ((D, N, N) or (N, N);
        numpy or torch) on the stored trajectory: dict(P1, mu1, omega2, alpha)."""
        import torch
        N = self.N
        if isinstance(H1, torch.Tensor):
            h = H1.detach().to(torch.float64).contiguous()
            if h.ndim == 2:
                h = h[None]
            on_in = 1 if h.is_cuda else 0
            ptr_in = h.data_ptr()
        else:
            h = np.ascontiguousarray(H1, dtype=np.float64)
            if h.ndim == 2:
                h = h[None]
            on_in = 0
            ptr_in = h.ctypes.data
        D = h.shape[0]
        dev = torch.device(device)
        if (dev.type == "cuda") != bool(on_in):   # one placement for inputs and outputs
            h = (torch.from_numpy(h) if not on_in else h.cpu()).to(dev).contiguous()
            ptr_in = h.data_ptr()
            on_in = 1 if dev.type == "cuda" else 0
        P1 = torch.empty((D, N, N), dtype=torch.float64, device=dev) if want_P1 else None
        mu1 = np.zeros(D)
        om2 = np.zeros(D)
        alpha = np.zeros(D)
        _check(lib().cdmpt_response1(self.h, D, ptr_in, _ptr(P1), mu1.ctypes.data,
                                     om2.ctypes.data, alpha.ctypes.data, on_in), self.h)
        return {"P1": P1, "mu1": mu1, "omega2": om2, "alpha": alpha}

    def response2(self, weights=None, want_P2=True, want_grad=True, device="cuda"):
        """Second-order canonical response of the last solve: dict(P2 (D, N, N), mu2 (D,),
        omega3 (D,), grad) with omega3 = 1/3 Tr[H1 P2] (Eq. Resp_0) and
        grad = d(sum_d w_d alpha_d)/dH0 = -4 sum_d w_d P2_d (float64 tensors)."""
        import torch
        N, D = self.N, self.D
        dev = torch.device(device)
        on_dev = 1 if dev.type == "cuda" else 0
        P2 = torch.empty((D, N, N), dtype=torch.float64, device=dev) if want_P2 else None
        G = torch.empty((N, N), dtype=torch.float64, device=dev) if want_grad else None
        w = None
        if weights is not None:
            w = np.ascontiguousarray(np.broadcast_to(np.asarray(weights, dtype=np.float64), (D,)))
        mu2 = np.zeros(max(D, 1))
        om3 = np.zeros(max(D, 1))
        _check(lib().cdmpt_response2(self.h, None if w is None else w.ctypes.data, _ptr(P2),
                                     mu2.ctypes.data, om3.ctypes.data, _ptr(G), on_dev), self.h)
        return {"P2": P2, "mu2": mu2[:D].copy(), "omega3": om3[:D].copy(), "grad": G}

    def response3(self, want_P3=True, device="cuda"):
        """Third-order canonical response of the last solve: dict(P3 (D, N, N), mu3 (D,),
        omega4 (D,)) with omega4 = 1/4 Tr[H1 P3] (Eq. Resp_0), float64 tensors."""
        import torch
        N, D = self.N, self.D
        dev = torch.device(device)
        on_dev = 1 if dev.type == "cuda" else 0
        P3 = torch.empty((D, N, N), dtype=torch.float64, device=dev) if want_P3 else None
        mu3 = np.zeros(max(D, 1))
        om4 = np.zeros(max(D, 1))
        _check(lib().cdmpt_response3(self.h, _ptr(P3), mu3.ctypes.data, om4.ctypes.data, on_dev),
               self.h)
        return {"P3": P3, "mu3": mu3[:D].copy(), "omega4": om4[:D].copy()}

    def free_energy(self, want_grad=True, device="cuda"):
        """Free energy of the last solve, Omega = Tr[P0 H0] - T_e S[P0] (Eqs. FreeE, SED), for
        the recursion's own P0: dict(omega, grad) with grad = dOmega/dH0 (float64 tensor)."""
        import torch
        N = self.N
        dev = torch.device(device)
        on_dev = 1 if dev.type == "cuda" else 0
        G = torch.empty((N, N), dtype=torch.float64, device=dev) if want_grad else None
        om = ctypes.c_double(0.0)
        _check(lib().cdmpt_free_energy(self.h, ctypes.addressof(om), _ptr(G), on_dev), self.h)
        return {"omega": om.value, "grad": G}

    def scc_solve(self, hcore, h1, gamma, beta, nocc, n, q0=None, tol=0.0, maxit=0, history=0,
                  mix=0.0, order=1):
        """Self-consistent charge solve and coupled-perturbed response (cdmpt_scc_solve) in
        the basis of the last set_overlap. Host (numpy) inputs and outputs: dict(D0, D1, mu,
        mu1, omega1, omega2, iters) with omega1 = 2 Tr[h1 D0], omega2 = Tr[h1 D1]; order=2
        adds D2, mu2 and omega3 = (2/3) Tr[h1 D2] (cdmpt_scc_solve2)."""
        hc = np.ascontiguousarray(hcore, dtype=np.float64)
        N = hc.shape[0]
        H1 = np.ascontiguousarray(np.zeros((0, N, N)) if h1 is None else h1, dtype=np.float64)
        if H1.ndim == 2:
            H1 = H1[None]
        D = H1.shape[0]
        g = np.ascontiguousarray(gamma, dtype=np.float64)
        q = None if q0 is None else np.ascontiguousarray(q0, dtype=np.float64)
        m = SccModel(g.ctypes.data, None if q is None else q.ctypes.data, tol, maxit, history, mix)
        D0 = np.empty((N, N))
        D1 = np.empty((max(D, 1), N, N))
        mu = ctypes.c_double(0.0)
        mu1, om1, om2 = np.zeros(max(D, 1)), np.zeros(max(D, 1)), np.zeros(max(D, 1))
        it = np.zeros(2, dtype=np.int32)
        D2 = np.empty((max(D, 1), N, N))
        mu2, om3 = np.zeros(max(D, 1)), np.zeros(max(D, 1))
        second = order >= 2 and D > 0
        _check(lib().cdmpt_scc_solve2(self.h, ctypes.byref(m), N, hc.ctypes.data, D,
                                      H1.ctypes.data if D else None, beta, nocc, n,
                                      D0.ctypes.data, D1.ctypes.data if D else None,
                                      ctypes.addressof(mu), mu1.ctypes.data, om1.ctypes.data,
                                      om2.ctypes.data, D2.ctypes.data if second else None,
                                      mu2.ctypes.data if second else None,
                                      om3.ctypes.data if second else None, it.ctypes.data, 0),
               self.h)
        self.N, self.D = N, 0
        out = {"D0": D0, "D1": D1[:D], "mu": mu.value, "mu1": mu1[:D].copy(),
               "omega1": om1[:D].copy(), "omega2": om2[:D].copy(),
               "iters": tuple(int(v) for v in it)}
        if second:
            out.update(D2=D2[:D], mu2=mu2[:D].copy(), omega3=om3[:D].copy())
        return out

    def stats(self):
        return get_stats(self.h)

    def close(self):
        if self.h:
            destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Batched canonical solves of uneven-size Hamiltonians (cdmpt_batch_*).

    B = Batch(sizes, D); B.set_H(H0_list, H1_list, n); r = B.solve(betas, noccs, n)
    returns dict(P0=[...], P1=[...], mu, mu1 (B x D), alpha (B x D)), P0/P1 as
    float64 torch CUDA tensors.
    """

    def __init__(self, sizes, D, stream=None, precision="fp32", **kw):
        o = default_opts()
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        for k, v in kw.items():
            setattr(o, k, v)
        o.stream = _stream_ptr(stream)
        self.sizes = [int(s) for s in sizes]
        self.D = int(D)
        arr = (ctypes.c_int * len(self.sizes))(*self.sizes)
        h = ctypes.c_void_p()
        self._err = lambda: (lib().cdmpt_batch_last_error(h) or b"").decode()
        st = lib().cdmpt_batch_create(ctypes.byref(o), len(self.sizes), arr, self.D,
                                      ctypes.byref(h))
        if st != 0:
            raise CdmptError(st, (lib().cdmpt_batch_last_error(None) or b"").decode())
        self.h = h.value
        self._keep = None

    def _check(self, st):
        if st != 0:
            m = lib().cdmpt_batch_last_error(self.h)
            raise CdmptError(st, m.decode() if m else "")

    def set_H(self, H0s, H1s, n):
        import torch
        H0t = [torch.as_tensor(np.ascontiguousarray(h), dtype=torch.float64).cuda() for h in H0s]
        H1t = [torch.as_tensor(np.ascontiguousarray(h), dtype=torch.float64).cuda() for h in H1s]
        P = ctypes.c_void_p
        a0 = (P * len(H0t))(*[t.data_ptr() for t in H0t])
        a1 = (P * len(H1t))(*[t.data_ptr() for t in H1t])
        self._check(lib().cdmpt_batch_set_H(self.h, a0, a1, int(n), 1))
        torch.cuda.synchronize()

    def solve(self, betas, noccs, n):
        import torch
        B, D = len(self.sizes), self.D
        P0 = [torch.empty((N, N), dtype=torch.float64, device="cuda") for N in self.sizes]
        P1 = [torch.empty((D, N, N), dtype=torch.float64, device="cuda") for N in self.sizes]
        P = ctypes.c_void_p
        a0 = (P * B)(*[t.data_ptr() for t in P0])
        a1 = (P * B)(*[t.data_ptr() for t in P1])
        be = np.ascontiguousarray(betas, dtype=np.float64)
        no = np.ascontiguousarray(noccs, dtype=np.float64)
        mu = np.zeros(B)
        mu1 = np.zeros(B * max(D, 1))
        al = np.zeros(B * max(D, 1))
        self._check(lib().cdmpt_batch_solve(self.h, be.ctypes.data, no.ctypes.data, int(n), a0, a1,
                                            mu.ctypes.data, mu1.ctypes.data, al.ctypes.data, 1))
        return {"P0": P0, "P1": P1, "mu": mu, "mu1": mu1[:B * D].reshape(B, D),
                "alpha": al[:B * D].reshape(B, D)}

    def tuning(self):
        """The tile autotuner's choice and timings, and whether CG iterations replay a graph."""
        tn = ctypes.c_int(0)
        ms = np.zeros(3)
        gr = ctypes.c_int(0)
        self._check(lib().cdmpt_batch_get_tuning(self.h, ctypes.addressof(tn), ms.ctypes.data,
                                                 ctypes.addressof(gr)))
        return {"tile_n": tn.value, "ms_128": float(ms[0]), "ms_64": float(ms[1]),
                "ms_256": float(ms[2]), "graphs": bool(gr.value)}

    def stats(self):
        s = Stats()
        self._check(lib().cdmpt_batch_get_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if self.h:
            lib().cdmpt_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DensityMatrix:
    """Differentiable canonical density matrix P0(H0) (torch.autograd).

    P0 = DensityMatrix.apply(H0, beta, nocc, n, handle) returns P0 for the
    symmetric CUDA float64 tensor H0; backward gives dL/dH0 through the
    hand-written adjoint of the recursion (cdmpt_vjp_P0). The handle keeps the
    trajectory of the forward solve, so call backward before the next solve on
    the same handle.
    """

    @staticmethod
    def apply(H0, beta, nocc, n, handle):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, H):
                handle.set_H(H.detach(), None)
                r = handle.solve(beta, nocc, n, want_P1=False)
                return r["P0"]

            @staticmethod
            def backward(ctx, G):
                return handle.vjp_P0(G)

        return _Fn.apply(H0)


class Polarizability:
    """Differentiable canonical polarizabilities alpha_d(H0) = -2 Tr(P1_d H1_d) (torch.autograd).

    alpha = Polarizability.apply(H0, H1, beta, nocc, n, handle) returns the (D,)
    tensor of alpha_d for the symmetric CUDA float64 tensor H0 and fixed
    perturbations H1 (D, N, N); backward gives dL/dH0 = sum_d (dL/dalpha_d)
    (-4 P2_d) through the second-order response (cdmpt_response2). Call
    backward before the next solve on the same handle.
    """

    @staticmethod
    def apply(H0, H1, beta, nocc, n, handle):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, H):
                handle.set_H(H.detach(), H1)
                handle.solve(beta, nocc, n, want_P0=False, want_P1=False)
                return torch.as_tensor(handle.polarizability(), dtype=torch.float64,
                                       device=H.device)

            @staticmethod
            def backward(ctx, g):
                w = g.detach().to(torch.float64).cpu().numpy()
                return handle.response2(weights=w, want_P2=False, device=g.device.type)["grad"]

        return _Fn.apply(H0)


class FreeEnergy:
    """Differentiable free energy Omega(H0) = Tr[P0 H0] - T_e S[P0] (torch.autograd).

    omega = FreeEnergy.apply(H0, beta, nocc, n, handle) returns the scalar free
    energy (Eqs. FreeE, SED) of the recursion's P0 for the symmetric CUDA
    float64 tensor H0; backward gives dL/dH0 = (dL/dOmega) dOmega/dH0 from
    cdmpt_free_energy (P0 plus one adjoint sweep). Call backward before the
    next solve on the same handle.
    """

    @staticmethod
    def apply(H0, beta, nocc, n, handle):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, H):
                handle.set_H(H.detach(), None)
                handle.solve(beta, nocc, n, want_P0=False, want_P1=False)
                r = handle.free_energy(want_grad=True, device=H.device.type)
                ctx.save_for_backward(r["grad"])
                return torch.tensor(r["omega"], dtype=torch.float64, device=H.device)

            @staticmethod
            def backward(ctx, g):
                (grad,) = ctx.saved_tensors
                return g * grad

        return _Fn.apply(H0)


def solve(H0, H1, beta, nocc, n, precision="fp32", **kw):
    """One-shot canonical solve: returns (P0, P1, mu, mu1) with P0/P1 on the GPU."""
    with Handle(precision=precision, **kw) as h:
        h.set_H(H0, H1)
        r = h.solve(beta, nocc, n)
        return r["P0"], r["P1"], r["mu"], r["mu1"]
