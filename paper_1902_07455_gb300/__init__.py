"""Python binding of liblrfg (low-rank Fourier–Galerkin homogenisation on GB300).

Argument marshalling only: every step of the computation runs in the CUDA kernels of liblrfg.so,
called through its C ABI (include/lrfg.h).  PyTorch provides device memory (CUDA tensors whose
pointers are passed to the library) and the stream.  There is no CPU fallback: without the built
library or a CUDA device the calls raise.

Objects
-------
``Context``   a device, a stream and the library's device pool.
``TTensor``   a tensor train held as a list of CUDA float64 carriages (r_j, N_j, r_{j+1}).
``Problem``   a resident coefficient with the operator and the solvers for one format (FULL or TT).
``Field``     a library-owned operand or solution (FULL half spectrum or TT carriages).
``Batch``     the serving executor: worker threads with their own streams and contexts that run
              submitted solves concurrently, admitted by HBM footprint.
"""
from __future__ import annotations

import ctypes as C
import weakref
from dataclasses import dataclass

import numpy as np

from . import _lib as L

__all__ = ["Context", "TTensor", "TuckerTensor", "Problem", "Field", "Batch", "BatchResult", "LrfgError", "FULL", "TT", "TUCKER", "CP", "FP64", "MIXED", "GANI", "GA", "MUL_IDENTITY", "MUL_DERIV",
           "MUL_GAUSS", "library_path"]

FULL, CP, TUCKER, TT = L.LRFG_FULL, L.LRFG_CP, L.LRFG_TUCKER, L.LRFG_TT
FP64, MIXED = L.LRFG_FP64, L.LRFG_MIXED
GANI, GA = L.LRFG_GANI, L.LRFG_GA
MUL_IDENTITY, MUL_DERIV, MUL_GAUSS = L.LRFG_MUL_IDENTITY, L.LRFG_MUL_DERIV, L.LRFG_MUL_GAUSS


def library_path() -> str:
    return L.LIB_PATH


class LrfgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{L.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _torch():
    import torch
    return torch


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _ivec(vals, n):
    arr = (C.c_int * n)()
    for i, v in enumerate(vals):
        arr[i] = int(v)
    return arr


def _dvec(vals):
    vals = [float(v) for v in vals]
    return (C.c_double * len(vals))(*vals)


@dataclass
class TTensor:
    """Tensor train with CUDA float64 carriages of shapes (r_j, N_j, r_{j+1})."""
    cores: list

    @property
    def d(self):
        return len(self.cores)

    @property
    def shape(self):
        return tuple(int(c.shape[1]) for c in self.cores)

    @property
    def ranks(self):
        return [1] + [int(c.shape[2]) for c in self.cores[:-1]] + [1]

    def to_struct(self) -> L.lrfg_tt:
        s = L.lrfg_tt()
        s.d = self.d
        for j, c in enumerate(self.cores):
            if c.dtype != _torch().float64 or not c.is_cuda or not c.is_contiguous():
                raise ValueError("TT carriages must be contiguous CUDA float64 tensors")
            s.N[j] = int(c.shape[1])
            s.cores[j] = c.data_ptr()
        for j, r in enumerate(self.ranks):
            s.r[j] = r
        return s

    @staticmethod
    def from_numpy(cores, device="cuda"):
        torch = _torch()
        return TTensor([torch.as_tensor(np.ascontiguousarray(c, dtype=np.float64), device=device) for c in cores])

    def numpy(self):
        return [c.detach().cpu().numpy() for c in self.cores]


@dataclass
class TuckerTensor:
    """Tucker tensor with a CUDA float64 core (r_0, .., r_{d-1}) and factors of shapes (N_j, r_j)."""
    core: object
    factors: list

    @property
    def d(self):
        return len(self.factors)

    @property
    def shape(self):
        return tuple(int(f.shape[0]) for f in self.factors)

    @property
    def ranks(self):
        return [int(f.shape[1]) for f in self.factors]

    def to_struct(self) -> L.lrfg_tucker:
        torch = _torch()
        s = L.lrfg_tucker()
        s.d = self.d
        for t in [self.core] + list(self.factors):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
                raise ValueError("Tucker core and factors must be contiguous CUDA float64 tensors")
        s.core = self.core.data_ptr()
        for j, f in enumerate(self.factors):
            s.N[j] = int(f.shape[0])
            s.r[j] = int(f.shape[1])
            s.factors[j] = f.data_ptr()
        return s

    @staticmethod
    def from_numpy(core, factors, device="cuda"):
        torch = _torch()
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=device)
        return TuckerTensor(t(core), [t(f) for f in factors])

    def numpy(self):
        return self.core.detach().cpu().numpy(), [f.detach().cpu().numpy() for f in self.factors]


class Context:
    """A liblrfg context on one CUDA device.  ``stream``: a torch.cuda.Stream, or None for torch's current
    stream at creation; the library issues all its work there, so torch ops on the same stream see its
    results in order.  ``budget``: cap of the library's device pool in bytes, 0 = none."""

    def __init__(self, device: int = 0, stream=None, budget: int = 0):
        torch = _torch()
        self.lib = L.load()
        self.device = int(device)
        torch.cuda.set_device(self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.stream = s
        h = C.c_void_p()
        self._check(self.lib.lrfg_create(C.byref(h), self.device, C.c_void_p(s.cuda_stream), int(budget)), None)
        self.h = h
        self._children = weakref.WeakSet()

    def _check(self, st, h=None):
        if st != L.LRFG_OK:
            msg = self.lib.lrfg_last_error(h if h is not None else getattr(self, "h", None))
            raise LrfgError(st, (msg or b"").decode())
        return st

    def check(self, st):
        return self._check(st, self.h)

    def close(self):
        """Free every problem and field of this context, then the context."""
        if getattr(self, "h", None):
            for child in list(self._children):
                child.free()
            self.lib.lrfg_destroy(self.h)
            self.h = None

    def _adopt(self, obj):
        self._children.add(obj)
        return obj

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        self.check(self.lib.lrfg_sync(self.h))

    def launch_count(self) -> int:
        return int(self.lib.lrfg_launch_count(self.h))

    def profile(self, on: bool = True):
        """Enable/disable event timing of every launch (accounting of counts/flops/bytes is always on)."""
        self.check(self.lib.lrfg_profile_enable(self.h, int(bool(on))))

    def profile_reset(self):
        self.check(self.lib.lrfg_profile_reset(self.h))

    def profile_read(self) -> dict:
        """Per kernel class: launches, algorithmic flops and bytes, device ms (while profiling)."""
        n = self.lib.lrfg_profile_classes()
        L_ = (C.c_longlong * n)()
        f, b, m = (C.c_double * n)(), (C.c_double * n)(), (C.c_double * n)()
        self.check(self.lib.lrfg_profile_read(self.h, n, L_, f, b, m))
        return {self.lib.lrfg_profile_class_name(k).decode(): dict(launches=L_[k], flops=f[k], bytes=b[k], ms=m[k])
                for k in range(n)}

    def probe_fp64(self):
        """Measured FP64 rates of the device, TFLOP/s: (fused multiply-add pipe, mma.sync FP64)."""
        a, b = C.c_double(), C.c_double()
        self.check(self.lib.lrfg_probe_fp64(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def pool_bytes(self):
        a, b = C.c_size_t(), C.c_size_t()
        self.check(self.lib.lrfg_pool_bytes(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    # ---- fibre operators (rows a1, a2) ---------------------------------------------------------
    def fft_fibres(self, x, sign: int, out=None):
        """Batched DFT along dim 1 of a complex128 (FP64) or complex64 (FP32 arithmetic) CUDA tensor of
        shape (outer, N, inner)."""
        torch = _torch()
        if x.dtype not in (torch.complex128, torch.complex64) or x.dim() != 3:
            raise ValueError("x must be a complex128 or complex64 tensor (outer, N, inner)")
        x = x.contiguous()
        out = torch.empty_like(x) if out is None else out
        if out.dtype != x.dtype or out.shape != x.shape or not out.is_contiguous():
            raise ValueError("out must be a contiguous tensor of the input's shape and type")
        outer, N, inner = x.shape
        fn = self.lib.lrfg_fft_fibres if x.dtype == torch.complex128 else self.lib.lrfg_fft_fibres_f32
        self.check(fn(self.h, _ptr(x), _ptr(out), outer, N, inner, int(sign)))
        return out

    def fibre_operator(self, x, kind: int, param: float = 0.0, scale: float = 1.0, out=None):
        """scale * F^-1 diag(m) F along dim 1 of a real float64 CUDA tensor (outer, N, inner)."""
        torch = _torch()
        if x.dtype != torch.float64 or x.dim() != 3:
            raise ValueError("x must be a float64 tensor (outer, N, inner)")
        x = x.contiguous()
        out = torch.empty_like(x) if out is None else out
        outer, N, inner = x.shape
        self.check(self.lib.lrfg_fibre_operator(self.h, _ptr(x), _ptr(out), outer, N, inner, int(kind), float(param),
                                                float(scale)))
        return out

    def sym_eig(self, A, k: int):
        """k largest eigenpairs of a batch of symmetric float64 CUDA matrices (batch, n, n) or (n, n):
        (w (batch, k) descending, V (batch, n, k) orthonormal columns) — the eigensolver of the truncations."""
        torch = _torch()
        if A.dtype != torch.float64 or A.dim() not in (2, 3) or A.shape[-1] != A.shape[-2]:
            raise ValueError("A must be a float64 tensor (n, n) or (batch, n, n)")
        single = A.dim() == 2
        A = (A[None] if single else A).contiguous()
        b, n, _ = A.shape
        k = min(int(k), n)
        w = torch.empty((b, n), dtype=torch.float64, device=A.device)
        V = torch.empty((b, n, n), dtype=torch.float64, device=A.device)
        self.check(self.lib.lrfg_sym_eig(self.h, _ptr(A), n, k, b, _ptr(w), _ptr(V)))
        w, V = w[:, :k], V[:, :, :k]
        return (w[0], V[0]) if single else (w, V)

    # ---- TT operations (rows a3..a7) -------------------------------------------------------------
    def _alloc_tt(self, shape, ranks):
        torch = _torch()
        return [torch.empty((ranks[j], shape[j], ranks[j + 1]), dtype=torch.float64, device=f"cuda:{self.device}")
                for j in range(len(shape))]

    @staticmethod
    def _shrink(bufs, s: L.lrfg_tt) -> TTensor:
        cores = []
        for j, b in enumerate(bufs):
            n = s.r[j] * s.N[j] * s.r[j + 1]
            cores.append(b.view(-1)[:n].view(s.r[j], s.N[j], s.r[j + 1]))
        return TTensor(cores)

    def _tt_out(self, shape, cap_ranks):
        bufs = self._alloc_tt(shape, cap_ranks)
        s = L.lrfg_tt()
        s.d = len(shape)
        for j, b in enumerate(bufs):
            s.cores[j] = b.data_ptr()
        return bufs, s

    def tt_hadamard(self, x: TTensor, y: TTensor) -> TTensor:
        cap = [a * b for a, b in zip(x.ranks, y.ranks)]
        bufs, s = self._tt_out(x.shape, cap)
        xs, ys = x.to_struct(), y.to_struct()
        self.check(self.lib.lrfg_tt_hadamard(self.h, C.byref(xs), C.byref(ys), C.byref(s)))
        return self._shrink(bufs, s)

    def tt_add(self, alpha: float, x: TTensor, beta: float, y: TTensor) -> TTensor:
        d = x.d
        cap = [1] + [a + b for a, b in zip(x.ranks[1:d], y.ranks[1:d])] + [1]
        bufs, s = self._tt_out(x.shape, cap)
        xs, ys = x.to_struct(), y.to_struct()
        self.check(self.lib.lrfg_tt_add(self.h, float(alpha), C.byref(xs), float(beta), C.byref(ys), C.byref(s)))
        return self._shrink(bufs, s)

    def tt_round(self, x: TTensor, rmax: int, tol: float = 0.0) -> TTensor:
        """TT rounding to rank rmax, or with tol > 0 to the smallest ranks <= rmax within tol."""
        cap = [min(int(rmax), r) for r in x.ranks]
        bufs, s = self._tt_out(x.shape, cap)
        xs = x.to_struct()
        self.check(self.lib.lrfg_tt_round_tol(self.h, C.byref(xs), int(rmax), float(tol), C.byref(s)))
        return self._shrink(bufs, s)

    def tt_round_sketch(self, x: TTensor, ell: int, seed: int, rmax: int, tol: float = 0.0) -> TTensor:
        """Randomised truncation (lrfg_tt_round_sketch): sketch of inner ranks ``ell`` from SplitMix64 stream
        ``seed``, then the deterministic rounding to rank rmax (tol > 0: within tol)."""
        cap = [1] + [int(rmax)] * (x.d - 1) + [1]
        bufs, s = self._tt_out(x.shape, cap)
        xs = x.to_struct()
        self.check(self.lib.lrfg_tt_round_sketch(self.h, C.byref(xs), int(ell), int(seed), int(rmax), float(tol),
                                                 C.byref(s)))
        return self._shrink(bufs, s)

    def tt_hadamard_round_sketch(self, x: TTensor, y: TTensor, ell: int, seed: int, rmax: int,
                                 tol: float = 0.0) -> TTensor:
        """The randomised truncation of x (.) y without forming the product (lrfg_tt_hadamard_round_sketch)."""
        cap = [1] + [int(rmax)] * (x.d - 1) + [1]
        bufs, s = self._tt_out(x.shape, cap)
        xs, ys = x.to_struct(), y.to_struct()
        self.check(self.lib.lrfg_tt_hadamard_round_sketch(self.h, C.byref(xs), C.byref(ys), int(ell), int(seed),
                                                          int(rmax), float(tol), C.byref(s)))
        return self._shrink(bufs, s)

    def tt_dot(self, x: TTensor, y: TTensor) -> float:
        out = C.c_double()
        xs, ys = x.to_struct(), y.to_struct()
        self.check(self.lib.lrfg_tt_dot(self.h, C.byref(xs), C.byref(ys), C.byref(out)))
        return out.value

    def tt_dot_noalloc(self, x: TTensor, y: TTensor, out):
        """<x, y> into the CUDA float64 tensor ``out`` (one element) without any device allocation by the
        library: for callers that cannot allocate at that point (an application-owned allocator, loops that
        must not wait on the driver's allocator).  Asynchronous on the context's stream; intermediates live
        in a fixed 4 MiB device array shared by all calls."""
        torch = _torch()
        if out.dtype != torch.float64 or not out.is_cuda or out.numel() < 1:
            raise ValueError("out must be a CUDA float64 tensor with at least one element")
        xs, ys = x.to_struct(), y.to_struct()
        self.check(self.lib.lrfg_tt_dot_noalloc(self.h, C.byref(xs), C.byref(ys), _ptr(out)))
        return out

    def tt_precond(self, x: TTensor, pinv_eps: float, rmax: int) -> TTensor:
        cap = [1] + [int(rmax)] * (x.d - 1) + [1]
        bufs, s = self._tt_out(x.shape, cap)
        xs = x.to_struct()
        self.check(self.lib.lrfg_tt_precond(self.h, C.byref(xs), float(pinv_eps), int(rmax), C.byref(s)))
        return self._shrink(bufs, s)

    def tt_compress(self, values, rmax: int, tol: float = 0.0) -> TTensor:
        torch = _torch()
        values = values.contiguous()
        if values.dtype != torch.float64 or not values.is_cuda:
            raise ValueError("values must be a CUDA float64 tensor")
        shape = tuple(values.shape)
        cap = [1] + [int(rmax)] * (len(shape) - 1) + [1]
        bufs, s = self._tt_out(shape, cap)
        self.check(self.lib.lrfg_tt_compress(self.h, len(shape), _ivec(shape, 3), _ptr(values), int(rmax), float(tol),
                                             C.byref(s)))
        return self._shrink(bufs, s)

    def tt_expand(self, x: TTensor):
        torch = _torch()
        out = torch.empty(x.shape, dtype=torch.float64, device=f"cuda:{self.device}")
        xs = x.to_struct()
        self.check(self.lib.lrfg_tt_expand(self.h, C.byref(xs), _ptr(out)))
        return out

    def tucker_round(self, x: TuckerTensor, rmax: int, tol: float = 0.0) -> TuckerTensor:
        """Tucker truncation to ranks rmax, or with tol > 0 to the smallest ranks <= rmax within tol."""
        torch = _torch()
        k = [min(int(rmax), r) for r in x.ranks]
        dev = f"cuda:{self.device}"
        core = torch.empty(tuple(k), dtype=torch.float64, device=dev)
        facs = [torch.empty((n, kk), dtype=torch.float64, device=dev) for n, kk in zip(x.shape, k)]
        out = TuckerTensor(core, facs).to_struct()
        xs = x.to_struct()
        self.check(self.lib.lrfg_tucker_round_tol(self.h, C.byref(xs), int(rmax), float(tol), C.byref(out)))
        r = [int(out.r[j]) for j in range(x.d)]
        core = core.reshape(-1)[: int(np.prod(r))].reshape(tuple(r))
        facs = [f.reshape(-1)[: n * rj].reshape(n, rj) for f, n, rj in zip(facs, x.shape, r)]
        return TuckerTensor(core, facs)

    def field_from_tucker(self, x: TuckerTensor) -> "Field":
        h = C.c_void_p()
        xs = x.to_struct()
        self.check(self.lib.lrfg_field_from_tucker(self.h, C.byref(xs), 1, C.byref(h)))
        return Field(self, h)

    # ---- problems and fields ---------------------------------------------------------------------
    def problem(self, coeff, fmt: int, rank: int = 10, pinv_eps: float = 0.1, tol: float = 1e-8, maxit: int = 200,
                stop_on_increase: bool = True, prec: int = L.LRFG_FP64, rank_tol: float = 0.0,
                coeff_rank: int = 0, rank_start: int = 0, rank_step: int = 1, B=None,
                disc: int = L.LRFG_GANI, sketch_over: int = 0, sketch_seed: int = 0,
                sketch_keep: bool = False) -> "Problem":
        """``prec``: LRFG_FP64, or LRFG_MIXED (FULL: FP32 storage and FFTs, FP64 scalars; TT: FP32 fibre transforms
        and sketch side in the solve's steps, FP64 residual, values, eigen-decompositions, dots and A_eff).
        ``rank_tol`` > 0: tolerance truncation with ``rank`` as the cap (0: fixed rank).  ``coeff_rank``:
        rank cap of a grid coefficient's TT compression (0: ``rank``).  ``rank_start`` > 0: rank-adapting
        MinRes from that rank up to ``rank`` in steps of ``rank_step`` (TT).  ``B``: constant symmetric
        positive semidefinite d x d anisotropic part, A~ = a I + B.  ``disc``: GANI, or GA (exact integration
        of the pixel-wise constant material on the double grid; FP64, every format, isotropic for low rank).  ``sketch_over`` > 0 (TT, GaNi):
        the material and P~^-1 products are truncated by the randomised rounding with a sketch of ranks
        rank + sketch_over from SplitMix64 stream ``sketch_seed``; ``sketch_keep``: those truncations keep the
        sketch's rank (no final rounding to ``rank``)."""
        return Problem(self, coeff, fmt, rank, pinv_eps, tol, maxit, stop_on_increase, prec, rank_tol, coeff_rank,
                       rank_start, rank_step, B, disc, sketch_over, sketch_seed, sketch_keep)

    def field_from_full(self, values) -> "Field":
        torch = _torch()
        if isinstance(values, np.ndarray):
            arr = np.ascontiguousarray(values, dtype=np.float64)
            ptr, on_dev, shape, keep = arr.ctypes.data_as(C.c_void_p), 0, arr.shape, arr
        else:
            t = values.contiguous()
            if t.dtype != torch.float64:
                raise ValueError("float64 values required")
            ptr, on_dev, shape, keep = _ptr(t), int(t.is_cuda), tuple(t.shape), t
        h = C.c_void_p()
        self.check(self.lib.lrfg_field_from_full(self.h, len(shape), _ivec(list(shape)[:3], 3), ptr, on_dev,
                                                 C.byref(h)))
        del keep
        return Field(self, h)

    def field_from_tt(self, x: TTensor) -> "Field":
        h = C.c_void_p()
        xs = x.to_struct()
        self.check(self.lib.lrfg_field_from_tt(self.h, C.byref(xs), 1, C.byref(h)))
        return Field(self, h)


class Field:
    """A library-owned field (FULL: Fourier half spectrum; TT: real-space carriages)."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.h = handle
        ctx._adopt(self)

    def info(self):
        fmt, d = C.c_int(), C.c_int()
        N, r = (C.c_int * 3)(), (C.c_int * 4)()
        self.ctx.check(self.ctx.lib.lrfg_field_info(self.h, C.byref(fmt), C.byref(d), N, r))
        return fmt.value, d.value, list(N)[: d.value], list(r)[: d.value + 1]

    def full(self, device: bool = False):
        """Grid values (N^d) as a numpy array (or a CUDA tensor with device=True)."""
        torch = _torch()
        _, d, N, _ = self.info()
        if device:
            out = torch.empty(tuple(N), dtype=torch.float64, device=f"cuda:{self.ctx.device}")
            self.ctx.check(self.ctx.lib.lrfg_field_export_full(self.ctx.h, self.h, _ptr(out), 1))
            return out
        out = np.empty(tuple(N), dtype=np.float64)
        self.ctx.check(self.ctx.lib.lrfg_field_export_full(self.ctx.h, self.h, out.ctypes.data_as(C.c_void_p), 0))
        return out

    def tt(self) -> TTensor:
        torch = _torch()
        fmt, d, N, r = self.info()
        if fmt != TT:
            raise ValueError("not a TT field")
        cores = [torch.empty((r[j], N[j], r[j + 1]), dtype=torch.float64, device=f"cuda:{self.ctx.device}")
                 for j in range(d)]
        arr = (C.c_void_p * 3)(*([c.data_ptr() for c in cores] + [None] * (3 - d)))
        self.ctx.check(self.ctx.lib.lrfg_field_export_tt(self.ctx.h, self.h, arr, 1))
        return TTensor(cores)

    def free(self):
        if self.h and self.ctx.h:
            self.ctx.lib.lrfg_field_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


@dataclass
class Result:
    Aeff: float
    iters: int
    rel_resid: float
    converged: bool
    applies: int
    ranks: list
    seconds: float
    status: int


class Problem:
    """Resident coefficient + operator + solver for one format.  ``coeff``: a numpy/torch grid array
    (isotropic a(x) samples) or a TTensor of the coefficient."""

    def __init__(self, ctx: Context, coeff, fmt, rank, pinv_eps, tol, maxit, stop_on_increase, prec=L.LRFG_FP64,
                 rank_tol=0.0, coeff_rank=0, rank_start=0, rank_step=1, B=None, disc=L.LRFG_GANI, sketch_over=0,
                 sketch_seed=0, sketch_keep=False):
        torch = _torch()
        self.ctx = ctx
        self.fmt = fmt
        c = L.lrfg_coeff()
        keep = None
        if isinstance(coeff, TuckerTensor):
            c.d = coeff.d
            for j, n in enumerate(coeff.shape):
                c.N[j] = n
            c.fmt = L.LRFG_TUCKER
            c.tk = coeff.to_struct()
            c.on_device = 1
            keep = coeff
        elif isinstance(coeff, TTensor):
            c.d = coeff.d
            for j, n in enumerate(coeff.shape):
                c.N[j] = n
            c.fmt = L.LRFG_TT
            c.tt = coeff.to_struct()
            c.on_device = 1
            keep = coeff
        else:
            if isinstance(coeff, np.ndarray):
                arr = np.ascontiguousarray(coeff, dtype=np.float64)
                c.values = arr.ctypes.data
                c.on_device = 0
                keep = arr
            else:
                t = coeff.contiguous()
                if t.dtype != torch.float64:
                    raise ValueError("float64 coefficient required")
                c.values = t.data_ptr()
                c.on_device = int(t.is_cuda)
                keep = t
            c.d = keep.ndim if isinstance(keep, np.ndarray) else keep.dim()
            for j, n in enumerate(list(keep.shape)[:3]):  # the library rejects d outside {2, 3}
                c.N[j] = int(n)
            c.fmt = L.LRFG_FULL
        _set_b(c, B)
        o = L.lrfg_opts()
        o.fmt, o.prec, o.rank, o.pinv_eps = int(fmt), int(prec), int(rank), float(pinv_eps)
        o.tol, o.maxit, o.stop_on_increase = float(tol), int(maxit), int(bool(stop_on_increase))
        o.rank_tol, o.coeff_rank = float(rank_tol), int(coeff_rank)
        o.rank_start, o.rank_step, o.disc = int(rank_start), int(rank_step), int(disc)
        o.sketch_over, o.sketch_seed, o.sketch_keep = int(sketch_over), int(sketch_seed), int(bool(sketch_keep))
        h = C.c_void_p()
        ctx.check(ctx.lib.lrfg_problem_create(ctx.h, C.byref(c), C.byref(o), C.byref(h)))
        del keep
        self.h = h
        self.d = c.d
        ctx._adopt(self)

    def coeff_ranks(self):
        r = (C.c_int * 4)()
        self.ctx.check(self.ctx.lib.lrfg_problem_coeff_ranks(self.h, r))
        return list(r)[: self.d + 1]

    def apply(self, field: Field) -> Field:
        h = C.c_void_p()
        self.ctx.check(self.ctx.lib.lrfg_problem_apply(self.h, field.h, C.byref(h)))
        return Field(self.ctx, h)

    def apply_into(self, field: Field, out: Field) -> Field:
        self.ctx.check(self.ctx.lib.lrfg_problem_apply_into(self.h, field.h, out.h))
        return out

    def rhs(self, E) -> Field:
        h = C.c_void_p()
        self.ctx.check(self.ctx.lib.lrfg_problem_rhs(self.h, _dvec(E), C.byref(h)))
        return Field(self.ctx, h)

    def solve(self, E, want_field: bool = True):
        res = L.lrfg_result()
        h = C.c_void_p()
        st = self.ctx.lib.lrfg_problem_solve(self.h, _dvec(E), C.byref(res), C.byref(h) if want_field else None)
        if st not in (L.LRFG_OK, L.LRFG_ENOCONV):
            self.ctx.check(st)
        out = Result(res.Aeff, res.iters, res.rel_resid, bool(res.converged), res.applies, list(res.ranks)[: self.d + 1],
                     res.seconds, st)
        return out, (Field(self.ctx, h) if want_field and h.value else None)

    def solve_many(self, Es):
        """Solve for every row of Es (nb x d) through lrfg_problem_solve_many (in lockstep for TT problems that
        allow it); returns the list of Results."""
        Es = np.ascontiguousarray(np.asarray(Es, dtype=np.float64).reshape(-1, self.d))
        nb = Es.shape[0]
        res = (L.lrfg_result * nb)()
        st = self.ctx.lib.lrfg_problem_solve_many(self.h, nb, Es.ctypes.data_as(C.POINTER(C.c_double)), res)
        if st not in (L.LRFG_OK, L.LRFG_ENOCONV):
            self.ctx.check(st)
        return [Result(r.Aeff, r.iters, r.rel_resid, bool(r.converged), r.applies, list(r.ranks)[: self.d + 1],
                       r.seconds, st) for r in res]

    @staticmethod
    def solve_together(problems, Es):
        """Solve problem i for row i of Es (len(problems) x d) through lrfg_problems_solve: in lockstep when the
        problems share grid, options and coefficient ranks (a batch of microstructures of one shape), else one
        after the other; returns the list of Results."""
        problems = list(problems)
        if not problems:
            raise ValueError("no problems")
        ctx, d = problems[0].ctx, problems[0].d
        Es = np.ascontiguousarray(np.asarray(Es, dtype=np.float64).reshape(len(problems), d))
        hs = (C.c_void_p * len(problems))(*[p.h for p in problems])
        res = (L.lrfg_result * len(problems))()
        st = ctx.lib.lrfg_problems_solve(len(problems), hs, Es.ctypes.data_as(C.POINTER(C.c_double)), res)
        if st not in (L.LRFG_OK, L.LRFG_ENOCONV):
            ctx.check(st)
        return [Result(r.Aeff, r.iters, r.rel_resid, bool(r.converged), r.applies, list(r.ranks)[: d + 1],
                       r.seconds, st) for r in res]

    def aeff(self, E, field: Field) -> float:
        out = C.c_double()
        self.ctx.check(self.ctx.lib.lrfg_problem_aeff(self.h, _dvec(E), field.h, C.byref(out)))
        return out.value

    def aeff_tensor(self, with_results: bool = False):
        """The homogenised tensor A_eff (d x d) of Eq. (homog) by lrfg_problem_aeff_tensor: d (d + 1) / 2
        solves in the library, the off-diagonal entries by polarisation of the quadratic form A_eff E.E
        (Sec. 2.1).  ``with_results``: also return the per-solve results."""
        d = self.d
        A = (C.c_double * (d * d))()
        res = (L.lrfg_result * (d * (d + 1) // 2))()
        st = self.ctx.lib.lrfg_problem_aeff_tensor(self.h, A, res)
        if st not in (L.LRFG_OK, L.LRFG_ENOCONV):
            self.ctx.check(st)
        T = np.array(list(A)).reshape(d, d)
        if not with_results:
            return T
        return T, [Result(r.Aeff, r.iters, r.rel_resid, bool(r.converged), r.applies, list(r.ranks)[: d + 1],
                          r.seconds, st) for r in res]

    def free(self):
        if self.h and self.ctx.h:
            self.ctx.lib.lrfg_problem_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _set_b(c, B):
    """Copy a d x d anisotropic part into the coefficient struct's 3 x 3 row-major array."""
    if B is None:
        return
    Bm = np.asarray(B, dtype=np.float64)
    if Bm.ndim != 2 or Bm.shape[0] != Bm.shape[1] or Bm.shape[0] != c.d:
        raise ValueError("B must be a d x d matrix")
    for i in range(c.d):
        for j in range(c.d):
            c.B[3 * i + j] = float(Bm[i, j])


def _host_coeff(coeff):
    """lrfg_coeff over host buffers for `coeff`: a grid array (numpy or torch), a TTensor or a list of
    TT carriages, or a TuckerTensor / (core, factors) pair.  Returns (struct, buffers to keep alive)."""
    c = L.lrfg_coeff()
    c.on_device = 0
    f64 = lambda a: np.ascontiguousarray(a.detach().cpu().numpy() if hasattr(a, "detach") else a, dtype=np.float64)
    if isinstance(coeff, TuckerTensor) or (isinstance(coeff, tuple) and len(coeff) == 2):
        core, factors = (coeff.core, coeff.factors) if isinstance(coeff, TuckerTensor) else coeff
        core, factors = f64(core), [f64(f) for f in factors]
        d = len(factors)
        c.d, c.fmt = d, L.LRFG_TUCKER
        c.tk.d = d
        c.tk.core = core.ctypes.data
        for j, f in enumerate(factors):
            c.N[j] = c.tk.N[j] = f.shape[0]
            c.tk.r[j] = f.shape[1]
            c.tk.factors[j] = f.ctypes.data
        return c, [core] + factors
    if isinstance(coeff, (TTensor, list)):
        cores = [f64(x) for x in (coeff.cores if isinstance(coeff, TTensor) else coeff)]
        d = len(cores)
        c.d, c.fmt = d, L.LRFG_TT
        c.tt.d = d
        for j, x in enumerate(cores):
            c.N[j] = c.tt.N[j] = x.shape[1]
            c.tt.r[j] = x.shape[0]
            c.tt.cores[j] = x.ctypes.data
        c.tt.r[d] = 1
        return c, cores
    arr = f64(coeff)
    if arr.ndim not in (2, 3):
        raise ValueError("grid coefficient must have 2 or 3 axes")
    c.d, c.fmt = arr.ndim, L.LRFG_FULL
    for j, n in enumerate(arr.shape):
        c.N[j] = n
    c.values = arr.ctypes.data
    return c, [arr]


@dataclass
class BatchResult:
    result: Result
    queue_s: float   # submission to start
    run_s: float     # start to completion
    total_s: float   # latency: submission to completion
    peak_bytes: float
    worker: int
    group: int = 1   # requests solved together with it in lockstep (itself included)


class Batch:
    """The serving executor of the library (``lrfg_batch_*``): ``workers`` threads, each with its own
    non-blocking stream and context, run submitted solves concurrently in FIFO order; a request starts
    when a worker is free and its HBM footprint fits in ``budget`` bytes (0: no cap) beside the requests
    running.  Coefficients are host arrays, copied at submission.  ``group`` > 1: a worker takes up to that many
    queued requests of one shape together and solves them in lockstep (lrfg_batch_set_group)."""

    def __init__(self, device: int = 0, workers: int = 4, budget: int = 0, group: int = 1):
        self.lib = L.load()
        h = C.c_void_p()
        st = self.lib.lrfg_batch_create(C.byref(h), int(device), int(workers), int(budget))
        if st != L.LRFG_OK:
            raise LrfgError(st, "lrfg_batch_create failed")
        self.h = h
        self.workers = int(workers)
        if int(group) != 1:
            st = self.lib.lrfg_batch_set_group(self.h, int(group))
            if st != L.LRFG_OK:
                self.close()
                raise LrfgError(st, "lrfg_batch_set_group rejected the group size")
        self.group = int(group)

    def submit(self, coeff, E, fmt: int, rank: int = 10, pinv_eps: float = 0.1, tol: float = 1e-8,
               maxit: int = 200, stop_on_increase: bool = True, prec: int = L.LRFG_FP64, rank_tol: float = 0.0,
               coeff_rank: int = 0, rank_start: int = 0, rank_step: int = 1, B=None,
               disc: int = L.LRFG_GANI, sketch_over: int = 0, sketch_seed: int = 0, sketch_keep: bool = False) -> int:
        c, keep = _host_coeff(coeff)
        _set_b(c, B)
        o = L.lrfg_opts()
        o.fmt, o.prec, o.rank, o.pinv_eps = int(fmt), int(prec), int(rank), float(pinv_eps)
        o.tol, o.maxit, o.stop_on_increase = float(tol), int(maxit), int(bool(stop_on_increase))
        o.rank_tol, o.coeff_rank = float(rank_tol), int(coeff_rank)
        o.rank_start, o.rank_step, o.disc = int(rank_start), int(rank_step), int(disc)
        o.sketch_over, o.sketch_seed, o.sketch_keep = int(sketch_over), int(sketch_seed), int(bool(sketch_keep))
        t = C.c_ulonglong()
        st = self.lib.lrfg_batch_submit(self.h, C.byref(c), _dvec(E), C.byref(o), C.byref(t))
        del keep
        if st != L.LRFG_OK:
            raise LrfgError(st, "lrfg_batch_submit rejected the request")
        return int(t.value)

    def poll(self, ticket: int, wait: bool = False):
        """The request's BatchResult once it has completed (None before); the ticket is then retired.
        A solve that failed (other than by reaching maxit) raises LrfgError."""
        ready, sst = C.c_int(), C.c_int()
        res, tm = L.lrfg_result(), L.lrfg_batch_report()
        st = self.lib.lrfg_batch_poll(self.h, C.c_ulonglong(ticket), int(bool(wait)), C.byref(ready), C.byref(sst),
                                      C.byref(res), C.byref(tm))
        if st != L.LRFG_OK:
            raise LrfgError(st, f"unknown or retired ticket {ticket}")
        if not ready.value:
            return None
        if sst.value not in (L.LRFG_OK, L.LRFG_ENOCONV):
            raise LrfgError(sst.value, f"request {ticket}: {tm.message.decode(errors='replace')}")
        r = Result(res.Aeff, res.iters, res.rel_resid, bool(res.converged), res.applies, list(res.ranks), res.seconds,
                   sst.value)
        return BatchResult(r, tm.queue_s, tm.run_s, tm.total_s, tm.peak_bytes, tm.worker, tm.group)

    def wait(self, ticket: int) -> BatchResult:
        return self.poll(ticket, wait=True)

    def info(self):
        """(queued, running, admitted footprint bytes of the running requests)"""
        q, r, b = C.c_int(), C.c_int(), C.c_size_t()
        self.lib.lrfg_batch_info(self.h, C.byref(q), C.byref(r), C.byref(b))
        return q.value, r.value, b.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.lrfg_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
