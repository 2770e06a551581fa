"""GB300 (sm_103a) library for the higher-order time-evolution MPO method of
arXiv:2302.14181 ("Efficient higher-order matrix product operators for time
evolution").

Thin Python binding over the C ABI declared in ``include/tevo.h``: the functions
below carry the C names and only marshal arguments (numpy arrays in, numpy
arrays out). Every step of the time-evolution path runs in the CUDA kernels of
``libtevo.so``; there is no Python or CPU fallback. Importing this package
raises if the library has not been built (``python -m paper_2302_14181_gb300._build``).

PyTorch, when importable with CUDA, supplies the stream (the current stream at
context creation) and the device memory (its caching allocator, registered as
the library's allocator).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _lib
from ._lib import (FP64, TF32, TF32X3, BF16X3, TC_ONLY, OZAKI, OZAKI_SLICES, TWO_SITE, MPO_PLAIN, MPO_EXACT,  # noqa: F401
                   MPO_EXTENDED, MPO_FULL, TevoError)

__all__ = [
    "Context", "MPO", "MPS", "mpo_build", "mpo_build_host", "mps_init", "evolve_step", "evolve_step_batched", "measure_local", "mps_overlap",
    "tevo_gemm", "tevo_gemm_noalloc", "tevo_wait_selftest", "tevo_strerror",
    "FP64", "TF32", "TF32X3", "BF16X3", "TC_ONLY", "OZAKI", "OZAKI_SLICES", "TWO_SITE", "MPO_PLAIN", "MPO_EXACT", "MPO_EXTENDED", "MPO_FULL",
    "TevoError", "library_path",
]


def library_path():
    return _lib.LIB_PATH


def _c128(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Context:
    """A library context bound to one CUDA stream of the current device."""

    def __init__(self, stream=None, use_torch=True):
        self._torch_cb = None
        h = _lib.tevo_ctx()
        if stream is None and use_torch:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                pass
        _lib.check(_lib.lib.tevo_ctx_create(ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.handle = h
        self.stream = stream or 0
        if use_torch:
            self._register_torch_allocator()

    def _register_torch_allocator(self):
        try:
            import torch
        except ImportError:
            return
        if not torch.cuda.is_available():
            return
        dev = torch.cuda.current_device()
        stream = self.stream

        @_lib.ALLOC_FN
        def _alloc(nbytes, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
            except Exception:  # allocation failure is reported to the library as NULL
                return None

        @_lib.FREE_FN
        def _free(ptr, user):
            torch.cuda.caching_allocator_delete(ptr)

        self._torch_cb = (_alloc, _free)
        _lib.check(_lib.lib.tevo_ctx_set_allocator(self.handle, _alloc, _free, None))

    def prof_enable(self, on=True):
        _lib.check(_lib.lib.tevo_prof_enable(self.handle, int(on)))

    def prof_read(self, cls):
        """(total ms, launches, algorithmic flops, algorithmic bytes) of one kernel class."""
        ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_longlong()
        _lib.check(_lib.lib.tevo_prof_read(self.handle, int(cls), ctypes.byref(ms), ctypes.byref(n),
                                           ctypes.byref(fl), ctypes.byref(by)))
        return ms.value, n.value, fl.value, by.value

    def launch_count(self, reset=False):
        n = ctypes.c_longlong()
        _lib.check(_lib.lib.tevo_launch_count(self.handle, ctypes.byref(n), int(reset)))
        return n.value

    def close(self):
        if self.handle:
            _lib.lib.tevo_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MPO:
    def __init__(self, ctx, handle, L, d, N, tau):
        self.ctx, self.handle, self.L, self.d, self.N, self.tau = ctx, handle, L, d, N, complex(tau)

    def bond_dims(self):
        w = (ctypes.c_int * (self.L + 1))()
        _lib.check(_lib.lib.mpo_bond_dims(self.handle, w))
        return list(w)

    def site(self, i):
        w = self.bond_dims()
        out = np.zeros((w[i], self.d, self.d, w[i + 1]), np.complex128)
        _lib.check(_lib.lib.mpo_get_site(self.handle, i, _ptr(out)))
        return out

    def close(self):
        if self.handle:
            _lib.lib.mpo_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MPS:
    def __init__(self, ctx, handle, L, d, D):
        self.ctx, self.handle, self.L, self.d, self.D = ctx, handle, L, d, D

    def bond_dims(self):
        w = (ctypes.c_int * (self.L + 1))()
        _lib.check(_lib.lib.mps_bond_dims(self.handle, w))
        return list(w)

    def site(self, i):
        dims = self.bond_dims()
        out = np.zeros((dims[i], self.d, dims[i + 1]), np.complex128)
        _lib.check(_lib.lib.mps_get_site(self.handle, i, _ptr(out)))
        return out

    def set_site(self, i, a):
        dims = self.bond_dims()
        a = _c128(a, (dims[i], self.d, dims[i + 1]))
        _lib.check(_lib.lib.mps_set_site(self.handle, i, _ptr(a)))

    def tensors(self):
        return [self.site(i) for i in range(self.L)]

    def log_norm(self):
        v = ctypes.c_double()
        _lib.check(_lib.lib.mps_log_norm(self.handle, ctypes.byref(v)))
        return v.value

    def close(self):
        if self.handle:
            _lib.lib.mps_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mpo_build(ctx, A, B, C, Dh, N, tau, variant=MPO_FULL):
    """W^(N)(tau) from per-site Hamiltonian MPO blocks (see include/tevo.h)."""
    Dh = _c128(Dh)
    L, d = Dh.shape[0], Dh.shape[1]
    A = _c128(A)
    chi = A.shape[1]
    A = _c128(A, (L, chi, chi, d, d))
    B = _c128(B, (L, chi, d, d))
    C = _c128(C, (L, chi, d, d))
    tau = complex(tau)
    h = _lib.tevo_mpo()
    _lib.check(_lib.lib.mpo_build(ctx.handle, L, d, chi, _ptr(A), _ptr(B), _ptr(C), _ptr(Dh), int(N),
                                  tau.real, tau.imag, int(variant), ctypes.byref(h)))
    return MPO(ctx, h, L, d, N, tau)


def mpo_build_host(A, B, C, Dh, N, tau, variant=MPO_FULL):
    """The host-side construction alone: list of W_i[w_l, d, d, w_r] (no GPU needed)."""
    Dh = _c128(Dh)
    L, d = Dh.shape[0], Dh.shape[1]
    A = _c128(A)
    chi = A.shape[1]
    A = _c128(A, (L, chi, chi, d, d))
    B = _c128(B, (L, chi, d, d))
    C = _c128(C, (L, chi, d, d))
    tau = complex(tau)
    w = (ctypes.c_int * (L + 1))()
    n = ctypes.c_size_t(0)
    args = (L, d, chi, _ptr(A), _ptr(B), _ptr(C), _ptr(Dh), int(N), tau.real, tau.imag, int(variant), w)
    _lib.check(_lib.lib.mpo_build_host(*args, None, ctypes.byref(n)))
    buf = np.zeros(n.value, np.complex128)
    _lib.check(_lib.lib.mpo_build_host(*args, _ptr(buf), ctypes.byref(n)))
    out, off = [], 0
    for i in range(L):
        k = w[i] * d * d * w[i + 1]
        out.append(buf[off:off + k].reshape(w[i], d, d, w[i + 1]))
        off += k
    return out


def mps_init(ctx, site_vectors, D):
    """Product state (site_vectors: complex [L, d]) at bond cap D."""
    v = _c128(site_vectors)
    L, d = v.shape
    h = _lib.tevo_mps()
    _lib.check(_lib.lib.mps_init(ctx.handle, L, d, int(D), _ptr(v), ctypes.byref(h)))
    return MPS(ctx, h, L, d, int(D))


def evolve_step(psi, W, tau, D, sweeps=1, precision=FP64):
    tau = complex(tau)
    _lib.check(_lib.lib.evolve_step(psi.handle, W.handle, tau.real, tau.imag, int(D), int(sweeps),
                                    int(precision)))


def evolve_step_batched(psis, Ws, sweeps=1, precision=FP64):
    """One time step of independent chains (each with its own MPO and its MPO's tau)."""
    n = len(psis)
    if n != len(Ws) or n == 0:
        raise ValueError("need one MPO per state")
    ps = (_lib.tevo_mps * n)(*[p.handle for p in psis])
    ws = (_lib.tevo_mpo * n)(*[w.handle for w in Ws])
    _lib.check(_lib.lib.evolve_step_batched(ps, ws, n, int(sweeps), int(precision)))


def measure_local(psi, ops):
    """<O_i> for every site and each operator: complex array [len(ops), L]."""
    ops = _c128(np.stack([np.asarray(o) for o in ops]))
    out = np.zeros((ops.shape[0], psi.L), np.complex128)
    _lib.check(_lib.lib.measure_local(psi.handle, ops.shape[0], _ptr(ops), _ptr(out)))
    return out


def mps_overlap(a, b):
    """(log|<a|b>|, arg <a|b>)."""
    la, ph = ctypes.c_double(), ctypes.c_double()
    _lib.check(_lib.lib.mps_overlap(a.handle, b.handle, ctypes.byref(la), ctypes.byref(ph)))
    return la.value, ph.value


def _device_matrix(t, name):
    """(rows, cols, device address) of a C-contiguous 2-D complex128 CUDA tensor."""
    try:
        import torch
    except ImportError as e:  # pragma: no cover - torch is a dependency of the device API
        raise TypeError(f"{name}: device operands are torch CUDA tensors") from e
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128 and t.dim() == 2
            and t.is_contiguous()):
        raise TypeError(f"{name} must be a C-contiguous 2-D complex128 CUDA tensor")
    return int(t.shape[0]), int(t.shape[1]), int(t.data_ptr())


def _gemm_args(A, B, C):
    M, K, pa = _device_matrix(A, "A")
    N, KB, pb = _device_matrix(B, "B")
    MC, NC, pc = _device_matrix(C, "C")
    if KB != K or (MC, NC) != (M, N):
        raise ValueError(f"shapes A {M}x{K}, B {N}x{KB}, C {MC}x{NC}: need B N x K and C M x N")
    return M, N, K, ctypes.c_void_p(pa), ctypes.c_void_p(pb), ctypes.c_void_p(pc)


def tevo_gemm(ctx, precision, A, B, C):
    """C[m, n] = sum_k A[m, k] B[n, k] on the device in the given precision.

    A [M, K], B [N, K] (rows of B, k contiguous) and C [M, N]: C-contiguous
    complex128 CUDA tensors. Returns C. Synchronises the context's stream."""
    M, N, K, pa, pb, pc = _gemm_args(A, B, C)
    _lib.check(_lib.lib.tevo_gemm(ctx.handle, int(precision), M, N, K, pa, pb, pc))
    return C


def tevo_gemm_noalloc(ctx, precision, A, B, C):
    """tevo_gemm without any device allocation (the library's fixed scratch
    array; shapes that do not fit it raise TevoError with TEVO_ESHAPE). A, B and
    C must sit on the context's device, which must be current."""
    M, N, K, pa, pb, pc = _gemm_args(A, B, C)
    import torch
    cur = torch.cuda.current_device()
    for name, t in (("A", A), ("B", B), ("C", C)):
        if t.device.index != cur:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{cur}")
    _lib.check(_lib.lib.tevo_gemm_noalloc(ctx.handle, int(precision), M, N, K, pa, pb, pc))
    return C


def tevo_wait_selftest(ctx, limit_ms):
    """Run the bounded device-side wait until it gives up after limit_ms.
    Returns (status, device code); the expected status is TEVO_ETIMEOUT."""
    code = ctypes.c_int(0)
    rc = _lib.lib.tevo_wait_selftest(ctx.handle, float(limit_ms), ctypes.byref(code))
    return rc, code.value


def tevo_strerror(code):
    """Name of a libtevo error code."""
    return _lib.lib.tevo_strerror(int(code)).decode()
