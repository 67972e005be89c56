"""Python binding of the FIO library: argument marshalling over the C ABI.

Vectors are complex64 CUDA tensors of shape (N,) (one vector) or (k, N)
(k vectors, each row contiguous -- the column-major N x k block of the C ABI
with leading dimension N).  Every computation runs in libfio_b300.so on the
current CUDA stream.
"""
import ctypes

import torch

from . import _lib
from ._lib import FioError, check, lib

__all__ = ["BF", "HSS", "Batch", "fio_solve", "fio_pcg", "device_status", "FioError"]


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _block(x, n, name):
    """(ptr, ld, k) of a (N,) or (k, N) complex64 CUDA tensor with unit inner stride."""
    if not isinstance(x, torch.Tensor) or x.dtype != torch.complex64 or not x.is_cuda:
        raise TypeError(f"{name}: expected a complex64 CUDA tensor")
    if x.dim() == 1:
        if x.shape[0] != n or x.stride(0) != 1:
            raise ValueError(f"{name}: expected a contiguous vector of length {n}")
        return x.data_ptr(), n, 1
    if x.dim() != 2 or x.shape[1] != n or x.stride(1) != 1 or (x.shape[0] > 1 and x.stride(0) < n):
        raise ValueError(f"{name}: expected shape (k, {n}) with rows contiguous")
    return x.data_ptr(), (x.stride(0) if x.shape[0] > 1 else n), x.shape[0]


def _dim(phase, d):
    return (2 if phase in ("elliptic2d", "iso2d") else 1) if d is None else int(d)


def _amp(amp):
    """ctypes pointer to the amplitude (None: a = 1) and the array it borrows."""
    import numpy as np
    if amp is None:
        return None, None
    kind = amp if isinstance(amp, str) else amp[0]
    a = _lib.Amp(_lib.AMP_KINDS[kind], 0, 1.0, None)
    keep = None
    if kind == "bumps":
        keep = np.ascontiguousarray(np.asarray(amp[1], dtype=np.float64).reshape(-1, 2))
        a.m, a.sigma2 = keep.shape[0], float(amp[2])
        a.centers = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return ctypes.pointer(a), (a, keep)


def _index_pair(rows, cols):
    import numpy as np
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64).ravel())
    c = np.ascontiguousarray(np.asarray(cols, dtype=np.int64).ravel())
    if r.shape != c.shape:
        raise ValueError("rows and cols must have the same length")
    P = ctypes.POINTER(ctypes.c_int64)
    return r.ctypes.data_as(P), c.ctypes.data_as(P), int(r.size), (r, c)


def entry_error(n, r, rows, cols, phase="cabs", s=1.0, d=None, amp=None, stream=None):
    """bf_entry_error: the FP64 relative error of the rank-r BF on the sampled entries, without
    building its tables."""
    d = _dim(phase, d)
    ph = _lib.Phase(_lib.PHASE_KINDS[phase], float(s))
    a, keep = _amp(amp)
    pr, pc, S, kp = _index_pair(rows, cols)
    e = ctypes.c_double()
    check(lib.bf_entry_error(ctypes.byref(ph), a, int(n), d, int(r), pr, pc, S, _stream(stream), ctypes.byref(e)))
    del keep, kp
    return e.value


class BF:
    """Butterfly factorization K~ of the FIO (bf_build / bf_apply).

    n points per dimension; d = 2 for the "elliptic2d" phase (and for "dft"
    when asked), else 1.  Vectors have length N = n^d (lexicographic in 2D)
    and are held as (k, N) complex64 CUDA tensors; `self.n` is N.
    """

    def __init__(self, n, r=16, phase="cabs", s=1.0, stream=None, d=None, amp=None, _handle=None):
        """amp: None (a = 1), ("bumps", centers, sigma2) with centers an (m, 2) array of (x_k, xi_k)
        (Section 5.1), or "hankel" (Section 5.3, with phase "iso2d")."""
        d = _dim(phase, d)
        if _handle is None:
            ph = _lib.Phase(_lib.PHASE_KINDS[phase], float(s))
            a, keep = _amp(amp)
            h = ctypes.c_void_p()
            check(lib.bf_build_amp(ctypes.byref(ph), a, int(n), d, int(r), _stream(stream), ctypes.byref(h)))
            del keep
        else:
            h = _handle
        self._h = h
        self.n_side, self.d = int(n), d
        self.n, self.r, self.phase, self.s = int(n) ** d, int(r), phase, float(s)
        self.entry_error = None

    @classmethod
    def with_tol(cls, n, tol, rows, cols, phase="cabs", s=1.0, d=None, amp=None, stream=None):
        """Adaptive rank (bf_build_tol): the smallest candidate rank whose FP64 error on the sampled
        entries (rows[e], cols[e]) is <= tol.  The handle's `r` and `entry_error` report the choice."""
        d = _dim(phase, d)
        ph = _lib.Phase(_lib.PHASE_KINDS[phase], float(s))
        a, keep = _amp(amp)
        pr, pc, S, kp = _index_pair(rows, cols)
        h = ctypes.c_void_p()
        r = ctypes.c_int()
        e = ctypes.c_double()
        check(lib.bf_build_tol(ctypes.byref(ph), a, int(n), d, float(tol), pr, pc, S, _stream(stream), ctypes.byref(h),
                               ctypes.byref(r), ctypes.byref(e)))
        del keep, kp
        bf = cls(n, r.value, phase, s, d=d, _handle=h)
        bf.entry_error = e.value
        return bf

    def entries(self, rows, cols, stream=None):
        """(S, 2) complex128: column 0 the sampled entries of K~ evaluated in FP64 from the factor
        definitions, column 1 the entries of K (bf_entries)."""
        import numpy as np
        pr, pc, S, kp = _index_pair(rows, cols)
        out = np.empty(4 * S, dtype=np.float64)
        check(lib.bf_entries(self._h, pr, pc, S, _stream(stream), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        del kp
        return out.view(np.complex128).reshape(S, 2)

    @property
    def handle(self):
        return self._h

    PATHS = {"auto": 0, "per_level": 1, "fused": 2, "fused_v2": 3, "fused_simt": 4}

    def set_path(self, path):
        """0 automatic, 1 per-level kernels, 2 fused two-pass kernels (transfer levels on the tensor
        cores), 3 fused without table staging, 4 ("fused_simt") the staged fused kernels with the
        FP32 transfer levels on the CUDA cores."""
        check(lib.bf_set_path(self._h, int(self.PATHS.get(path, path))))
        return self

    def set_precision(self, precision):
        """"fp32" (default; FP32 accuracy, tensor-core transfer levels on FP16 hi + lo parts) or
        "split_bf16" (tensor-core transfer levels on BF16 hi + lo parts)."""
        check(lib.bf_set_precision(self._h, int({"fp32": 0, "split_bf16": 1}.get(precision, precision))))
        return self

    def info(self):
        o = (ctypes.c_int64 * 8)()
        check(lib.bf_info(self._h, o))
        return dict(zip(["n", "d", "r", "L", "h", "sU", "sV", "table_bytes"], list(o)))

    def apply(self, X, adjoint=False, out=None, stream=None):
        px, ld, k = _block(X, self.n, "X")
        if out is None:
            out = torch.empty_like(X)
        py, ldy, ky = _block(out, self.n, "out")
        if ky != k or ldy != ld:
            raise ValueError("out must match X in shape and row stride")
        check(lib.bf_apply(self._h, ctypes.c_void_p(px), ctypes.c_void_p(py), ld, k, int(bool(adjoint)),
                           _stream(stream)))
        return out

    def adjoint(self, X, out=None, stream=None):
        return self.apply(X, adjoint=True, out=out, stream=stream)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.bf_free(h)
            self._h = ctypes.c_void_p()


class HSS:
    """HSS approximation G~ with its ULV factorization (hss_* calls)."""

    def __init__(self, handle, n):
        self._h = handle
        self.n = int(n)
        self.factored = False
        self._keep = None

    @classmethod
    def from_samples(cls, bf=None, dense=None, n=None, leaf=128, oversample=10, tol=1e-3, seed=0, stream=None):
        sm = _lib.Sampler()
        if bf is not None:
            sm.kind, sm.bf, n = _lib.SAMPLER_NORMAL, bf.handle.value, bf.n
        else:
            if dense is None or dense.dtype != torch.complex64 or not dense.is_cuda:
                raise TypeError("dense sampler: complex64 CUDA tensor (N, N) expected")
            n = dense.shape[0]
            # The C ABI takes H column-major; the row-major storage of H^T is exactly that.
            dense = dense.transpose(0, 1).contiguous()
            sm.kind, sm.dense, sm.ld = _lib.SAMPLER_DENSE, dense.data_ptr(), dense.stride(0)
        h = ctypes.c_void_p()
        check(lib.hss_build_from_samples(ctypes.byref(sm), int(n), int(leaf), int(oversample), float(tol),
                                         ctypes.c_uint64(int(seed)), _stream(stream), ctypes.byref(h)))
        obj = cls(h, n)
        obj._keep = (bf, dense)
        return obj

    @classmethod
    def from_generators(cls, n, leaf, ranks, U, B, D, stream=None):
        """Host generators (numpy complex arrays in the C layout, see hss_from_generators)."""
        import numpy as np
        rk = (ctypes.c_int * len(ranks))(*[int(v) for v in ranks])
        Ua = np.ascontiguousarray(U, dtype=np.complex64)
        Ba = np.ascontiguousarray(B, dtype=np.complex64)
        Da = np.ascontiguousarray(D, dtype=np.complex64)
        h = ctypes.c_void_p()
        check(lib.hss_from_generators(int(n), int(leaf), rk, Ua.ctypes.data_as(ctypes.c_void_p),
                                      Ba.ctypes.data_as(ctypes.c_void_p), Da.ctypes.data_as(ctypes.c_void_p),
                                      _stream(stream), ctypes.byref(h)))
        return cls(h, n)

    @property
    def handle(self):
        return self._h

    def info(self):
        o = (ctypes.c_int64 * 64)()
        smp = ctypes.c_int64()
        check(lib.hss_info(self._h, o, 64, ctypes.byref(smp)))
        Lh = int(o[2])
        return dict(N=int(o[0]), leaf=int(o[1]), Lh=Lh, ranks=[int(o[3 + l]) for l in range(Lh + 1)],
                    samples=int(smp.value))

    def matvec(self, X, out=None, stream=None):
        px, ld, k = _block(X, self.n, "X")
        out = torch.empty_like(X) if out is None else out
        py, _, _ = _block(out, self.n, "out")
        check(lib.hss_matvec(self._h, ctypes.c_void_p(px), ctypes.c_void_p(py), ld, k, _stream(stream)))
        return out

    def factor(self, stream=None):
        check(lib.hss_ulv_factor(self._h, _stream(stream)))
        self.factored = True
        return self

    def set_solve_path(self, path):
        """"cuda_cores" (default) or "tensor_cores" (node products of k > 8 columns on tcgen05 with
        FP16 or, under a split-precision BF handle, BF16 parts; hss_set_solve_path)."""
        check(lib.hss_set_solve_path(self._h, int({"cuda_cores": 0, "tensor_cores": 1}.get(path, path))))
        return self

    def solve(self, Bm, out=None, stream=None):
        px, ld, k = _block(Bm, self.n, "B")
        out = torch.empty_like(Bm) if out is None else out
        py, _, _ = _block(out, self.n, "out")
        check(lib.hss_solve(self._h, ctypes.c_void_p(px), ctypes.c_void_p(py), ld, k, _stream(stream)))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.hss_free(h)
            self._h = ctypes.c_void_p()


def device_status():
    """Raise FioError (FIO_ETIMEOUT) if a bounded wait inside a tensor-core kernel ran out since
    the last call; synchronizes with the device."""
    check(lib.fio_device_status())


def fio_solve(bf, hss, U, out=None, refine_steps=0, stream=None):
    """f = G~^{-1} K~^* u (+ refinement steps)."""
    px, ld, k = _block(U, bf.n, "U")
    out = torch.empty_like(U) if out is None else out
    py, _, _ = _block(out, bf.n, "F")
    check(lib.fio_solve(bf.handle, hss.handle, ctypes.c_void_p(px), ctypes.c_void_p(py), ld, k,
                        int(refine_steps), _stream(stream)))
    return out


def fio_pcg(bf, hss, U, out=None, tol=1e-6, maxit=50, stream=None):
    """CG on K~^* K~ f = K~^* u preconditioned by the ULV factorization of G~ (Section 4.1).
    Returns (F, iterations, relative residual per column)."""
    px, ld, k = _block(U, bf.n, "U")
    out = torch.empty_like(U) if out is None else out
    py, _, _ = _block(out, bf.n, "F")
    it = ctypes.c_int(0)
    rr = (ctypes.c_double * max(k, 1))()
    check(lib.fio_pcg(bf.handle, hss.handle, ctypes.c_void_p(px), ctypes.c_void_p(py), ld, k, float(tol), int(maxit),
                      ctypes.byref(it), rr, _stream(stream)))
    return out, int(it.value), [float(rr[i]) for i in range(k)]


class Batch:
    """Batched online solves over resident operators of uneven size (fio_batch_*).

    ops: list of (BF, HSS) with factored HSS.  solve(Us) takes one (k_i, N_i)
    complex64 CUDA tensor per operator and returns the solutions.
    """

    MODES = {"per_operator": 0, "grouped": 1, "graph": 2, "persistent": 3}

    def __init__(self, ops):
        self.ops = list(ops)
        n = len(self.ops)
        bfs = (ctypes.c_void_p * n)(*[b.handle.value for b, _ in self.ops])
        hss = (ctypes.c_void_p * n)(*[h.handle.value for _, h in self.ops])
        h = ctypes.c_void_p()
        check(lib.fio_batch_create(bfs, hss, n, ctypes.byref(h)))
        self._h = h

    def set_mode(self, mode):
        check(lib.fio_batch_set_mode(self._h, int(self.MODES.get(mode, mode))))
        return self

    def _arrays(self, Us, Fs):
        n = len(self.ops)
        if len(Us) != n or len(Fs) != n:
            raise ValueError("one U and one F per operator")
        ks = []
        for (bf, _), U, F in zip(self.ops, Us, Fs):
            pu, ld, k = _block(U, bf.n, "U")
            pf, ldf, kf = _block(F, bf.n, "F")
            if ld != bf.n or ldf != bf.n or kf != k:
                raise ValueError("U and F must be contiguous (k, N) blocks of equal shape")
            ks.append(k)
        U_arr = (ctypes.c_void_p * n)(*[U.data_ptr() for U in Us])
        F_arr = (ctypes.c_void_p * n)(*[F.data_ptr() for F in Fs])
        k_arr = (ctypes.c_int * n)(*ks)
        return U_arr, F_arr, k_arr

    def solve(self, Us, Fs=None, stream=None):
        Fs = [torch.empty_like(U) for U in Us] if Fs is None else Fs
        U_arr, F_arr, k_arr = self._arrays(Us, Fs)
        check(lib.fio_batch_solve(self._h, U_arr, F_arr, k_arr, _stream(stream)))
        return Fs

    def autotune(self, Us, Fs, reps=3, stream=None):
        U_arr, F_arr, k_arr = self._arrays(Us, Fs)
        buf = ctypes.create_string_buffer(4096)
        check(lib.fio_batch_autotune(self._h, U_arr, F_arr, k_arr, int(reps), _stream(stream), buf, len(buf)))
        return buf.value.decode()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.fio_batch_free(h)
            self._h = ctypes.c_void_p()


def set_large_node(m_min):
    """Node size from which HSS levels of at most 16 nodes use the FP64 level-3 kernels (default 384)."""
    check(lib.fio_set_large_node(int(m_min)))
