"""bf_apply_noalloc (collected last): the allocation-free apply for callers
that cannot let the library allocate device memory.  Called through the C
ABI and compared with bf_apply on the same inputs, twice in a row (the second
call must not see anything left in the shared fixed scratch array), on the
fused path, the per-level path (two state arrays in the scratch) and split
precision; and the first call on a fresh handle leaves the device's free
memory unchanged."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
TOL = 1e-5   # the tolerance of the BF apply tests


def _call(name, bf, X, Y, adjoint):
    from paper_2609_11520_b300 import _lib
    fn = getattr(_lib.lib, name)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(bf.handle, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), X.shape[1], X.shape[0],
              int(adjoint), st)


def _rand(rng, k, n):
    return torch.from_numpy((rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n)))
                            .astype(np.complex64)).cuda()


def _configure(bf, path, precision):
    bf.set_path(path)
    bf.set_precision(precision)
    return bf


# (N, k, path, precision): the per-level path at N = 2^17 needs 2 N r = 2^22 elements, the
# whole fixed scratch, so it runs one column per chunk
CASES = [(1 << 16, 9, "auto", "fp32"), (4096, 3, "auto", "fp32"), (1 << 17, 3, "per_level", "fp32"),
         (2048, 5, "per_level", "fp32"), (1 << 16, 5, "auto", "split_bf16")]


@pytest.mark.parametrize("n,k,path,precision", CASES)
def test_noalloc_matches_bf_apply_twice(n, k, path, precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_11520_b300 import BF, _lib
    bf = _configure(BF(n, 16), path, precision)
    rng = np.random.default_rng(n + k)
    for call in range(2):
        for adjoint in (0, 1):
            X = _rand(rng, k, n)
            ref = torch.empty_like(X)
            out = torch.full_like(X, complex(np.nan, np.nan))
            assert _call("bf_apply", bf, X, ref, adjoint) == _lib.FIO_OK
            assert _call("bf_apply_noalloc", bf, X, out, adjoint) == _lib.FIO_OK, _lib.lib.fio_last_error()
            torch.cuda.synchronize()
            err = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
            assert err <= TOL, (call, adjoint, err)


@pytest.mark.parametrize("path,precision", [("auto", "fp32"), ("per_level", "fp32"), ("auto", "split_bf16")])
def test_noalloc_first_call_allocates_nothing(path, precision):
    """A fresh handle has no apply scratch yet: bf_apply would allocate it, bf_apply_noalloc
    must not.  The kernels are loaded beforehand through another handle (lazy module loading
    may allocate on a kernel's first launch), then the device's free memory is compared."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_11520_b300 import BF, _lib
    n, k = 1 << 15, 4
    rng = np.random.default_rng(7)
    X = _rand(rng, k, n)
    Y = torch.empty_like(X)
    warm = _configure(BF(n, 16), path, precision)
    for adjoint in (0, 1):
        assert _call("bf_apply", warm, X, Y, adjoint) == _lib.FIO_OK
        assert _call("bf_apply_noalloc", warm, X, Y, adjoint) == _lib.FIO_OK
    fresh = _configure(BF(n, 16), path, precision)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for adjoint in (0, 1):
        assert _call("bf_apply_noalloc", fresh, X, Y, adjoint) == _lib.FIO_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_too_large():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_11520_b300 import BF, _lib
    bf = BF(1 << 19, 16)          # per-level path: 2 N r = 2^24 elements > 2^22
    X = torch.zeros(1, 1 << 19, dtype=torch.complex64, device="cuda")
    Y = torch.empty_like(X)
    assert _call("bf_apply_noalloc", bf, X, Y, 0) == _lib.FIO_EINVAL
    assert b"fixed scratch" in _lib.lib.fio_last_error()
