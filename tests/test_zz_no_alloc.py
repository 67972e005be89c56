"""bf_apply_noalloc (collected last): the allocation-free apply for callers
that cannot let the library allocate device memory.  Called through the C
ABI and compared with bf_apply on the same inputs, twice in a row (the second
call must not see anything left in the shared fixed scratch array)."""
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


@pytest.mark.parametrize("n,k", [(1 << 16, 9), (4096, 3)])
def test_noalloc_matches_bf_apply_twice(n, k):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_11520_b300 import BF, _lib
    bf = BF(n, 16)
    rng = np.random.default_rng(n + k)
    for call in range(2):
        for adjoint in (0, 1):
            X = torch.from_numpy((rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n)))
                                 .astype(np.complex64)).cuda()
            ref = torch.empty_like(X)
            out = torch.full_like(X, complex(np.nan, np.nan))
            assert _call("bf_apply", bf, X, ref, adjoint) == _lib.FIO_OK
            assert _call("bf_apply_noalloc", bf, X, out, adjoint) == _lib.FIO_OK, _lib.lib.fio_last_error()
            torch.cuda.synchronize()
            err = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
            assert err <= TOL, (call, adjoint, err)


def test_noalloc_rejects_too_large():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_11520_b300 import BF, _lib
    bf = BF(1 << 19, 16)          # per-level path: 2 N r = 2^24 elements > 2^22
    X = torch.zeros(1, 1 << 19, dtype=torch.complex64, device="cuda")
    Y = torch.empty_like(X)
    assert _call("bf_apply_noalloc", bf, X, Y, 0) == _lib.FIO_EINVAL
    assert b"fixed scratch" in _lib.lib.fio_last_error()
