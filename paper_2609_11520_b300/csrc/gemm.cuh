// Batched complex GEMM of the HSS large-node and ULV steps (plain dense
// products of Sections 2.4 and 3.1-3.3): for b = 0 .. batch-1
//   C_b = alpha op(A_b) op(B_b) + beta C_b,   op = identity ('N') or conjugate transpose ('C'),
// column-major blocks with leading dimensions lda, ldb, ldc and element
// strides sA, sB, sC between consecutive blocks.  complex64 (float2) or
// complex128 (double2); alpha, beta real.  beta = 0 never reads C.
#pragma once
#include "common.cuh"

namespace fio {
template <class C>
fio_status bgemm(char ta, char tb, int m, int n, int k, double alpha, const C* A, int64_t lda, int64_t sA, const C* B,
                 int64_t ldb, int64_t sB, double beta, C* Cm, int64_t ldc, int64_t sC, int batch, cudaStream_t st);
}
