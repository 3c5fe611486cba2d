// Internal entry point of the tensor-core Gram matrix (gram_tc.cu).
#pragma once
#include "common.cuh"

namespace ssm {

// G[a][b] += sum_i d_ia^2 d_ib^2 for a <= b < k as 128-bit integers (Glo, Ghi
// zeroed by the caller), on tcgen05 with BF16 digit planes; *dmax (device)
// must hold the largest d_ip entry.  Asynchronous on s.
int launch_gram_tc(int32_t n, int32_t k, const uint16_t *dip, const unsigned *dmax, unsigned long long *Glo,
                   unsigned long long *Ghi, int32_t *status, cudaStream_t s);

}  // namespace ssm
