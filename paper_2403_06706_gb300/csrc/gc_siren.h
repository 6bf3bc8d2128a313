// gc_siren.h -- host-side entry points of the tensor-core kernels (gc_siren.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace gcs {
// C = A B^T (+= with atomic != 0), A: M x K, B: N x K bf16 row-major; M, N multiples of 128,
// K a multiple of 64; splits > 1 splits K (atomic must be set)
cudaError_t gemm_bf16_tn(const void *A, const void *B, float *C, int M, int N, int K, int splits, int atomic,
                         cudaStream_t s);
// 2-D bf16 tensor map: inner (contiguous) extent, outer extent, box of 64 x box_outer, SW128
cudaError_t make_map_bf16(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer, uint32_t box_outer);
// error word of the tensor-core kernels (0 = none); reading clears it (synchronises s)
int read_error(cudaStream_t s);
} // namespace gcs
