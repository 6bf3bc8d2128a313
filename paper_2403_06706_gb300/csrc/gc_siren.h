// gc_siren.h -- host-side entry points of the tensor-core kernels (gc_siren.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace gcs {
// C = A B^T (+= with atomic != 0) for bf16 A (M x K) and B (N x K), each stored K-major
// (row-major M x K / N x K) or, with a_mn / b_mn set, MN-major (row-major K x M / K x N);
// M, N multiples of 128, K a multiple of 64; splits > 1 splits K (atomic must be set)
cudaError_t gemm_bf16(const void *A, int a_mn, const void *B, int b_mn, float *C, int M, int N, int K,
                      int splits, int atomic, cudaStream_t s);
// 2-D bf16 tensor map: inner (contiguous) extent, outer extent, box of 64 x box_outer, SW128
cudaError_t make_map_bf16(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer, uint32_t box_outer);
// error word of the tensor-core kernels (0 = none); reading clears it (synchronises s)
int read_error(cudaStream_t s);
} // namespace gcs

// ------------------------------------------------------------------- the neural field
// SIREN 3 -> 256 x 4 -> 8 (Sitzmann et al. 2020). Flat FP32 parameter layout: W1 (256 x 3),
// b1 (256), then W2, b2, W3, b3, W4, b4 (256 x 256 [out][in], 256), then W5 (8 x 256), b5 (8).
namespace gcs {
constexpr int kSirenH = 256;
constexpr int kSirenOut = 8;
constexpr int64_t kSirenNParams = 768 + 256 + 3 * (65536 + 256) + 2048 + 8;
__host__ __device__ constexpr int64_t siren_oW(int L) { return L == 1 ? 0 : (L == 5 ? 198400 : 1024 + (int64_t)(L - 2) * 65792); }
__host__ __device__ constexpr int64_t siren_oB(int L) { return L == 1 ? 768 : (L == 5 ? 200448 : siren_oW(L) + 65536); }
static_assert(siren_oB(5) + 8 == kSirenNParams, "layout");

// what the fused evaluation reads: FP32 master parameters (first layer, biases) and the
// BF16 copies of W2..W4 ([3][256][256]) and of W5 padded to 16 rows, with their TMA maps
struct SirenNet {
    const float *P;
    const void *Wh;
    const void *W5p;
    float omega0;
    int *err;  // device error word of the evaluation kernel (0 = none)
    CUtensorMap map_wh, map_w5;
};

// Output of a fused evaluation. Raw mode (field == null): y (n x 8) and, if J is set,
// J (n x 8 x 3) = dy/dx. Field mode: per point `field_stride` floats starting with the
// physical B (3), E (3), dB[d][c] = dB_c/dR_d (9), dE[d][c] (9), from the product rule on
// B = B_scale y_B (1 AU / r)^2, E = E_scale y_E (1 AU / r).
struct SirenOut {
    float *y, *J;
    float *field;
    int field_stride;
    double B_scale, E_scale;
};

// Inputs: n points p (n x 3); the network sees x = x_scale p and the field mode's physical
// position is R = pos_scale p. n_dev, if set, holds the point count on the device (read by
// the kernel; n is then the capacity of the buffers).
struct SirenIn {
    const float *p;
    int64_t n;
    const int32_t *n_dev;
    float x_scale, pos_scale;
};

// build the two tensor maps of net (Wh and W5p must be set)
cudaError_t siren_maps(SirenNet &net);
// evaluate the network (and its Jacobian) at the input points (device)
cudaError_t siren_eval(const SirenNet &net, const SirenIn &in, const SirenOut &out, cudaStream_t s);
// CTAs of the fused evaluation per launch (one per SM)
int siren_eval_grid(int64_t n);
} // namespace gcs
