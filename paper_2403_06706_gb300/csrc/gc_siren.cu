// gc_siren.cu -- BF16 tensor-core (tcgen05) kernels of the neural field.
//
// Part 1: a general GEMM C = op(A) op(B)^T with bf16 operands: A is M x K stored K-major
// (row-major M x K) or MN-major (row-major K x M), B likewise N x K or K x N. FP32
// accumulation in tensor memory, TMA loads through a 4-stage mbarrier pipeline, and split-K
// with FP32 atomics for long K. One CTA of four warps computes a 128 x BN tile: thread 0
// issues the TMA loads and the MMAs, all four warps drain the accumulator (warp w owns TMEM
// lanes 32w..32w+31, i.e. rows 32w..32w+31 of the tile). MN-major operands arrive as
// 64 x 64 boxes, one per 64 rows (or columns) of the tile.
#include <cstdio>
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "../../include/gcpush.h"
#include "gc_internal.h"
#include "gc_siren.h"
#include "gc_tc.cuh"

namespace gcs {

using namespace tc;

// set by a kernel whose bounded wait ran out (0 = no error); read after the launch
__device__ int g_tc_error;

__device__ __forceinline__ void report(int code) { atomicExch(&g_tc_error, code); }

constexpr int kBM = 128, kBK = 64, kStages = 4;

template <int BN>
constexpr size_t gemm_smem_bytes()
{
    return (size_t)kStages * (kBM * 128 + BN * 128) + 1024 + 256;
}

// one stage of operand X: rows x 64 K (K-major, one box) or 64-element MN blocks x 64 K rows
template <bool MN>
__device__ __forceinline__ void load_operand(uint8_t *dst, const CUtensorMap *m, int k, int r0, int rows,
                                             uint64_t *bar)
{
    if (!MN) {
        tma_load_2d(dst, m, k, r0, bar);
    } else {
        for (int j = 0; j < rows / 64; ++j)
            tma_load_2d(dst + j * 8192, m, r0 + 64 * j, k, bar);
    }
}

template <bool MN>
__device__ __forceinline__ uint64_t operand_desc(uint32_t base, int k16)
{
    return MN ? desc_sw128_mn(base + (uint32_t)k16 * 2048u, 8192u, 1024u) : desc_sw128(base + (uint32_t)k16 * 32u);
}

template <int BN, bool AMN, bool BMN>
__global__ void __launch_bounds__(128, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                     float *__restrict__ C, int M, int N, int K, int ldc, int k_per_split, int atomic)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + kStages * kBM * 128;
    uint64_t *full = (uint64_t *)(sB + kStages * BN * 128);
    uint64_t *empty = full + kStages;
    uint64_t *done = empty + kStages;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    __shared__ int s_ok;

    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int k_lo = blockIdx.z * k_per_split;
    const int k_hi = min(K, k_lo + k_per_split);
    const int nkb = (k_hi - k_lo) / kBK;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        mbar_fence_init();
        s_ok = 1;
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, BN < 32 ? 32 : BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        const uint32_t idesc = idesc_bf16_f32(kBM, BN, AMN, BMN);
        const uint32_t tx = (uint32_t)(kBM + BN) * 128u;
        const int pro = nkb < kStages ? nkb : kStages;
        for (int kb = 0; kb < pro; ++kb) {
            mbar_expect_tx(&full[kb], tx);
            load_operand<AMN>(sA + kb * kBM * 128, &ta, k_lo + kb * kBK, m0, kBM, &full[kb]);
            load_operand<BMN>(sB + kb * BN * 128, &tb, k_lo + kb * kBK, n0, BN, &full[kb]);
        }
        int issued = pro;
        bool ok = true;
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int s = kb % kStages;
            if (!mbar_wait(&full[s], (kb / kStages) & 1)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + s * kBM * 128), b0 = smem_u32(sB + s * BN * 128);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
                mma_bf16(tmem, operand_desc<AMN>(a0, k), operand_desc<BMN>(b0, k), idesc, (kb | k) ? 1u : 0u);
            mma_commit(&empty[s]);
            // refill the stage consumed one iteration ago (its MMAs have had time to finish)
            const int kn = kb - 1 + kStages;
            if (kb >= 1 && kn < nkb) {
                const int sp = (kb - 1) % kStages;
                if (!mbar_wait(&empty[sp], ((kb - 1) / kStages) & 1)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(&full[sp], tx);
                load_operand<AMN>(sA + sp * kBM * 128, &ta, k_lo + kn * kBK, m0, kBM, &full[sp]);
                load_operand<BMN>(sB + sp * BN * 128, &tb, k_lo + kn * kBK, n0, BN, &full[sp]);
                ++issued;
            }
        }
        if (ok) {
            mma_commit(done);
        } else {
            report(1);
            s_ok = 0;
            // let the copies already in flight land before the CTA's memory is released
            for (int j = 0; j < issued; ++j)
                mbar_wait(&full[j % kStages], (j / kStages) & 1);
            mbar_arrive(done);
        }
    }
    if (!mbar_wait(done, 0)) {
        report(2);
        atomicExch(&s_ok, 0);
    }
    tc_fence_after();
    __syncwarp();
    if (nkb > 0) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row < M && s_ok) {
                // N is a multiple of the tile width and ldc of 4: whole float4 chunks
                float4 *dst = reinterpret_cast<float4 *>(C + (size_t)row * ldc + n0 + c0);
                if (atomic) {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        atomicAdd(dst + j, make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        tmem_dealloc(tmem, BN < 32 ? 32 : BN);
}

// ------------------------------------------------------------------------------- host
namespace {
std::mutex g_enc_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
} // namespace

cudaError_t encode_fn(PFN_cuTensorMapEncodeTiled_v12000 *out)
{
    std::lock_guard<std::mutex> lk(g_enc_mu);
    if (!g_encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return e != cudaSuccess ? e : cudaErrorNotSupported;
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    *out = g_encode;
    return cudaSuccess;
}

cudaError_t make_map_bf16(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer, uint32_t box_outer)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc;
    cudaError_t e = encode_fn(&enc);
    if (e != cudaSuccess) return e;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {inner * 2};
    const cuuint32_t box[2] = {64, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int read_error(cudaStream_t s)
{
    int v = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbolAsync(g_tc_error, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
    }
    return v;
}

template <int BN, bool AMN, bool BMN>
static cudaError_t launch_gemm(const CUtensorMap &ma, const CUtensorMap &mb, float *C, int M, int N, int K,
                               int ldc, int splits, int atomic, cudaStream_t s)
{
    const size_t smem = gemm_smem_bytes<BN>();
    cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel<BN, AMN, BMN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int kps = ((K / kBK + splits - 1) / splits) * kBK;
    dim3 grid((M + kBM - 1) / kBM, (N + BN - 1) / BN, (K + kps - 1) / kps);
    gemm_bf16_kernel<BN, AMN, BMN><<<grid, 128, smem, s>>>(ma, mb, C, M, N, K, ldc, kps, atomic);
    return cudaGetLastError();
}

template <int BN>
static cudaError_t launch_gemm_any(const CUtensorMap &ma, const CUtensorMap &mb, int a_mn, int b_mn, float *C,
                                   int M, int N, int K, int splits, int atomic, cudaStream_t s)
{
    if (!a_mn && !b_mn) return launch_gemm<BN, false, false>(ma, mb, C, M, N, K, N, splits, atomic, s);
    if (!a_mn && b_mn) return launch_gemm<BN, false, true>(ma, mb, C, M, N, K, N, splits, atomic, s);
    if (a_mn && !b_mn) return launch_gemm<BN, true, false>(ma, mb, C, M, N, K, N, splits, atomic, s);
    return launch_gemm<BN, true, true>(ma, mb, C, M, N, K, N, splits, atomic, s);
}

cudaError_t gemm_bf16(const void *A, int a_mn, const void *B, int b_mn, float *C, int M, int N, int K,
                      int splits, int atomic, cudaStream_t s)
{
    const int BN = (N % 256 == 0) ? 256 : 128;
    CUtensorMap ma, mb;
    cudaError_t e = a_mn ? make_map_bf16(&ma, A, (uint64_t)M, (uint64_t)K, 64)
                         : make_map_bf16(&ma, A, (uint64_t)K, (uint64_t)M, kBM);
    if (e == cudaSuccess)
        e = b_mn ? make_map_bf16(&mb, B, (uint64_t)N, (uint64_t)K, 64)
                 : make_map_bf16(&mb, B, (uint64_t)K, (uint64_t)N, (uint32_t)BN);
    if (e != cudaSuccess) return e;
    cudaGetLastError();
    if (BN == 256) return launch_gemm_any<256>(ma, mb, a_mn, b_mn, C, M, N, K, splits, atomic, s);
    return launch_gemm_any<128>(ma, mb, a_mn, b_mn, C, M, N, K, splits, atomic, s);
}

} // namespace gcs

// ------------------------------------------------------------------------------- C ABI
extern "C" int gc_gemm_bf16(const void *A, int a_mn, const void *B, int b_mn, float *C, int M, int N, int K,
                            int split_k, int accumulate, void *stream)
{
    char buf[256];
    if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || split_k < 1 || (a_mn | 1) != 1 || (b_mn | 1) != 1) {
        gcp::set_last_error("gc_gemm_bf16: bad argument");
        return GC_ERR_INVALID;
    }
    if (K % 64 != 0 || N % 128 != 0 || M % 128 != 0) {
        gcp::set_last_error("gc_gemm_bf16: need M % 128 == 0, N % 128 == 0, K % 64 == 0");
        return GC_ERR_INVALID;
    }
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) & 15) {
        gcp::set_last_error("gc_gemm_bf16: A, B and C must be 16-byte aligned");
        return GC_ERR_INVALID;
    }
    if (split_k > 1 && !accumulate) {
        gcp::set_last_error("gc_gemm_bf16: split-K needs accumulate = 1");
        return GC_ERR_INVALID;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = gcs::gemm_bf16(A, a_mn, B, b_mn, C, M, N, K, split_k, accumulate, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        snprintf(buf, sizeof(buf), "gc_gemm_bf16: %s", cudaGetErrorString(e));
        gcp::set_last_error(buf);
        return GC_ERR_CUDA;
    }
    const int te = gcs::read_error(s);
    if (te) {
        snprintf(buf, sizeof(buf), "gc_gemm_bf16: a pipeline wait ran out (code %d)", te);
        gcp::set_last_error(buf);
        return GC_ERR_DEVICE_ANOMALY;
    }
    return GC_OK;
}

extern "C" int gc_gemm_bf16_tn(const void *A, const void *B, float *C, int M, int N, int K, int split_k,
                               int accumulate, void *stream)
{
    return gc_gemm_bf16(A, 0, B, 0, C, M, N, K, split_k, accumulate, stream);
}
