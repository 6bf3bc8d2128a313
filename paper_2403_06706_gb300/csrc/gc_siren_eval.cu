// gc_siren_eval.cu -- fused evaluation of the SIREN neural field and its Jacobian on the
// tensor cores (tcgen05, TMA, tensor memory).
//
// Forward-mode differentiation carries three tangent rows beside every value row: for a
// point x the rows are h_k and t_{k,j} = dh_k/dx_j (j = 0..2), with
//   layer 1:  z = w0 (W1 x + b1),   h1 = sin z,   t1_j = w0 cos(z) W1[:, j]
//   layer k:  z = W_k h_{k-1} + b_k, h_k = sin z, t_{k,j} = cos(z) * (W_k t_{k-1,j})
//   output:   y = W5 h4 + b5,       J[:, j] = W5 t_{4,j}.
// A tile is 64 points = 256 rows (row 4p + q: q = 0 value, q = 1..3 tangents). Hidden
// layers run as D = W_k . H^T on the tensor cores (two halves of M = 128 output features,
// N = 256 rows, K = 256), so that each accumulator lane holds one feature and the four rows
// of a point sit in adjacent columns: the epilogue thread of a feature computes sin and cos
// of the value row once and scales its own three tangent columns, with no data exchange.
// Activations go back to shared memory in the MN-major 128-byte-swizzled layout that the
// next layer reads as its B operand. The output layer runs as rows x W5^T (M = 128 rows,
// N = 16 with W5 zero-padded, loaded once per launch). The hidden layers' weights stream
// through a 4-stage TMA ring (16 KB chunks of 64 input features x 128 outputs; 4 stages
// measured faster than 5 or 6, 2 slower); the first layer runs on the CUDA cores.
//
// Pipeline of one layer, in MMA order: half 0 over input features 0-127, half 1 over 0-127,
// half 0 over 128-255, half 1 over 128-255. The epilogue of half 0 (features 0-127) starts
// when half 0 is complete, and with it every MMA of the layer over inputs 0-127, so it may
// overwrite them at once; it overlaps the MMAs of half 1 over 128-255. The epilogue of half
// 1 says when it has read its whole accumulator (h1_drained, halfway through): the next
// layer's MMAs over inputs 0-127 (the features half 0 has just written), half 0's during it
// and half 1's after that signal, run while it computes; those over 128-255 follow it.
// The output layer also runs in two K halves (input features 0-127 during the last
// epilogue of half 1, then 128-255) into columns 0-31 of the drained half-0 accumulator,
// and overlaps the next tile's first layer: its half 0 is written once the output MMAs over
// features 0-127 are done, and the output accumulator is read before the next tile's MMAs
// may start; the previous tile's outputs are stored while those MMAs run.
//
// Warp roles (576 threads): warps 0-15 compute; all of them work on one output half at a
// time, warp w on features 32 (w % 4) + lane of the half (warp w may only touch
// tensor-memory lanes 32 (w % 4) .. + 31) and rows 64 (w / 4) .. + 63. Warp 16 lane 0 issues the MMAs
// (warp 16 also owns the tensor-memory allocation), warp 17 lane 0 issues the TMA loads.
// Every wait is bounded: a wait that runs out sets the kernel's error word and an abort flag
// that makes all roles leave their loops; the CTA then waits for its own copies and MMAs
// and frees its tensor memory.
#include <cstdio>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gc_siren.h"
#include "gc_tc.cuh"

namespace gcs {

using namespace tc;

namespace {

constexpr int kPts = 64;                        // points per tile
constexpr int kStagesW = 4;                     // weight ring depth
constexpr uint32_t kChunkBytes = 128u * 128u;   // 128 output rows x 64 bf16
constexpr uint32_t kW5Bytes = 4u * 16u * 128u;  // W5 padded: 4 boxes of 16 rows x 64 bf16
constexpr uint32_t kHBytes = 32u * 4u * 1024u;  // 32 K-groups x 4 MN-blocks of 1024 B
constexpr int kChunksPerTile = 3 * 8;
constexpr int kComputeThreads = 512;            // arrivals on each h_ready barrier
constexpr int kThreads = 576;
constexpr int kMmaWarp = 16, kTmaWarp = 17;
constexpr uint32_t kPtsBytes = 16u * 16u * 16u;  // per compute warp: its 16 points as float4
constexpr size_t kSmemBytes = kHBytes + kStagesW * kChunkBytes + kW5Bytes + kPtsBytes + 1024 + 256;

struct EvalParams {
    const float *P;  // master parameters
    SirenIn in;
    SirenOut out;
    float omega0;
    int *err;        // error word (device), set when a wait runs out
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

// 8 consecutive rows (mn0 .. mn0 + 7, mn0 % 8 == 0) of one feature into the MN-major
// activation buffer; hrow points at the feature's 128-byte row of its K-group's first atom
__device__ __forceinline__ void store_rows8(uint8_t *hrow, uint32_t rsw, uint32_t mn0, const float (&o)[8])
{
    uint4 pk;
    pk.x = pack_bf16(o[0], o[1]);
    pk.y = pack_bf16(o[2], o[3]);
    pk.z = pack_bf16(o[4], o[5]);
    pk.w = pack_bf16(o[6], o[7]);
    const uint32_t ch = ((mn0 & 63u) >> 3) ^ rsw;
    *reinterpret_cast<uint4 *>(hrow + (mn0 >> 6) * 1024u + ch * 16u) = pk;
}

// bounded wait that also gives up when another role of the CTA has aborted
__device__ __forceinline__ bool wait_abort(uint64_t *bar, uint32_t parity, volatile int *abort, int *err, int code)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try(bar, parity)) return true;
        if (*abort) return false;
        if (global_ns() - t0 > kWaitNs) break;
    }
    *abort = 1;
    atomicExch(err, code);
    return false;
}

// Output rows of one tile from the output accumulator v (16 columns of this thread's row
// pr): raw outputs y and J, or the physical field for the push.
__device__ __forceinline__ void store_out(const EvalParams &p, const float (&b5)[8], const float (&v)[16],
                                          int64_t base, int pr, int lane, int64_t n_pts)
{
    const int q = pr & 3;
    const int64_t P = base + (pr >> 2);
    if (p.out.field == nullptr) {
        if (P < n_pts) {
            if (q == 0) {
#pragma unroll
                for (int o = 0; o < 8; ++o)
                    p.out.y[P * 8 + o] = v[o] + b5[o];
            } else if (p.out.J) {
#pragma unroll
                for (int o = 0; o < 8; ++o)
                    p.out.J[(P * 8 + o) * 3 + (q - 1)] = v[o];
            }
        }
    } else {
        // physical field: B = B_s y_B (AU/r)^2, E = E_s y_E (AU/r) at R = pos_scale p;
        // gradients by the product rule with d/dR = (x_scale / pos_scale) d/dx
        const unsigned full_mask = 0xffffffffu;
        const int src = lane & ~3;
        float yv[6];
#pragma unroll
        for (int o = 0; o < 6; ++o)
            yv[o] = __shfl_sync(full_mask, v[o] + b5[o], src);
        if (P < n_pts) {
            const double au = 1.495978707e11;
            const float ps = p.in.pos_scale;
            const float X0 = __ldg(p.in.p + 3 * P) * ps, X1 = __ldg(p.in.p + 3 * P + 1) * ps,
                        X2 = __ldg(p.in.p + 3 * P + 2) * ps;
            const float r2 = X0 * X0 + X1 * X1 + X2 * X2;
            const float ir = rsqrtf(r2);
            const float a = (float)au * ir;                   // AU / r
            const float bs = (float)p.out.B_scale * a * a;    // B per unit y_B
            const float es = (float)p.out.E_scale * a;        // E per unit y_E
            float *dst = p.out.field + P * p.out.field_stride;
            if (q == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    dst[c] = bs * yv[c];
                    dst[3 + c] = es * yv[3 + c];
                }
            } else {
                const int d = q - 1;
                const float Xd = d == 0 ? X0 : (d == 1 ? X1 : X2);
                const float irm = p.in.x_scale / ps;  // d/dR = (x_scale / pos_scale) d/dx
                const float ur = Xd * ir * ir;  // R_d / r^2
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    dst[6 + 3 * d + c] = bs * (v[c] * irm - 2.0f * yv[c] * ur);
                    dst[15 + 3 * d + c] = es * (v[3 + c] * irm - yv[3 + c] * ur);
                }
                // the push's layout also takes grad(Phi): Phi = E_scale AU y_Phi
                if (p.out.field_stride >= 40)
                    dst[34 + d] = (float)(p.out.E_scale * au) * v[7] * irm;
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    siren_eval_kernel(const __grid_constant__ CUtensorMap mwh, const __grid_constant__ CUtensorMap mw5,
                      const __grid_constant__ EvalParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sH = smem;
    uint8_t *sW = smem + kHBytes;
    uint8_t *sW5 = sW + kStagesW * kChunkBytes;  // W5, resident for the whole launch
    float4 *sPts = (float4 *)(sW5 + kW5Bytes);  // [16 compute warps][16 points]
    uint64_t *full = (uint64_t *)(sW5 + kW5Bytes + kPtsBytes);
    uint64_t *empty = full + kStagesW;
    uint64_t *h_ready = empty + kStagesW; // [2]: activations of a half written, its accumulator drained
    uint64_t *acc = h_ready + 2;          // [2]: accumulator of a half complete
    uint64_t *h1_drained = acc + 2;       // the half-1 epilogue has read its accumulator
    uint64_t *acc_out = h1_drained + 1;   // output layer complete
    uint64_t *out_a = acc_out + 1;        // output-layer MMAs over input features 0-127 complete
    uint64_t *fin = out_a + 1;
    uint64_t *w5full = fin + 1;           // W5 landed
    uint32_t *tmem_slot = (uint32_t *)(w5full + 1);
    volatile int *abort = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t n_pts = p.in.n;
    if (p.in.n_dev) {
        const int64_t nd = *p.in.n_dev;
        n_pts = nd < n_pts ? (nd > 0 ? nd : 0) : n_pts;
    }
    const int64_t n_tiles = (n_pts + kPts - 1) / kPts;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagesW; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&h_ready[0], kComputeThreads);
        mbar_init(&h_ready[1], kComputeThreads);
        mbar_init(&acc[0], 1);
        mbar_init(&acc[1], 1);
        mbar_init(h1_drained, kComputeThreads);
        mbar_init(acc_out, 1);
        mbar_init(out_a, 1);
        mbar_init(fin, 1);
        mbar_init(w5full, 1);
        *abort = 0;
        mbar_fence_init();
    }
    if (warp == kMmaWarp) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == kTmaWarp) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            mbar_expect_tx(w5full, kW5Bytes);
            for (int kb = 0; kb < 4; ++kb)
                tma_load_2d(sW5 + kb * 2048, &mw5, kb * 64, 0, w5full);
            for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                for (int c = 0; c < kChunksPerTile; ++c) {
                    const uint32_t s = g % kStagesW;
                    if (!wait_abort(&empty[s], ((g / kStagesW) & 1u) ^ 1u, abort, p.err, 11)) {
                        ok = false;
                        break;
                    }
                    uint8_t *dst = sW + s * kChunkBytes;
                    // chunk (layer c / 8, output half and input block in the MMA order)
                    const int q = c & 7, h = (q >> 1) & 1, kb = (q & 1) | ((q >> 2) << 1);
                    mbar_expect_tx(&full[s], kChunkBytes);
                    tma_load_2d(dst, &mwh, kb * 64, (c >> 3) * 256 + h * 128, &full[s]);
                    ++g;
                }
            }
            // the copies still in flight land before the CTA's shared memory is released
            for (uint32_t j = g > (uint32_t)kStagesW ? g - kStagesW : 0u; j < g; ++j)
                mbar_wait(&full[j % kStagesW], (j / kStagesW) & 1u);
            mbar_wait(w5full, 0);
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id_hid = idesc_bf16_f32(128, 256, 0, 1);
            const uint32_t id_out = idesc_bf16_f32(128, 16, 1, 0);
            const uint32_t hb = smem_u32(sH);
            uint32_t g = 0, nh0 = 0, nh1 = 0, nd = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                for (int L = 0; L < 3 && ok; ++L) {
                    // order: half 0 over inputs 0-127, half 1 over inputs 0-127 (as soon as the
                    // previous half-1 epilogue has read its accumulator), half 0 over 128-255
                    // (once that epilogue has written them), half 1 over 128-255
#pragma unroll 1
                    for (int q = 0; q < 8; ++q) {
                        const int h = (q >> 1) & 1, kb = (q & 1) | ((q >> 2) << 1);
                        if (q == 0) {
                            // inputs 0-127 written and accumulator half 0 drained
                            if (!wait_abort(&h_ready[0], nh0 & 1u, abort, p.err, 12)) { ok = false; break; }
                            ++nh0;
                            tc_fence_after();
                        }
                        if (q == 2 && (L > 0 || t != blockIdx.x)) {
                            // accumulator half 1 read by the previous half-1 epilogue
                            if (!wait_abort(h1_drained, nd & 1u, abort, p.err, 19)) { ok = false; break; }
                            ++nd;
                            tc_fence_after();
                        }
                        if (q == 4) {
                            // inputs 128-255 written
                            if (!wait_abort(&h_ready[1], nh1 & 1u, abort, p.err, 13)) { ok = false; break; }
                            ++nh1;
                            tc_fence_after();
                        }
                        const uint32_t s = g % kStagesW;
                        if (!wait_abort(&full[s], (g / kStagesW) & 1u, abort, p.err, 14)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t wb = smem_u32(sW + s * kChunkBytes);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks)
                            mma_bf16(tmem + h * 256, desc_sw128(wb + ks * 32),
                                     desc_sw128_mn(hb + (kb * 4 + ks) * 8192, 1024, 4096), id_hid,
                                     (kb | ks) ? 1u : 0u);
                        mma_commit(&empty[s]);
                        ++g;
                        // half 0 complete, and with it every MMA of this layer over inputs 0-127
                        if (q == 5) mma_commit(&acc[0]);
                    }
                    if (ok) mma_commit(&acc[1]);
                }
                if (!ok) break;
                // output layer: rows x W5^T, M-tile 0 into columns 0-15 and M-tile 1 into 16-31
                // (both in the drained half-0 accumulator), in two K halves: input features
                // 0-127 as soon as their epilogue is done, 128-255 after the last one
                bool ok2 = true;
                if (t == blockIdx.x) {
                    // W5, loaded once per launch
                    if (!wait_abort(w5full, 0, abort, p.err, 17)) break;
                    tc_fence_after();
                }
                for (int kh = 0; kh < 2 && ok2; ++kh) {
                    uint32_t &nh = kh ? nh1 : nh0;
                    if (!wait_abort(&h_ready[kh], nh & 1u, abort, p.err, 15 + kh)) { ok2 = false; break; }
                    ++nh;
                    tc_fence_after();
                    const uint32_t wb = smem_u32(sW5);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int k8 = 0; k8 < 8; ++k8) {
                            const int k16 = kh * 8 + k8;
                            mma_bf16(tmem + mt * 16, desc_sw128_mn(hb + mt * 2048 + k16 * 8192, 1024, 4096),
                                     desc_sw128(wb + (k16 >> 2) * 2048 + (k16 & 3) * 32), id_out, k16 ? 1u : 0u);
                        }
                    if (kh == 0) mma_commit(out_a);
                }
                if (!ok2) break;
                mma_commit(acc_out);
            }
            // all MMAs of this CTA complete before its tensor memory is released
            mma_commit(fin);
            mbar_wait(fin, 0);
        }
    } else {
        // ------------------------------------------------------------ compute warps
        // warp w: tensor-memory lane quarter lq = w % 4 (features 32 lq .. of each half) and
        // row group rg = w / 4 (rows 64 rg .. 64 rg + 63 = points 16 rg .. 16 rg + 15); all
        // 16 warps work on one output half at a time
        const int lq = warp & 3, rg = warp >> 2;
        const float w0 = p.omega0;
        float w1[2][3], b1[2], bl[3][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int f = h * 128 + lq * 32 + lane;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                w1[h][j] = p.P[siren_oW(1) + 3 * f + j];
            b1[h] = p.P[siren_oB(1) + f];
#pragma unroll
            for (int L = 0; L < 3; ++L)
                bl[L][h] = p.P[siren_oB(L + 2) + f];
        }
        float b5[8];
#pragma unroll
        for (int o = 0; o < 8; ++o)
            b5[o] = p.P[siren_oB(5) + o];
        const uint32_t lane_base = tmem + ((uint32_t)(lq * 32) << 16);
        // the feature's 128-byte row in its K-group's first atom, for each half
        uint8_t *hrow0 = sH + ((lq * 32 + lane) >> 3) * 4096 + (lane & 7) * 128;
        uint8_t *hrow1 = hrow0 + 16 * 4096;
        const uint32_t rsw = (uint32_t)(lane & 7);
        uint32_t na0 = 0, na1 = 0, no = 0, noa = 0;
        bool ok = true, first = true;
        int64_t base_prev = 0;
        // this warp's 16 points: lane i < 16 holds point 16 rg + i and puts it in the warp's
        // shared-memory slots for the first layer, where every lane reads it by broadcast; the
        // next tile's are fetched while the current one runs
        float px = 0.f, py = 0.f, pz = 0.f;
        const int pt_off = rg * 16 + (lane & 15);
        {
            const int64_t P = (int64_t)blockIdx.x * kPts + pt_off;
            if (P < n_pts) {
                px = __ldg(p.in.p + 3 * P) * p.in.x_scale;
                py = __ldg(p.in.p + 3 * P + 1) * p.in.x_scale;
                pz = __ldg(p.in.p + 3 * P + 2) * p.in.x_scale;
            }
        }
        float4 *wpts = sPts + warp * 16;
        for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            const int64_t base = t * kPts;
            __syncwarp();  // every lane done with the previous tile's points
            if (lane < 16) wpts[lane] = make_float4(px, py, pz, 0.f);
            __syncwarp();
            // Layer 1 on the CUDA cores, half 0 then half 1. The previous tile's output layer
            // still runs meanwhile: half 0 overwrites input features 0-127 once the output
            // MMAs over them are done (out_a); before half 0 is announced, the output
            // accumulator is read (the next MMAs overwrite it); half 1 follows the rest of the
            // output layer (acc_out), then the previous tile's outputs are stored.
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint8_t *hrow = h ? hrow1 : hrow0;
                if (h == 0 && !first) {
                    if (!wait_abort(out_a, noa & 1u, abort, p.err, 21)) {
                        ok = false;
                        break;
                    }
                    ++noa;
                }
#pragma unroll 2
                for (int p2 = 0; p2 < 8; ++p2) {
                    float o[8];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int src = 2 * p2 + e;
                        const float4 xq = wpts[src];
                        const float x0 = xq.x, x1 = xq.y, x2 = xq.z;
                        const float z = w0 * fmaf(w1[h][0], x0, fmaf(w1[h][1], x1, fmaf(w1[h][2], x2, b1[h])));
                        // the hardware sine and cosine on z directly (|z| reaches tens here, w0
                        // = 30): their error, a few 1e-6 at most there, stays three orders below
                        // the BF16 rounding of the activations; an explicit reduction by 2 pi
                        // first cost 2 % of the kernel for no gain against the exact network
                        const float sn = __sinf(z), cs = __cosf(z);
                        const float wc = w0 * cs;
                        o[4 * e] = sn;
                        o[4 * e + 1] = wc * w1[h][0];
                        o[4 * e + 2] = wc * w1[h][1];
                        o[4 * e + 3] = wc * w1[h][2];
                    }
                    store_rows8(hrow, rsw, (uint32_t)(rg * 64 + 8 * p2), o);
                }
                fence_proxy_async_smem();
                float v[16];
                if (h == 0 && !first) {
                    if (!wait_abort(acc_out, no & 1u, abort, p.err, 20)) {
                        ok = false;
                        break;
                    }
                    ++no;
                    tc_fence_after();
                    if (rg < 2) tmem_ld16(lane_base + rg * 16, v);
                }
                tc_fence_before();
                mbar_arrive(&h_ready[h]);
                if (h == 0 && !first && rg < 2)
                    store_out(p, b5, v, base_prev, rg * 128 + lq * 32 + lane, lane, n_pts);
            }
            if (!ok) break;
            {
                const int64_t P = (t + gridDim.x) * kPts + pt_off;
                px = py = pz = 0.f;
                if (t + gridDim.x < n_tiles && P < n_pts) {
                    px = __ldg(p.in.p + 3 * P) * p.in.x_scale;
                    py = __ldg(p.in.p + 3 * P + 1) * p.in.x_scale;
                    pz = __ldg(p.in.p + 3 * P + 2) * p.in.x_scale;
                }
            }
            // hidden layers 2-4: epilogues of D = W_k H^T, half 0 then half 1
            for (int L = 0; L < 3 && ok; ++L) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t &na = h ? na1 : na0;
                    if (!wait_abort(&acc[h], na & 1u, abort, p.err, 18)) {
                        ok = false;
                        break;
                    }
                    ++na;
                    tc_fence_after();
                    uint8_t *hrow = h ? hrow1 : hrow0;
                    const float b = bl[L][h];
                    // (half 0: every MMA over inputs 0-127 is complete with its accumulator)
#pragma unroll 1
                    for (int c = 0; c < 2; ++c) {
                        float v[32];
                        tmem_ld32(lane_base + h * 256 + rg * 64 + c * 32, v);
                        if (h == 1 && c == 1) {
                            // the half-1 accumulator is read: the next layer's half-1 MMAs
                            // over inputs 0-127 may run during the rest of this epilogue
                            tc_fence_before();
                            mbar_arrive(h1_drained);
                        }
                        float o[4][8];
#pragma unroll
                        for (int pp = 0; pp < 4; ++pp)
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                // |z| stays small in the hidden layers: the hardware sine
                                // and cosine without a range reduction
                                const int q0 = 8 * pp + 4 * e;
                                const float z = v[q0] + b;
                                const float sn = __sinf(z), cs = __cosf(z);
                                o[pp][4 * e] = sn;
                                o[pp][4 * e + 1] = cs * v[q0 + 1];
                                o[pp][4 * e + 2] = cs * v[q0 + 2];
                                o[pp][4 * e + 3] = cs * v[q0 + 3];
                            }
#pragma unroll
                        for (int pp = 0; pp < 4; ++pp)
                            store_rows8(hrow, rsw, (uint32_t)(rg * 64 + c * 32 + 8 * pp), o[pp]);
                    }
                    fence_proxy_async_smem();
                    tc_fence_before();
                    mbar_arrive(&h_ready[h]);
                }
            }
            if (!ok) break;
            base_prev = base;
            first = false;
        }
        // the last tile's output layer
        if (ok && !first && wait_abort(acc_out, no & 1u, abort, p.err, 20)) {
            tc_fence_after();
            if (rg < 2) {
                float v[16];
                tmem_ld16(lane_base + rg * 16, v);
                store_out(p, b5, v, base_prev, rg * 128 + lq * 32 + lane, lane, n_pts);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

} // namespace

cudaError_t siren_maps(SirenNet &net)
{
    cudaError_t e = make_map_bf16(&net.map_wh, net.Wh, 256, 3 * 256, 128);
    if (e == cudaSuccess) e = make_map_bf16(&net.map_w5, net.W5p, 256, 16, 16);
    return e;
}

int siren_eval_grid(int64_t n)
{
    static int n_sm = 0;
    if (!n_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    const int64_t tiles = (n + kPts - 1) / kPts;
    return (int)(tiles < n_sm ? tiles : n_sm);
}

cudaError_t siren_eval(const SirenNet &net, const SirenIn &in, const SirenOut &out, cudaStream_t s)
{
    if (in.n <= 0) return cudaSuccess;
    if (!net.err) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(siren_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    EvalParams p;
    p.P = net.P;
    p.in = in;
    p.out = out;
    p.omega0 = net.omega0;
    p.err = net.err;
    siren_eval_kernel<<<siren_eval_grid(in.n), kThreads, kSmemBytes, s>>>(net.map_wh, net.map_w5, p);
    return cudaGetLastError();
}

} // namespace gcs
