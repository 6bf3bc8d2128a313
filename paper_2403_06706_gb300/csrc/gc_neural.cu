// gc_neural.cu -- the neural field: parameters on the device, the training targets, the
// training's forward and backward passes, and Adam.
//
// Network and conventions (SIREN, Sitzmann et al. 2020): x = R / r_max; z1 = w0 (W1 x + b1),
// h_k = sin z_k, z_k = W_k h_{k-1} + b_k (k = 2..4), y = W5 h4 + b5. Outputs are the grid's
// eight channels scaled to O(1): B and |B| times (r / 1 AU)^2 / B_scale, E times
// (r / 1 AU) / E_scale, Phi / (E_scale 1 AU). The training minimises the mean squared error
// over samples and channels (Kingma & Ba 2015 for Adam) with the same arithmetic as the
// fused evaluation: W2..W5 and the activations h_1..h_4 in BF16, FP32 accumulation, FP32
// first layer and biases. Products with W2..W4 (forward, dW = dZ^T H, dH = dZ W) run on the
// tensor-core GEMM; the first and last layers and the elementwise steps run here.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gc_neural.h"
#include "gc_siren.h"

namespace gcn {

using gcs::kSirenNParams;
using gcs::siren_oB;
using gcs::siren_oW;

namespace {

constexpr double kAU = 1.495978707e11;
constexpr double kPi = 3.14159265358979323846;

inline int blocks_for(int64_t n, int block, int cap = 152 * 16)
{
    const int64_t b = (n + block - 1) / block;
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// BF16 copy of parameter i if it belongs to W2..W5
__device__ __forceinline__ void put_bf16(int64_t i, float p, __nv_bfloat16 *Wh, __nv_bfloat16 *W5p)
{
#pragma unroll
    for (int L = 2; L <= 4; ++L) {
        const int64_t o = siren_oW(L);
        if (i >= o && i < o + 65536) {
            Wh[(int64_t)(L - 2) * 65536 + (i - o)] = __float2bfloat16_rn(p);
            return;
        }
    }
    if (i >= siren_oW(5) && i < siren_oW(5) + 2048)
        W5p[i - siren_oW(5)] = __float2bfloat16_rn(p);
}

__global__ void k_to_bf16(const float *__restrict__ P, __nv_bfloat16 *Wh, __nv_bfloat16 *W5p)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < kSirenNParams;
         i += (int64_t)gridDim.x * blockDim.x)
        put_bf16(i, P[i], Wh, W5p);
}

// Adam (Kingma & Ba 2015) with bias corrections bc1 = 1 - beta1^t, bc2 = 1 - beta2^t
__global__ void k_adam(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                       float *__restrict__ V, float lr, float b1, float b2, float eps, float bc1, float bc2,
                       __nv_bfloat16 *Wh, __nv_bfloat16 *W5p)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < kSirenNParams;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * M[i] + (1.0f - b1) * g;
        const float v = b2 * V[i] + (1.0f - b2) * g * g;
        M[i] = m;
        V[i] = v;
        const float p = P[i] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        P[i] = p;
        put_bf16(i, p, Wh, W5p);
    }
}

// The eight channels of the trilinear grid interpolant at x (scaled by r_max), scaled as the
// network's outputs. Same cell conventions as the push's gather: node-centred, poles
// included, periodic in phi, clamped to the edge cells.
template <typename T>
__global__ void k_targets(const T *__restrict__ nodes, int n_r, int n_th, int n_ph, double r_min, double dr,
                          const float *__restrict__ x, int64_t n, double r_max, double B_scale, double E_scale,
                          float *__restrict__ out)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const double X = (double)x[3 * q] * r_max, Y = (double)x[3 * q + 1] * r_max, Zc = (double)x[3 * q + 2] * r_max;
        const double rho = sqrt(X * X + Y * Y), r = sqrt(X * X + Y * Y + Zc * Zc);
        const double th = atan2(rho, Zc);
        double ph = atan2(Y, X);
        if (ph < 0) ph += 2.0 * kPi;
        const double xr = (r - r_min) / dr, xt = th / (kPi / (n_th - 1)), xp = ph / (2.0 * kPi / n_ph);
        int i = (int)floor(xr);
        double fr = xr - i;
        if (i < 0) { i = 0; fr = 0; }
        else if (i > n_r - 2) { i = n_r - 2; fr = 1; }
        int j = (int)floor(xt);
        double ft = xt - j;
        if (j < 0) { j = 0; ft = 0; }
        else if (j > n_th - 2) { j = n_th - 2; ft = 1; }
        int k = (int)floor(xp);
        const double fp = xp - k;
        if (k >= n_ph) k -= n_ph;
        if (k < 0) k += n_ph;
        const int k1 = (k + 1 == n_ph) ? 0 : k + 1;
        double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c) {
                    const double w = (a ? fr : 1 - fr) * (b ? ft : 1 - ft) * (c ? fp : 1 - fp);
                    const T *p = nodes + (((int64_t)(c ? k1 : k) * n_th + (j + b)) * n_r + (i + a)) * 8;
                    for (int ch = 0; ch < 8; ++ch)
                        v[ch] += w * (double)p[ch];
                }
        const double a1 = r / kAU;
        const double sb = a1 * a1 / B_scale, se = a1 / E_scale;
        for (int ch = 0; ch < 3; ++ch) {
            out[8 * q + ch] = (float)(v[ch] * sb);
            out[8 * q + 3 + ch] = (float)(v[3 + ch] * se);
        }
        out[8 * q + 6] = (float)(v[6] * sb);
        out[8 * q + 7] = (float)(v[7] / (E_scale * kAU));
    }
}

// first layer: z1 = w0 (W1 x + b1), h1 = sin z1 (rows x 256)
__global__ void k_layer1(const float *__restrict__ P, const float *__restrict__ x, int64_t n, float w0,
                         float *__restrict__ Z, __nv_bfloat16 *__restrict__ H)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * 256;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = q >> 8;
        const int f = (int)(q & 255);
        const float *w = P + siren_oW(1) + 3 * f;
        const float z = w0 * fmaf(w[0], x[3 * row], fmaf(w[1], x[3 * row + 1], fmaf(w[2], x[3 * row + 2],
                                                                                      P[siren_oB(1) + f])));
        Z[q] = z;
        H[q] = __float2bfloat16_rn(sinf(z));
    }
}

// hidden layer L: z = (W_L h)_GEMM + b_L in place, h_L = sin z
__global__ void k_act(const float *__restrict__ P, int L, int64_t n, float *__restrict__ Z,
                      __nv_bfloat16 *__restrict__ H)
{
    const float *b = P + siren_oB(L);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * 256;
         q += (int64_t)gridDim.x * blockDim.x) {
        const float z = Z[q] + b[q & 255];
        Z[q] = z;
        H[q] = __float2bfloat16_rn(sinf(z));
    }
}

// Output layer forward and its backward: y = W5 h4 + b5, r = y - t, loss += sum r^2,
// dy = gscale r, dW5 += dy h4^T, db5 += dy, dz4 = (W5^T dy) cos z4, db4 += dz4. One warp
// per sample (lane: features 8 lane .. 8 lane + 7); block sums go to the gradient by atomics.
__global__ void __launch_bounds__(256) k_out(const float *__restrict__ P, const __nv_bfloat16 *__restrict__ W5p,
                                             const __nv_bfloat16 *__restrict__ H4, const float *__restrict__ Z4,
                                             const float *__restrict__ T, int64_t n, float gscale,
                                             __nv_bfloat16 *__restrict__ dZ4, float *__restrict__ G,
                                             double *__restrict__ loss)
{
    __shared__ float sW[8][256];
    __shared__ float sAcc[2048 + 256 + 8];
    __shared__ double sLoss[8];
    for (int i = threadIdx.x; i < 2048; i += 256)
        sW[i >> 8][i & 255] = __bfloat162float(W5p[i]);
    for (int i = threadIdx.x; i < 2048 + 264; i += 256)
        sAcc[i] = 0.f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, f0 = lane * 8;
    float b5[8];
#pragma unroll
    for (int o = 0; o < 8; ++o)
        b5[o] = P[siren_oB(5) + o];
    float aW[8][8], aB4[8], aB5[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        aB4[o] = 0.f;
        aB5[o] = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            aW[o][i] = 0.f;
    }
    double ls = 0.0;
    for (int64_t row = (int64_t)blockIdx.x * 8 + warp; row < n; row += (int64_t)gridDim.x * 8) {
        const uint4 hv = *reinterpret_cast<const uint4 *>(H4 + row * 256 + f0);
        const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&hv);
        float h[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 t2 = __bfloat1622float2(h2[i]);
            h[2 * i] = t2.x;
            h[2 * i + 1] = t2.y;
        }
        float part[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            float a = 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                a = fmaf(sW[o][f0 + i], h[i], a);
            part[o] = a;
        }
#pragma unroll
        for (int o = 0; o < 8; ++o)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                part[o] += __shfl_xor_sync(0xffffffffu, part[o], off);
        float dy[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const float r = part[o] + b5[o] - T[row * 8 + o];
            if (lane == 0) ls += (double)r * (double)r;
            dy[o] = gscale * r;
            aB5[o] += dy[o];
        }
        const float4 za = *reinterpret_cast<const float4 *>(Z4 + row * 256 + f0);
        const float4 zb = *reinterpret_cast<const float4 *>(Z4 + row * 256 + f0 + 4);
        const float zz[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
        float dz[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float dh = 0.f;
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                dh = fmaf(dy[o], sW[o][f0 + i], dh);
                aW[o][i] = fmaf(dy[o], h[i], aW[o][i]);
            }
            dz[i] = dh * cosf(zz[i]);
            aB4[i] += dz[i];
        }
        uint4 pk;
        __nv_bfloat162 p0 = __floats2bfloat162_rn(dz[0], dz[1]), p1 = __floats2bfloat162_rn(dz[2], dz[3]),
                       p2 = __floats2bfloat162_rn(dz[4], dz[5]), p3 = __floats2bfloat162_rn(dz[6], dz[7]);
        pk.x = *reinterpret_cast<uint32_t *>(&p0);
        pk.y = *reinterpret_cast<uint32_t *>(&p1);
        pk.z = *reinterpret_cast<uint32_t *>(&p2);
        pk.w = *reinterpret_cast<uint32_t *>(&p3);
        *reinterpret_cast<uint4 *>(dZ4 + row * 256 + f0) = pk;
    }
    for (int w = 0; w < 8; ++w) {
        if (warp == w) {
#pragma unroll
            for (int o = 0; o < 8; ++o)
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    sAcc[o * 256 + f0 + i] += aW[o][i];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                sAcc[2048 + f0 + i] += aB4[i];
            if (lane == 0)
#pragma unroll
                for (int o = 0; o < 8; ++o)
                    sAcc[2304 + o] += aB5[o];
        }
        __syncthreads();
    }
    if (lane == 0) sLoss[warp] = ls;
    __syncthreads();
    for (int i = threadIdx.x; i < 2048; i += 256)
        atomicAdd(G + siren_oW(5) + i, sAcc[i]);
    atomicAdd(G + siren_oB(4) + threadIdx.x, sAcc[2048 + threadIdx.x]);
    if (threadIdx.x < 8) atomicAdd(G + siren_oB(5) + threadIdx.x, sAcc[2304 + threadIdx.x]);
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w)
            t += sLoss[w];
        atomicAdd(loss, t);
    }
}

// dz_L = dh_L cos z_L (BF16 for the next products) and db_L += sum over rows; for the
// first layer dz_1 = w0 dh_1 cos z_1, dW1 += dz_1 x^T, db1 += dz_1 instead. Thread = feature,
// block = a slab of rows.
__global__ void __launch_bounds__(256) k_bwd_act(const float *__restrict__ dH, const float *__restrict__ Z,
                                                 int64_t n, int rows_per_block, int L, float w0,
                                                 const float *__restrict__ x, __nv_bfloat16 *__restrict__ dZ,
                                                 float *__restrict__ G)
{
    const int f = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = r0 + rows_per_block < n ? r0 + rows_per_block : n;
    float acc = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (int64_t row = r0; row < r1; ++row) {
        const int64_t q = row * 256 + f;
        float d = dH[q] * cosf(Z[q]);
        if (L == 1) {
            d *= w0;
            a0 = fmaf(d, x[3 * row], a0);
            a1 = fmaf(d, x[3 * row + 1], a1);
            a2 = fmaf(d, x[3 * row + 2], a2);
        } else {
            dZ[q] = __float2bfloat16_rn(d);
        }
        acc += d;
    }
    atomicAdd(G + siren_oB(L) + f, acc);
    if (L == 1) {
        atomicAdd(G + siren_oW(1) + 3 * f, a0);
        atomicAdd(G + siren_oW(1) + 3 * f + 1, a1);
        atomicAdd(G + siren_oW(1) + 3 * f + 2, a2);
    }
}

template <typename P>
cudaError_t dev_alloc(P **p, size_t bytes)
{
    return cudaMalloc((void **)p, bytes);
}

cudaError_t ensure_work(Neural &nn, int64_t rows)
{
    if (rows <= nn.wcap) return cudaSuccess;
    cudaFree(nn.Z);
    cudaFree(nn.H);
    cudaFree(nn.dZ);
    cudaFree(nn.dH);
    nn.Z = nullptr;
    nn.H = nullptr;
    nn.dZ = nullptr;
    nn.dH = nullptr;
    nn.wcap = 0;
    cudaError_t e = dev_alloc(&nn.Z, (size_t)4 * rows * 256 * sizeof(float));
    if (e == cudaSuccess) e = dev_alloc(&nn.H, (size_t)4 * rows * 256 * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = dev_alloc(&nn.dZ, (size_t)rows * 256 * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = dev_alloc(&nn.dH, (size_t)rows * 256 * sizeof(float));
    if (e == cudaSuccess) nn.wcap = rows;
    return e;
}

// forward and backward of one batch; adds sum r^2 to nn.d_loss and the gradient to grad
cudaError_t fwd_bwd(Neural &nn, const float *x, const float *t, int64_t n, float *grad, cudaStream_t s)
{
    cudaError_t e = ensure_work(nn, n);
    if (e != cudaSuccess) return e;
    const size_t slab = (size_t)nn.wcap * 256;
    float *Z[4];
    __nv_bfloat16 *H[4];
    for (int k = 0; k < 4; ++k) {
        Z[k] = nn.Z + k * slab;
        H[k] = nn.H + k * slab;
    }
    const float w0 = (float)nn.omega0;
    const int eb = blocks_for(n * 256, 256);
    k_layer1<<<eb, 256, 0, s>>>(nn.P, x, n, w0, Z[0], H[0]);
    for (int L = 2; L <= 4; ++L) {
        e = gcs::gemm_bf16(H[L - 2], 0, nn.Wh + (size_t)(L - 2) * 65536, 0, Z[L - 1], (int)n, 256, 256, 1, 0, s);
        if (e != cudaSuccess) return e;
        k_act<<<eb, 256, 0, s>>>(nn.P, L, n, Z[L - 1], H[L - 1]);
    }
    k_out<<<blocks_for(n, 8, 152 * 4), 256, 0, s>>>(nn.P, nn.W5p, H[3], Z[3], t, n, (float)(2.0 / (double)(n * 8)),
                                                    nn.dZ, grad, nn.d_loss);
    // K = n split so that about two waves of CTAs share each dW product
    const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(n / 64, 152));
    const int rows_per_block = 32;
    const int bb = (int)((n + rows_per_block - 1) / rows_per_block);
    for (int L = 4; L >= 2; --L) {
        e = gcs::gemm_bf16(nn.dZ, 1, H[L - 2], 1, grad + siren_oW(L), 256, 256, (int)n, splits, 1, s);
        if (e != cudaSuccess) return e;
        e = gcs::gemm_bf16(nn.dZ, 0, nn.Wh + (size_t)(L - 2) * 65536, 1, nn.dH, (int)n, 256, 256, 1, 0, s);
        if (e != cudaSuccess) return e;
        k_bwd_act<<<bb, 256, 0, s>>>(nn.dH, Z[L - 2], n, rows_per_block, L - 1, w0, x, nn.dZ, grad);
    }
    return cudaGetLastError();
}

} // namespace

cudaError_t neural_free(Neural &nn)
{
    void *ptrs[] = {nn.P, nn.G, nn.Mo, nn.Vo, nn.Wh, nn.W5p, nn.Z, nn.H, nn.dZ, nn.dH, nn.d_loss, nn.d_err, nn.Xs, nn.Ts};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    nn = Neural{};
    return cudaSuccess;
}

cudaError_t neural_set(Neural &nn, const float *params, bool on_device, double omega0, double r_max,
                       double B_scale, double E_scale, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    const size_t pb = (size_t)kSirenNParams * sizeof(float);
    if (!nn.P) {
        e = dev_alloc(&nn.P, pb);
        if (e == cudaSuccess) e = dev_alloc(&nn.G, pb);
        if (e == cudaSuccess) e = dev_alloc(&nn.Mo, pb);
        if (e == cudaSuccess) e = dev_alloc(&nn.Vo, pb);
        if (e == cudaSuccess) e = dev_alloc(&nn.Wh, (size_t)3 * 65536 * sizeof(__nv_bfloat16));
        if (e == cudaSuccess) e = dev_alloc(&nn.W5p, (size_t)16 * 256 * sizeof(__nv_bfloat16));
        if (e == cudaSuccess) e = dev_alloc(&nn.d_loss, sizeof(double));
        if (e == cudaSuccess) e = dev_alloc(&nn.d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(nn.d_err, 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(nn.W5p, 0, (size_t)16 * 256 * sizeof(__nv_bfloat16), s);
        if (e != cudaSuccess) {
            neural_free(nn);
            return e;
        }
        nn.net.P = nn.P;
        nn.net.Wh = nn.Wh;
        nn.net.W5p = nn.W5p;
        nn.net.err = nn.d_err;
        e = gcs::siren_maps(nn.net);
        if (e != cudaSuccess) {
            neural_free(nn);
            return e;
        }
    }
    e = cudaMemcpyAsync(nn.P, params, pb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(nn.Mo, 0, pb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(nn.Vo, 0, pb, s);
    if (e != cudaSuccess) return e;
    k_to_bf16<<<blocks_for(kSirenNParams, 256), 256, 0, s>>>(nn.P, nn.Wh, nn.W5p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    nn.omega0 = omega0;
    nn.net.omega0 = (float)omega0;
    nn.r_max = r_max;
    nn.B_scale = B_scale;
    nn.E_scale = E_scale;
    nn.adam_t = 0;
    nn.ready = true;
    return cudaSuccess;
}

cudaError_t neural_eval(Neural &nn, const float *x, int64_t n, float *y, float *J, cudaStream_t s)
{
    gcs::SirenIn in{x, n, nullptr, 1.0f, (float)nn.r_max};
    gcs::SirenOut o{};
    o.y = y;
    o.J = J;
    return gcs::siren_eval(nn.net, in, o, s);
}

cudaError_t neural_field(Neural &nn, const float *x, int64_t n, float *field, cudaStream_t s)
{
    gcs::SirenIn in{x, n, nullptr, 1.0f, (float)nn.r_max};
    gcs::SirenOut o{};
    o.field = field;
    o.field_stride = 24;
    o.B_scale = nn.B_scale;
    o.E_scale = nn.E_scale;
    return gcs::siren_eval(nn.net, in, o, s);
}

cudaError_t neural_field_at(Neural &nn, const float *R, int64_t cap, const int32_t *n_dev, float *samples,
                            int stride, cudaStream_t s)
{
    gcs::SirenIn in{R, cap, n_dev, (float)(1.0 / nn.r_max), 1.0f};
    gcs::SirenOut o{};
    o.field = samples;
    o.field_stride = stride;
    o.B_scale = nn.B_scale;
    o.E_scale = nn.E_scale;
    return gcs::siren_eval(nn.net, in, o, s);
}

cudaError_t neural_targets(const Neural &nn, const GridRef &g, const float *x, int64_t n, float *t, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int b = blocks_for(n, 128);
    if (g.is_f64)
        k_targets<double><<<b, 128, 0, s>>>((const double *)g.nodes, g.n_r, g.n_th, g.n_ph, g.r_min, g.dr, x, n,
                                            nn.r_max, nn.B_scale, nn.E_scale, t);
    else
        k_targets<float><<<b, 128, 0, s>>>((const float *)g.nodes, g.n_r, g.n_th, g.n_ph, g.r_min, g.dr, x, n,
                                           nn.r_max, nn.B_scale, nn.E_scale, t);
    return cudaGetLastError();
}

cudaError_t neural_loss_grad(Neural &nn, const float *x, const float *t, int64_t n, float *grad, double *loss,
                             cudaStream_t s)
{
    float *g = grad ? grad : nn.G;
    cudaError_t e = cudaMemsetAsync(g, 0, (size_t)kSirenNParams * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(nn.d_loss, 0, sizeof(double), s);
    if (e == cudaSuccess) e = fwd_bwd(nn, x, t, n, g, s);
    if (e != cudaSuccess) return e;
    if (loss) {
        double v = 0.0;
        e = cudaMemcpyAsync(&v, nn.d_loss, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        *loss = v / (double)(n * 8);
    }
    return e;
}

int neural_read_error(Neural &nn, cudaStream_t s)
{
    int v = 0;
    if (!nn.d_err) return 0;
    if (cudaMemcpyAsync(&v, nn.d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    if (v && cudaMemsetAsync(nn.d_err, 0, sizeof(int), s) != cudaSuccess) return -1;
    return v;
}

cudaError_t neural_adam(Neural &nn, double lr, double beta1, double beta2, double eps, cudaStream_t s)
{
    ++nn.adam_t;
    const double bc1 = 1.0 - std::pow(beta1, (double)nn.adam_t), bc2 = 1.0 - std::pow(beta2, (double)nn.adam_t);
    k_adam<<<blocks_for(kSirenNParams, 256), 256, 0, s>>>(nn.P, nn.G, nn.Mo, nn.Vo, (float)lr, (float)beta1,
                                                         (float)beta2, (float)eps, (float)bc1, (float)bc2, nn.Wh,
                                                         nn.W5p);
    return cudaGetLastError();
}

cudaError_t neural_fit(Neural &nn, const GridRef &g, const float *samples, bool on_device, int64_t n_samples,
                       int64_t batch, int n_epochs, double lr, double beta1, double beta2, double eps,
                       float *loss_out, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (n_samples > nn.scap) {
        cudaFree(nn.Xs);
        cudaFree(nn.Ts);
        nn.Xs = nullptr;
        nn.Ts = nullptr;
        nn.scap = 0;
        e = dev_alloc(&nn.Xs, (size_t)n_samples * 3 * sizeof(float));
        if (e == cudaSuccess) e = dev_alloc(&nn.Ts, (size_t)n_samples * 8 * sizeof(float));
        if (e != cudaSuccess) return e;
        nn.scap = n_samples;
    }
    e = cudaMemcpyAsync(nn.Xs, samples, (size_t)n_samples * 3 * sizeof(float),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = neural_targets(nn, g, nn.Xs, n_samples, nn.Ts, s);
    if (e != cudaSuccess) return e;
    const int64_t nb = n_samples / batch;
    for (int ep = 0; ep < n_epochs; ++ep) {
        e = cudaMemsetAsync(nn.d_loss, 0, sizeof(double), s);
        for (int64_t b = 0; b < nb && e == cudaSuccess; ++b) {
            e = cudaMemsetAsync(nn.G, 0, (size_t)kSirenNParams * sizeof(float), s);
            if (e == cudaSuccess) e = fwd_bwd(nn, nn.Xs + b * batch * 3, nn.Ts + b * batch * 8, batch, nn.G, s);
            if (e == cudaSuccess) e = neural_adam(nn, lr, beta1, beta2, eps, s);
        }
        if (e != cudaSuccess) return e;
        double v = 0.0;
        e = cudaMemcpyAsync(&v, nn.d_loss, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        if (loss_out) loss_out[ep] = (float)(v / (double)(nb * batch * 8));
    }
    return cudaSuccess;
}

} // namespace gcn
