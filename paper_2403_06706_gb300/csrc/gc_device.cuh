// gc_device.cuh -- device building blocks of the guiding-centre push (sm_103a).
//
// Field gather (trilinear interpolation, Sect. 2.2), the relativistic guiding-centre
// right-hand side (Eqs. 1-3), the predictor-corrector weights (Eqs. 5-6), Philox-4x32-10
// (Salmon et al., SC'11) and the double-float accumulators of the FP32 path.
//
// Formulation (not a copy of any listing): the gather keeps the interpolant's derivatives
// in index space (d/di_r, d/di_theta, d/di_phi per channel) and the Cartesian gradients of
// the three index coordinates; every Jacobian-vector product the right-hand side needs is
// contracted in that basis, so no 3x3 Jacobian is ever formed.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "unit_circle_table.h"

namespace gcp {

enum : uint32_t { FLAG_OUT_OF_GRID = 1u, FLAG_AXIS = 2u, FLAG_NONFINITE = 4u };

// How an evaluation takes E_par: decided at compile time for the fused push (the grid's mode
// is known at launch), at run time from GridMeta::ideal for the split-step kernels.
//   POT_IDEAL  ideal mode (ideal == 1): E_par = 0, its terms compiled out
//   POT_NONE   no potential channel, E_par from the run-time mode (E.b or 0)
//   POT_ON     the two-fluid potential channel (ideal == 2): E_par = -b.grad(Phi)
// The fused push gathers from the grid, whose phi-index gradient has no z component; the
// split-step kernels (POT_RUNTIME) may take Cartesian derivatives from other sources.
enum : int { POT_NONE = 0, POT_ON = 1, POT_IDEAL = 2, POT_RUNTIME = -1 };

// ----------------------------------------------------------------------------------------
// Philox-4x32-10: ten rounds of two 32x32 -> 64 multiplies; the two key words are bumped
// by the Weyl constants 0x9E3779B9 / 0xBB67AE85 before every round but the first.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// A particle's event e: key (particle id, seed), counter (e, 0, 0, 0).
__device__ __forceinline__ uint4 draw(uint32_t id, uint32_t seed, uint32_t event)
{
    return philox4x32_10(make_uint4(event, 0u, 0u, 0u), id, seed);
}

// 53-bit uniform on (0, 1]: 27 high bits of hi, 26 high bits of lo.
__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo)
{
    const unsigned long long a = ((unsigned long long)(hi >> 5) << 26) | (lo >> 6);
    return ((double)a + 1.0) * 0x1.0p-53;
}

// ----------------------------------------------------------------------------------------
// Double-float accumulator (hi + lo, |lo| <= ulp(hi)/2), used by the FP32 path for R,
// gamma v_par and the free path. Adding a float b: the increment joins the low word first,
// l = lo + b (the one rounding, 2^-24 relative to l, i.e. to the increment whenever the
// increment exceeds ulp(hi)), then Dekker's Fast2Sum moves l into the high word:
// h = hi + l, lo' = l - (h - hi), and h + lo' = hi + l exactly whenever |hi| >= |l|. That
// fails only while the accumulated value is as small as its increments (a component of R
// or gamma v_par passing through zero, the free path's last step), where the error is a
// rounding of that small value.
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_from(double d)
{
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}

__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_add(df a, float b)
{
    const float l = __fadd_rn(a.lo, b);
    const float h = __fadd_rn(a.hi, l);
    return {h, __fsub_rn(l, __fsub_rn(h, a.hi))};
}

// ----------------------------------------------------------------------------------------
// precision helpers. FP64: library functions of at most a few ulp (the plain path; rsqrt is
// the library's 1-ulp reciprocal square root, a fraction of the double-pipe work of a
// correctly rounded square root followed by a division). FP32: fast forms whose few-ulp
// errors sit far below the FP32 path's 1e-4 tolerance.
__device__ __forceinline__ float m_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double m_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float m_rsqrt(float a) { return rsqrtf(a); }
__device__ __forceinline__ double m_rsqrt(double a) { return rsqrt(a); }
__device__ __forceinline__ float m_floor(float a) { return floorf(a); }
__device__ __forceinline__ double m_floor(double a) { return floor(a); }
__device__ __forceinline__ float m_rcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double m_rcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float m_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double m_div(double a, double b) { return a / b; }
__device__ __forceinline__ bool m_finite(float a) { return isfinite(a); }
__device__ __forceinline__ bool m_finite(double a) { return isfinite(a); }
template <typename T> __device__ __forceinline__ T two_pi();
template <> __device__ __forceinline__ float two_pi<float>() { return 6.28318530717958647692f; }
template <> __device__ __forceinline__ double two_pi<double>() { return 6.28318530717958647692; }

// FP32 atan2: reduce to t = min(|x|,|y|) / max(|x|,|y|) in [0, 1], atan(t) ~ t p(t^2) with
// p of degree 7 fitted for minimal maximum error on [0, 1] (|error| < 4e-8 for the fitted
// coefficients, < 7.1e-8 at t = 1 with them rounded to the float literals below; the fit is
// reproduced by csrc/atan_coeffs.py), then unfold the octant.
__device__ __forceinline__ float m_atan2(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = mx > 0.0f ? __fdividef(mn, mx) : 0.0f;
    const float s = t * t;
    float p = -4.059181749e-03f;
    p = fmaf(p, s, 2.188265529e-02f);
    p = fmaf(p, s, -5.594641340e-02f);
    p = fmaf(p, s, 9.645255098e-02f);
    p = fmaf(p, s, -1.391013498e-01f);
    p = fmaf(p, s, 1.994696012e-01f);
    p = fmaf(p, s, -3.332990914e-01f);
    p = fmaf(p, s, 9.999993549e-01f);
    float r = t * p;
    if (ay > ax) r = 1.57079632679489662f - r;
    if (x < 0.0f) r = 3.14159265358979324f - r;
    return copysignf(r, y);
}

// FP64 polar angle of (X, Y) given inv_h = 1 / hypot(X, Y) and an FP32 estimate `est` of
// the angle (within 1e-6 rad), without a double-precision atan2. Take the reference angle
// a_m = m (2 pi / 256) nearest the estimate, with its cosine c and sine s from a table; the
// offset d = angle - a_m satisfies sin d = (Y c - X s) / hypot(X, Y) and |d| < 0.0123, so the
// arcsine's Maclaurin series d = t + t^3/6 + 3 t^5/40 + 5 t^7/112 (t = sin d) leaves a
// truncation error below 2e-19 and the result is as accurate as a library atan2 (the
// rounding of Y c - X s, about 2e-16 rad). Returns a_m + d: in (-0.0123, 2 pi) for any
// estimate in [-pi, pi].
__device__ __forceinline__ double refine_angle(double X, double Y, double inv_h, float est)
{
    const int m = __float2int_rn(est * (float)kCircleInvStep) & (GC_CIRCLE_N - 1);
    const double2 cs = __ldg(&kUnitCircle[m]);
    const double t = fma(Y, cs.x, -X * cs.y) * inv_h;
    const double t2 = t * t;
    double p = fma(t2, 5.0 / 112.0, 3.0 / 40.0);
    p = fma(t2, p, 1.0 / 6.0);
    const double d = fma(t * t2, p, t);
    return __dmul_rn((double)m, kCircleStep) + d;
}

// Polar and azimuthal angles of (x, y, z): theta in [0, pi] from the z axis, phi in
// (-pi, 2 pi) (the caller folds negative values).
__device__ __forceinline__ void polar_angles(float x, float y, float z, float rho, float, float,
                                             float &theta, float &phi)
{
    theta = m_atan2(rho, z);
    phi = m_atan2(y, x);
}
__device__ __forceinline__ void polar_angles(double x, double y, double z, double rho, double inv_rho,
                                             double inv_r, double &theta, double &phi)
{
    theta = refine_angle(z, rho, inv_r, m_atan2((float)rho, (float)z));
    phi = refine_angle(x, y, inv_rho, m_atan2((float)y, (float)x));
}

// ----------------------------------------------------------------------------------------
// Grid description in the precision of the push.
template <typename T>
struct GridMeta {
    const T *nodes;   // [n_ph][n_th][n_r][8]
    int n_r, n_th, n_ph, ideal;
    T r_min, inv_dr, inv_dth, inv_dph;
    // time-dependent fields: a second snapshot span seconds after the first (null: steady),
    // the first snapshot's time (s)
    const T *nodes1;
    T span, inv_span;
    double t_snap0;
};

// Interpolated field at one point.
//   B, E: values; dB[d][c], dE[d][c]: derivative of Cartesian component c along index
//   direction d (0 = i_r, 1 = i_theta, 2 = i_phi); g[d]: Cartesian gradient of index
//   coordinate d, so dF_c/dx_j = sum_d dF[d][c] g[d][j].
template <typename T>
struct Sample {
    T B[3], E[3];
    T dB[3][3], dE[3][3];
    T g[3][3];
    T dPhi[3]; // derivatives of the potential channel (two-fluid fields only), like dB[d]
    T dBdt[3], dEdt[3]; // time derivatives (time-dependent fields only)
    uint32_t flags;
};

__device__ __forceinline__ void load_node(const float *__restrict__ p, float v[6])
{
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    const float2 b = __ldg(reinterpret_cast<const float2 *>(p + 4));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
}

__device__ __forceinline__ void load_node(const double *__restrict__ p, double v[6])
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p + 2));
    const double2 c = __ldg(reinterpret_cast<const double2 *>(p + 4));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}

// A whole FP32 node record (32 bytes, 32-byte aligned) in one 256-bit read-only load.
__device__ __forceinline__ void load_node_pairs(const float *p, unsigned long long q[4])
{
    asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
        : "=l"(q[0]), "=l"(q[1]), "=l"(q[2]), "=l"(q[3])
        : "l"(p));
}

// Two FP32 channels in one 64-bit register and the packed f32x2 arithmetic of sm_100+ (two
// independent IEEE operations per instruction, the same results as two scalar ones).
__device__ __forceinline__ unsigned long long p2_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ unsigned long long p2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long p2_bcast(float x)
{
    unsigned long long d;
    asm("mov.b64 %0, {%1, %1};" : "=l"(d) : "f"(x));
    return d;
}

__device__ __forceinline__ unsigned long long p2_pack(float lo, float hi)
{
    unsigned long long d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}

__device__ __forceinline__ unsigned long long p2_mul(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ void p2_split(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// The trilinear interpolant of one node array at a located point (cell offsets o0 / o1 of
// the two phi planes, theta-row stride nr8, fractions fr, ft, fp): values and index-space
// derivatives of B and E, and of the potential channel when use_pot.
template <typename T>
__device__ __forceinline__ void interp_nodes(const T *__restrict__ nodes, uint32_t o0, uint32_t o1, uint32_t nr8,
                                             T fr, T ft, T fp, bool use_pot, Sample<T> &s)
{
    // FP32: each 32-byte node record in one 256-bit load, as four packed channel pairs
    // (Bx By | Bz Ex | Ey Ez | |B| Phi), interpolated two channels at a time (the fourth
    // pair for the potential's gradient only)
    unsigned long long c2[2][2][2][4];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const float *p = (const float *)nodes + (cc ? o1 : o0) + (b ? nr8 : 0u);
#pragma unroll
                for (int a = 0; a < 2; ++a)
                    load_node_pairs(p + 8 * a, c2[b][cc][a]);
            }
        }
        const unsigned long long FR = p2_bcast((float)fr), FT = p2_bcast((float)ft), FP = p2_bcast((float)fp);
#pragma unroll
        for (int pr = 0; pr < 4; ++pr) {
            if (pr == 3 && !use_pot)
                break;
            unsigned long long L[2][2], D[2][2];
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    D[b][cc] = p2_sub(c2[b][cc][1][pr], c2[b][cc][0][pr]);
                    L[b][cc] = p2_fma(FR, D[b][cc], c2[b][cc][0][pr]);
                }
            unsigned long long V[2], Dr[2], Dt[2];
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                Dt[cc] = p2_sub(L[1][cc], L[0][cc]);
                V[cc] = p2_fma(FT, Dt[cc], L[0][cc]);
                Dr[cc] = p2_fma(FT, p2_sub(D[1][cc], D[0][cc]), D[0][cc]);
            }
            const unsigned long long dv = p2_sub(V[1], V[0]);
            const unsigned long long val = p2_fma(FP, dv, V[0]);
            const unsigned long long d_r = p2_fma(FP, p2_sub(Dr[1], Dr[0]), Dr[0]);
            const unsigned long long d_t = p2_fma(FP, p2_sub(Dt[1], Dt[0]), Dt[0]);
            float v0, v1, r0, r1, t0, t1, p0, p1;
            p2_split(val, v0, v1);
            p2_split(d_r, r0, r1);
            p2_split(d_t, t0, t1);
            p2_split(dv, p0, p1);
            const float vv[2] = {v0, v1}, rr[2] = {r0, r1}, tt[2] = {t0, t1}, pp[2] = {p0, p1};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ch = 2 * pr + h;
                if (ch == 6) {
                    // |B|: not used
                } else if (ch == 7) {
                    s.dPhi[0] = rr[h]; s.dPhi[1] = tt[h]; s.dPhi[2] = pp[h];
                } else if (ch < 3) {
                    s.B[ch] = vv[h]; s.dB[0][ch] = rr[h]; s.dB[1][ch] = tt[h]; s.dB[2][ch] = pp[h];
                } else {
                    s.E[ch - 3] = vv[h]; s.dE[0][ch - 3] = rr[h]; s.dE[1][ch - 3] = tt[h]; s.dE[2][ch - 3] = pp[h];
                }
            }
        }
    } else {
    // c[b][cc][a][ch]: a = r offset, b = theta offset, cc = phi offset
    T c[2][2][2][6];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const T *p = nodes + (cc ? o1 : o0) + (b ? nr8 : 0u);
            load_node(p, c[b][cc][0]);
            load_node(p + 8, c[b][cc][1]);
        }
    }

#pragma unroll
    for (int ch = 0; ch < 6; ++ch) {
        // along r: value and d/di_r on the four (theta, phi) edges
        T L[2][2], D[2][2];
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const T d = c[b][cc][1][ch] - c[b][cc][0][ch];
                D[b][cc] = d;
                L[b][cc] = c[b][cc][0][ch] + fr * d;
            }
        // along theta
        T V[2], Dr[2], Dt[2];
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const T dl = L[1][cc] - L[0][cc];
            V[cc] = L[0][cc] + ft * dl;
            Dt[cc] = dl;
            Dr[cc] = D[0][cc] + ft * (D[1][cc] - D[0][cc]);
        }
        // along phi
        const T dv = V[1] - V[0];
        const T val = V[0] + fp * dv;
        const T d_r = Dr[0] + fp * (Dr[1] - Dr[0]);
        const T d_t = Dt[0] + fp * (Dt[1] - Dt[0]);
        if (ch < 3) {
            s.B[ch] = val; s.dB[0][ch] = d_r; s.dB[1][ch] = d_t; s.dB[2][ch] = dv;
        } else {
            s.E[ch - 3] = val; s.dE[0][ch - 3] = d_r; s.dE[1][ch - 3] = d_t; s.dE[2][ch - 3] = dv;
        }
    }
    }

    // two-fluid fields: the potential channel's index-space gradient (its value is not
    // used; the FP32 branch above takes it from the fourth pairs)
    if (sizeof(T) == 8 && use_pot) {
        T ph[2][2][2];
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int cc = 0; cc < 2; ++cc)
#pragma unroll
                for (int a = 0; a < 2; ++a)
                    ph[b][cc][a] = __ldg(nodes + (cc ? o1 : o0) + (b ? nr8 : 0u) + 8 * a + 7);
        T L[2][2], D[2][2];
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                D[b][cc] = ph[b][cc][1] - ph[b][cc][0];
                L[b][cc] = ph[b][cc][0] + fr * D[b][cc];
            }
        T V[2], Dr[2], Dt[2];
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            Dt[cc] = L[1][cc] - L[0][cc];
            V[cc] = L[0][cc] + ft * Dt[cc];
            Dr[cc] = D[0][cc] + ft * (D[1][cc] - D[0][cc]);
        }
        s.dPhi[0] = Dr[0] + fp * (Dr[1] - Dr[0]);
        s.dPhi[1] = Dt[0] + fp * (Dt[1] - Dt[0]);
        s.dPhi[2] = V[1] - V[0];
    } else if (!use_pot) {
        s.dPhi[0] = s.dPhi[1] = s.dPhi[2] = T(0);
    }

}

// Trilinear interpolation in (r, theta, phi) index space with the index-space gradient of
// the interpolant (Sect. 2.2). Node-centred grid, poles included in theta, periodic in phi.
// Positions more than one radial cell outside the grid are flagged; beyond the edge nodes
// the interpolant is extended as a constant.
template <typename T, int POT = POT_RUNTIME>
__device__ __forceinline__ void gather(const GridMeta<T> &gm, T x, T y, T z, Sample<T> &s,
                                       Sample<T> *s1 = nullptr)
{
    uint32_t flags = 0;
    T rho2 = x * x + y * y;
    if (!(rho2 > T(1e-30))) {
        flags |= FLAG_AXIS;
        rho2 = T(1e-30);
    }
    const T r2 = rho2 + z * z;
    const T inv_rho = m_rsqrt(rho2), inv_r = m_rsqrt(r2);
    const T rho = rho2 * inv_rho, r = r2 * inv_r;
    T theta, phi;
    polar_angles(x, y, z, rho, inv_rho, inv_r, theta, phi);
    if (phi < T(0))
        phi += two_pi<T>();
    T xr = (r - gm.r_min) * gm.inv_dr;
    T xt = theta * gm.inv_dth;
    T xp = phi * gm.inv_dph;
    if (!(m_finite(xr) && m_finite(xt) && m_finite(xp))) {
        flags |= FLAG_NONFINITE;
        xr = T(0); xt = T(0); xp = T(0);
    }
    if (xr < T(-1) || xr > T(gm.n_r))
        flags |= FLAG_OUT_OF_GRID;

    const T flr = m_floor(xr);
    int i = (int)flr;
    T fr = xr - flr;
    if (i < 0) { i = 0; fr = T(0); }
    else if (i > gm.n_r - 2) { i = gm.n_r - 2; fr = T(1); }
    const T flt = m_floor(xt);
    int j = (int)flt;
    T ft = xt - flt;
    if (j < 0) { j = 0; ft = T(0); }
    else if (j > gm.n_th - 2) { j = gm.n_th - 2; ft = T(1); }
    const T flp = m_floor(xp);
    int k = (int)flp;
    const T fp = xp - flp;
    if (k >= gm.n_ph) k -= gm.n_ph;
    if (k < 0) k += gm.n_ph;
    const int k1 = (k + 1 == gm.n_ph) ? 0 : k + 1;

    const uint32_t nr8 = (uint32_t)gm.n_r * 8u;
    const uint32_t o0 = (((uint32_t)k * (uint32_t)gm.n_th + (uint32_t)j) * (uint32_t)gm.n_r + (uint32_t)i) * 8u;
    const uint32_t o1 = (((uint32_t)k1 * (uint32_t)gm.n_th + (uint32_t)j) * (uint32_t)gm.n_r + (uint32_t)i) * 8u;

    const bool use_pot = POT == POT_ON || (POT == POT_RUNTIME && gm.ideal == 2);
    interp_nodes<T>(gm.nodes, o0, o1, nr8, fr, ft, fp, use_pot, s);
    if (s1)  // time-dependent fields: the second snapshot at the same point
        interp_nodes<T>(gm.nodes1, o0, o1, nr8, fr, ft, fp, use_pot, *s1);

    // Cartesian gradients of the index coordinates: rhat/dr, thetahat/(r dtheta),
    // phihat/(r sin(theta) dphi)
    const T sr = inv_r * gm.inv_dr;
    s.g[0][0] = x * sr; s.g[0][1] = y * sr; s.g[0][2] = z * sr;
    const T st = inv_r * inv_r * gm.inv_dth;
    const T zr = z * inv_rho;
    s.g[1][0] = zr * x * st; s.g[1][1] = zr * y * st; s.g[1][2] = -rho * st;
    const T sp = inv_rho * inv_rho * gm.inv_dph;
    s.g[2][0] = -y * sp; s.g[2][1] = x * sp; s.g[2][2] = T(0);
    s.flags = flags;
}

// Time-dependent fields: both snapshots interpolated at the point (located once), every
// quantity blended linearly at t_rel seconds after the first snapshot (held constant
// outside the window), and the time derivatives taken as the snapshots' secant slope
// inside it.
template <typename T, int POT = POT_RUNTIME>
__device__ __forceinline__ void gather_td(const GridMeta<T> &gm, T x, T y, T z, T t_rel, Sample<T> &s)
{
    Sample<T> s1;
    gather<T, POT>(gm, x, y, z, s, &s1);
    // the window test on the time itself: at t_rel == span the weight may round above 1
    const bool inside = (t_rel >= T(0)) && (t_rel <= gm.span);
    T w = t_rel * gm.inv_span;
    w = w < T(0) ? T(0) : (w > T(1) ? T(1) : w);
    const T rate = inside ? gm.inv_span : T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s.dBdt[c] = (s1.B[c] - s.B[c]) * rate;
        s.dEdt[c] = (s1.E[c] - s.E[c]) * rate;
        s.B[c] += w * (s1.B[c] - s.B[c]);
        s.E[c] += w * (s1.E[c] - s.E[c]);
        s.dPhi[c] += w * (s1.dPhi[c] - s.dPhi[c]);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            s.dB[d][c] += w * (s1.dB[d][c] - s.dB[d][c]);
            s.dE[d][c] += w * (s1.dE[d][c] - s.dE[d][c]);
        }
    }
}

// ----------------------------------------------------------------------------------------
// Relativistic guiding-centre right-hand side, Eqs. 1-2 (Eq. 3: mu_B constant).
template <typename T>
struct Phys {
    T qm;     // q / m
    T inv_qm; // m / q
    T inv_m;  // 1 / m
    T inv_c2; // 1 / c^2
    T mc2;    // m c^2
    int drift_mask;
};

template <typename T>
struct Aux {
    T gamma, vpar, Bm;
    T b[3]; // unit vector along B (the frame change of wind-frame collisions)
};

template <typename T>
__device__ __forceinline__ void cross3(const T a[3], const T b[3], T c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename T>
__device__ __forceinline__ T dot3(const T a[3], const T b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// J w for the channel block dF (J_cj = sum_d dF[d][c] g[d][j]) given p_d = g[d].w
template <typename T>
__device__ __forceinline__ void jvec(const T dF[3][3], const T p[3], T out[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c)
        out[c] = dF[0][c] * p[0] + dF[1][c] * p[1] + dF[2][c] * p[2];
}

// J_B p and J_E p together; FP32: the six channels as three packed pairs (Bx By | Bz Ex |
// Ey Ez), the pairs the gather interpolated, two FMAs per instruction
template <typename T>
__device__ __forceinline__ void jvec2(const T dB[3][3], const T dE[3][3], const T p[3], T JB[3], T JE[3])
{
    if constexpr (sizeof(T) == 4) {
        unsigned long long acc[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const unsigned long long P = p2_bcast(p[d]);
            const unsigned long long q0 = p2_pack(dB[d][0], dB[d][1]);
            const unsigned long long q1 = p2_pack(dB[d][2], dE[d][0]);
            const unsigned long long q2 = p2_pack(dE[d][1], dE[d][2]);
            if (d == 0) {
                acc[0] = p2_mul(q0, P);
                acc[1] = p2_mul(q1, P);
                acc[2] = p2_mul(q2, P);
            } else {
                acc[0] = p2_fma(q0, P, acc[0]);
                acc[1] = p2_fma(q1, P, acc[1]);
                acc[2] = p2_fma(q2, P, acc[2]);
            }
        }
        p2_split(acc[0], JB[0], JB[1]);
        p2_split(acc[1], JB[2], JE[0]);
        p2_split(acc[2], JE[1], JE[2]);
    } else {
        jvec(dB, p, JB);
        jvec(dE, p, JE);
    }
}

template <typename T, bool TD = false, int POT = POT_RUNTIME>
__device__ __forceinline__ void rhs(const Sample<T> &s, const Phys<T> &ph, int ideal, T u, T mub,
                                    T F[4], Aux<T> &aux)
{
    const T B2 = dot3(s.B, s.B);
    const T inv_B = m_rsqrt(B2);
    const T Bm = B2 * inv_B;
    const T inv_B2 = inv_B * inv_B;
    T b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        b[c] = s.B[c] * inv_B;

    // grad|B| = J_B^T b
    T sb[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        sb[d] = s.dB[d][0] * b[0] + s.dB[d][1] * b[1] + s.dB[d][2] * b[2];
    // the grid's phi-index gradient has no z component (g[2][2] = 0)
    constexpr bool kGridG = POT != POT_RUNTIME;
    T gB[3];
#pragma unroll
    for (int jx = 0; jx < 3; ++jx)
        gB[jx] = (kGridG && jx == 2) ? sb[0] * s.g[0][2] + sb[1] * s.g[1][2]
                                     : sb[0] * s.g[0][jx] + sb[1] * s.g[1][jx] + sb[2] * s.g[2][jx];
    const T b_gB = dot3(b, gB);

    // E x B drift
    T vE[3];
    cross3(s.E, s.B, vE);
#pragma unroll
    for (int c = 0; c < 3; ++c)
        vE[c] *= inv_B2;

    // ideal 1: E_par = 0 (ideal Ohm's law); 0: the interpolated E.b; 2: the two-fluid
    // correction -grad(Phi) (Sect. 2.2): E_par = -b.grad(Phi) = -sum_d dPhi/di_d (g_d . b)
    T Epar = T(0);
    if constexpr (POT == POT_IDEAL) {
    } else if (POT == POT_ON || (POT == POT_RUNTIME && ideal == 2)) {
        T pb[3];
#pragma unroll
        for (int d = 0; d < 3; ++d)
            pb[d] = dot3(s.g[d], b);
        Epar = -(s.dPhi[0] * pb[0] + s.dPhi[1] * pb[1] + s.dPhi[2] * pb[2]);
    } else {
        Epar = ideal ? T(0) : dot3(s.E, b);
    }
    // gamma^2 = 1 + (gamma v)^2 / c^2 with (gamma v)^2 = u^2 + 2 mu_B B / m
    const T g2 = T(1) + (u * u + T(2) * mub * Bm * ph.inv_m) * ph.inv_c2;
    const T inv_g = m_rsqrt(g2);
    const T gamma = g2 * inv_g;
    const T vpar = u * inv_g;

    if (ph.drift_mask == 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            F[c] = vpar * b[c];
        if constexpr (POT == POT_IDEAL)
            F[3] = -(mub * ph.inv_m * inv_g * b_gB);
        else
            F[3] = ph.qm * Epar - mub * ph.inv_m * inv_g * b_gB;
    } else {
        // Every directional derivative of Eqs. 1-2 is along w = v_par b + v_E (the guiding
        // centre's velocity without the drifts): the bracket's v_par^2 (b.grad)b +
        // v_par (v_E.grad)b = v_par (w.grad)b and v_par (b.grad)v_E + (v_E.grad)v_E =
        // (w.grad)v_E, and Eq. 2's v_par (b.grad)b + (v_E.grad)b = (w.grad)b.
        T wv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            wv[c] = vpar * b[c] + vE[c];
        T pw[3];
#pragma unroll
        for (int d = 0; d < 3; ++d)
            pw[d] = (kGridG && d == 2) ? s.g[2][0] * wv[0] + s.g[2][1] * wv[1] : dot3(s.g[d], wv);
        T JBw[3], JEw[3];
        jvec2(s.dB, s.dE, pw, JBw, JEw);
        const T w_gB = dot3(wv, gB);
        // (w.grad)b = (J_B w - b (w.grad|B|)) / |B|
        T wgb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            wgb[c] = (JBw[c] - b[c] * w_gB) * inv_B;
        // (w.grad)v_E = ((J_E w) x B + E x (J_B w)) / B^2 - 2 v_E (w.grad|B|) / |B|
        T t1[3], t2[3], wgv[3];
        cross3(JEw, s.B, t1);
        cross3(s.E, JBw, t2);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            wgv[c] = (t1[c] + t2[c]) * inv_B2 - T(2) * vE[c] * w_gB * inv_B;

        // Eq. 1 bracket
        const T c_gB = mub * ph.inv_m * inv_g * inv_g;
        T br[3];
        if constexpr (POT == POT_IDEAL) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                br[c] = c_gB * gB[c] + vpar * wgb[c] + wgv[c];
        } else {
            const T c_vE = ph.qm * vpar * Epar * ph.inv_c2 * inv_g;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                br[c] = c_gB * gB[c] + c_vE * vE[c] + vpar * wgb[c] + wgv[c];
        }
        // time-dependent fields: v_par db/dt + dv_E/dt in the bracket, and db/dt in Eq. 2's
        // v_E product, with db/dt = (dB/dt - b (b.dB/dt)) / B and
        // dv_E/dt = (dE/dt x B + E x dB/dt) / B^2 - 2 v_E (b.dB/dt) / B
        T dbdt[3] = {T(0), T(0), T(0)};
        if constexpr (TD) {
            const T bdB = dot3(b, s.dBdt);
            T e1[3], e2[3];
            cross3(s.dEdt, s.B, e1);
            cross3(s.E, s.dBdt, e2);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dbdt[c] = (s.dBdt[c] - b[c] * bdB) * inv_B;
                br[c] += vpar * dbdt[c] + (e1[c] + e2[c]) * inv_B2 - T(2) * vE[c] * bdB * inv_B;
            }
        }
        T bxbr[3];
        cross3(b, br, bxbr);
        const T pre = gamma * inv_B * ph.inv_qm;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            F[c] = vpar * b[c] + vE[c] + pre * bxbr[c];
        // Eq. 2
        T w2[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            w2[c] = wgb[c] + dbdt[c];
        if constexpr (POT == POT_IDEAL)
            F[3] = gamma * dot3(vE, w2) - mub * ph.inv_m * inv_g * b_gB;
        else
            F[3] = ph.qm * Epar - mub * ph.inv_m * inv_g * b_gB + gamma * dot3(vE, w2);
    }
    aux.gamma = gamma;
    aux.vpar = vpar;
    aux.Bm = Bm;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        aux.b[c] = b[c];
}

template <typename T, bool TD = false, int POT = POT_RUNTIME>
__device__ __forceinline__ uint32_t eval_F(const GridMeta<T> &gm, const Phys<T> &ph, T x, T y, T z,
                                           T u, T mub, T F[4], Aux<T> &aux, T t_rel = T(0))
{
    Sample<T> s;
    if constexpr (TD)
        gather_td<T, POT>(gm, x, y, z, t_rel, s);
    else
        gather<T, POT>(gm, x, y, z, s);
    rhs<T, TD, POT>(s, ph, gm.ideal, u, mub, F, aux);
    return s.flags;
}

} // namespace gcp
