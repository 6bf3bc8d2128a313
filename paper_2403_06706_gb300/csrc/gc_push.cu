// gc_push.cu -- persistent guiding-centre push and injection kernels (sm_103a).
//
// One thread owns one particle at a time and keeps its whole state in registers for all
// the steps of a launch (grid-stride over particles). Per step (Sect. 2.2):
//   predictor X* (Eq. 5) -> F* = F(X*) -> corrector X^{n+1} (Eq. 6) -> F^{n+1}
//   -> free path decrement by dt (|v_par^n| + |v_par^{n+1}|)/2 (Sect. 2.3, Eq. 9)
//   -> rebirth if the particle left [r_in, r_out], else a collision if the free path is
//      used up (new pitch cosine from Eq. 10 or Eq. 12, |p| kept; inertial frame, Sect. 3)
//   -> backward-Euler start-up of the history after either (Sect. 2.2)
//   -> every `cadence` steps a snapshot sample into the tallies (Sect. 3).
//
// Precision: GC_PREC_FP64 runs everything in double. GC_PREC_FP32_MIXED evaluates the
// field and Eqs. 1-2 in float and accumulates R, gamma v_par and the free path in
// double-float pairs; the rare collision and rebirth updates run in double.
#include "gc_device.cuh"
#include "gc_internal.h"

namespace gcp {

// ----------------------------------------------------------------------------------------
// accumulator policy
template <typename T> struct AccOf;
template <> struct AccOf<double> {
    using A = double;
    static __device__ __forceinline__ A from(double d) { return d; }
    static __device__ __forceinline__ double to(A a) { return a; }
    static __device__ __forceinline__ A add(A a, double v) { return a + v; }
    static __device__ __forceinline__ double val(A a) { return a; }
    static __device__ __forceinline__ bool nonpos(A a) { return a <= 0.0; }
};
template <> struct AccOf<float> {
    using A = df;
    static __device__ __forceinline__ A from(double d) { return df_from(d); }
    static __device__ __forceinline__ double to(A a) { return df_to(a); }
    static __device__ __forceinline__ A add(A a, float v) { return df_add(a, v); }
    static __device__ __forceinline__ float val(A a) { return a.hi; }
    static __device__ __forceinline__ bool nonpos(A a) { return a.hi < 0.0f || (a.hi == 0.0f && a.lo <= 0.0f); }
};

// FP32-path uniform from one Philox word: u = (k + 1/2) 2^-31 with k the word's top 31
// bits (the FP64 path's 53-bit draw starts with the same bits, so the two agree to 2^-32),
// together with its complement 1 - u, each with full float relative precision.
struct UPair {
    float u, ub;
};

__device__ __forceinline__ UPair u31(uint32_t w)
{
    const uint32_t k = w >> 1;
    return {fmaf(__uint2float_rn(k), 0x1p-31f, 0x1p-32f),
            fmaf(__uint2float_rn(0x7FFFFFFFu - k), 0x1p-31f, 0x1p-32f)};
}

// -ln(u) without cancellation at either end of (0, 1)
__device__ __forceinline__ float neg_log_u(UPair p) { return p.u < 0.5f ? -logf(p.u) : -log1pf(-p.ub); }

// Time of the end of local step k. Out of line so that the FP64 arithmetic stays in the
// rare branches that need it (rebirth, tally) instead of being hoisted into every step.
__device__ __noinline__ double step_time(double t0, long long kk, double dt)
{
    return __dadd_rn(t0, __dmul_rn((double)kk, dt));
}

// warp-aggregated increment of base[idx] (idx < 0: no increment for this lane)
__device__ __forceinline__ void agg_inc(uint32_t *base, int idx)
{
    const unsigned mask = __activemask();
    const unsigned grp = __match_any_sync(mask, idx);
    const int leader = __ffs(grp) - 1;
    if (idx >= 0 && (int)(threadIdx.x & 31u) == leader)
        atomicAdd(base + idx, (uint32_t)__popc(grp));
}

__device__ __forceinline__ void agg_inc64(unsigned long long *base, int idx)
{
    const unsigned mask = __activemask();
    const unsigned grp = __match_any_sync(mask, idx);
    const int leader = __ffs(grp) - 1;
    if (idx >= 0 && (int)(threadIdx.x & 31u) == leader)
        atomicAdd(base + idx, (unsigned long long)__popc(grp));
}

// Snapshot sample of one particle (Sect. 3). FP64: the bins are computed with the same
// operations as the definition (double); FP32: the same formulas in float, with
// gamma - 1 formed without cancellation.
template <typename T>
__device__ __forceinline__ void tally_sample(const TallyDev &T_, const PushParams &P, const Phys<T> &ph,
                                             uint32_t e, T x, T y, T z, T u, T mub, T Bm, double age,
                                             uint32_t ncoll, bool take)
{
    int im = -1, iE = -1, ir = -1, ia = -1, ipad = -1;
    unsigned long long s2 = 0;
    if (take) {
        if constexpr (sizeof(T) == 8) {
            const double r = sqrt((double)x * x + (double)y * y + (double)z * z);
            const double gv2 = (double)u * u + 2.0 * (double)mub * (double)Bm / P.m;
            const double gamma = sqrt(1.0 + gv2 / P.c2);
            const double mu = (double)u / sqrt(gv2);
            const double Ek = (gamma - 1.0) * P.m * P.c2;
            const double sin2 = 1.0 - mu * mu;
            im = (int)floor((mu + 1.0) / 2.0 * T_.n_mu);
            if (im >= T_.n_mu) im = T_.n_mu - 1;
            if (im < 0) im = 0;
            const double xe = log(Ek / T_.E_lo) / T_.log_E_ratio * T_.n_E;
            iE = (xe >= 0.0 && xe < T_.n_E) ? (int)floor(xe) : -1;
            const double xr = (r - T_.r_lo) / T_.r_span * T_.n_r;
            ir = (xr >= 0.0 && xr < T_.n_r) ? (int)floor(xr) : -1;
            s2 = (unsigned long long)floor(sin2 * 4294967296.0 + 0.5);
            if (r >= T_.rwin_lo && r < T_.rwin_hi) {
                const double xa = age / T_.age_max * T_.n_age;
                if (xa >= 0.0 && xa < T_.n_age && iE >= 0)
                    ia = (int)(((int64_t)e * T_.n_age + (int)floor(xa)) * T_.n_E + iE);
                if (age < T_.age_young && ncoll >= 1)
                    ipad = (int)e * T_.n_mu + im;
            }
        } else {
            // FP32 path: the same bins from float arithmetic (gamma - 1 without cancellation)
            const float xf = (float)x, yf = (float)y, zf = (float)z, uf = (float)u;
            const float rf = sqrtf(xf * xf + yf * yf + zf * zf);
            const float gv2 = uf * uf + 2.0f * (float)mub * (float)Bm * (float)ph.inv_m;
            const float q = gv2 * (float)ph.inv_c2;
            const float gm1 = q / (sqrtf(1.0f + q) + 1.0f);
            const float muf = uf * rsqrtf(gv2);
            const float Ekf = gm1 * (float)ph.mc2;
            const float s2f = 1.0f - muf * muf;
            im = (int)floorf((muf + 1.0f) * 0.5f * (float)T_.n_mu);
            if (im >= T_.n_mu) im = T_.n_mu - 1;
            if (im < 0) im = 0;
            const float xe = logf(Ekf * T_.inv_E_lo_f) * T_.E_scale_f;
            iE = (xe >= 0.0f && xe < (float)T_.n_E) ? (int)floorf(xe) : -1;
            const float xr = (rf - T_.r_lo_f) * T_.r_scale_f;
            ir = (xr >= 0.0f && xr < (float)T_.n_r) ? (int)floorf(xr) : -1;
            s2 = (unsigned long long)__float2ull_rn(s2f * 4294967296.0f);
            if (rf >= T_.rwin_lo_f && rf < T_.rwin_hi_f) {
                const float agef = (float)age;
                const float xa = agef * T_.age_scale_f;
                if (xa >= 0.0f && xa < (float)T_.n_age && iE >= 0)
                    ia = (int)(((int64_t)e * T_.n_age + (int)floorf(xa)) * T_.n_E + iE);
                if (agef < T_.age_young_f && ncoll >= 1)
                    ipad = (int)e * T_.n_mu + im;
            }
        }
    }
    agg_inc64(T_.n_seen, take ? 0 : -1);
    agg_inc64(T_.n_seen, (take && (iE < 0 || ir < 0)) ? 1 : -1);
    const int ih = (take && iE >= 0 && ir >= 0)
                       ? (int)((((int64_t)e * T_.n_mu + im) * T_.n_E + iE) * T_.n_r + ir)
                       : -1;
    agg_inc(T_.h_mer, ih);
    const int irr = (take && ir >= 0) ? (int)e * T_.n_r + ir : -1;
    agg_inc64(T_.m_cnt, irr);
    if (irr >= 0)
        atomicAdd(T_.m_sin2 + irr, s2);
    agg_inc(T_.h_age, ia);
    agg_inc(T_.h_pad, ipad);
}

// ----------------------------------------------------------------------------------------
// The per-step work is a loop over evaluation phases so that one copy of the field
// evaluation serves all of them (instruction-cache footprint):
//   phase 0  F* at the predictor point (Eq. 5), then the corrector (Eq. 6)
//   phase 1  F^{n+1} at the corrector point, then free path, rebirth and collision tests
//   phase 2  F^n of the new state after a rebirth or collision (start-up, Sect. 2.2)
//   phase 3  F^{n-1} at X^n - dt F^n
// Phases 2-3 run only for the lanes that restart.
template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 2) push_kernel(const GridMeta<T> gm, const Phys<T> ph,
                                                   const PushParams P)
{
    using Acc = AccOf<T>;
    using A = typename Acc::A;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned n_coll = 0, n_reb = 0;
    const T dtT = (T)P.dt;
    double t0 = P.t0;
    int64_t step0 = P.step0;
    if (P.clock) {
        t0 = P.clock[0];
        step0 = (int64_t)P.clock[1] + P.kbase;
    }
    // Eq. 5-6 weights at tau = 1: 3/2, -1/2 (AB2) and 2/3, 5/12, -1/12 (AM3)
    const T a0_1 = dtT * T(1.5), a1_1 = dtT * T(-0.5);
    const T c0_1 = dtT * T(2.0 / 3.0), cs_1 = dtT * T(5.0 / 12.0), c1_1 = dtT * T(-1.0 / 12.0);

    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.st.n; i += stride) {
        const int64_t cap = P.st.cap;
        const uint32_t e = P.st.ens[i];
        const EnsDev &E = P.ens[e];
        const double lambda = P.lambda_override > 0.0 ? P.lambda_override : E.lambda;
        const double r_in = E.r_in, r_out = E.r_out;
        const float ri2 = E.r_in2, ro2 = E.r_out2;
        const float lambda_f = P.lambda_override > 0.0 ? (float)P.lambda_override : E.lambda_f;
        const int scatter_law = E.scatter_law;
        const uint32_t id = P.st.id[i];

        A Rx = Acc::from(P.st.x[i]), Ry = Acc::from(P.st.y[i]), Rz = Acc::from(P.st.z[i]);
        A U = Acc::from(P.st.u[i]);
        A S = Acc::from(P.st.s_rem[i]);
        T mub = (T)P.st.mub[i];
        T F0[4], F1[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            F0[c] = (T)P.st.F0[c * cap + i];
            F1[c] = (T)P.st.F1[c * cap + i];
        }
        T vpar0 = (T)P.st.vpar[i];
        T hprev = (T)P.st.h_prev[i];
        double t_birth = P.st.t_birth[i];
        uint32_t event = P.st.event[i], ncoll = P.st.ncoll[i], flags = P.st.flags[i];
        T Bm0 = T(0);
        int next_tally = -1;
        if (P.tally_on) {
            const int64_t K = P.tally.cadence;
            next_tally = (int)((K - 1 - (step0 % K)) % K);
        }

        for (int k = 0; k < P.n_steps; ++k) {
            T a0 = a0_1, a1 = a1_1, c0 = c0_1, cs = cs_1, c1 = c1_1;
            if (hprev != dtT) {
                // variable step: tau = dt^n / dt^{n-1}; weights (3+tau)/6,
                // (3+2 tau)/(6(1+tau)), -tau^2/(6(1+tau)) of Eq. 6
                const T tau = dtT / hprev;
                a0 = dtT * (T(1) + T(0.5) * tau);
                a1 = -dtT * T(0.5) * tau;
                const T w = dtT / (T(6) * (T(1) + tau));
                c0 = dtT * (T(3) + tau) / T(6);
                cs = w * (T(3) + T(2) * tau);
                c1 = -w * tau * tau;
            }
            int n_phase = 2;
#pragma unroll 1
            for (int phase = 0; phase < n_phase; ++phase) {
                T px = Acc::val(Rx), py = Acc::val(Ry), pz = Acc::val(Rz), pu = Acc::val(U);
                if (phase == 0) {
                    px += a0 * F0[0] + a1 * F1[0];
                    py += a0 * F0[1] + a1 * F1[1];
                    pz += a0 * F0[2] + a1 * F1[2];
                    pu += a0 * F0[3] + a1 * F1[3];
                } else if (phase == 3) {
                    px -= dtT * F0[0];
                    py -= dtT * F0[1];
                    pz -= dtT * F0[2];
                    pu -= dtT * F0[3];
                }
                T Fo[4];
                Aux<T> ax;
                flags |= eval_F(gm, ph, px, py, pz, pu, mub, Fo, ax);

                if (phase == 0) {
                    Rx = Acc::add(Rx, c0 * F0[0] + cs * Fo[0] + c1 * F1[0]);
                    Ry = Acc::add(Ry, c0 * F0[1] + cs * Fo[1] + c1 * F1[1]);
                    Rz = Acc::add(Rz, c0 * F0[2] + cs * Fo[2] + c1 * F1[2]);
                    U = Acc::add(U, c0 * F0[3] + cs * Fo[3] + c1 * F1[3]);
                } else if (phase == 1) {
                    // Sect. 2.3: path length along B in this step
                    const T ds = dtT * (fabs(vpar0) + fabs(ax.vpar)) * T(0.5);
                    bool collide = false;
                    if (!P.no_scatter) {
                        if (P.collision_form == 0) {
                            S = Acc::add(S, -ds);
                            collide = Acc::nonpos(S);
                        } else {
                            // the per-step draw of Eq. 9: collide if a < 1 - exp(-ds / lambda)
                            const uint4 wd = draw(id, P.seed, event++);
                            if constexpr (sizeof(T) == 8)
                                collide = u53(wd.x, wd.y) < 1.0 - exp(-(double)ds / lambda);
                            else
                                collide = u31(wd.x).u < -expm1f(-(float)ds / lambda_f);
                        }
                    }
                    bool reborn = false;
                    if (!P.no_rebirth) {
                        if (sizeof(T) == 8) {
                            const double xx = Acc::to(Rx), yy = Acc::to(Ry), zz = Acc::to(Rz);
                            const double r1 = sqrt(xx * xx + yy * yy + zz * zz);
                            reborn = (r1 < r_in || r1 > r_out);
                        } else {
                            const float xx = (float)px, yy = (float)py, zz = (float)pz;
                            const float r2 = xx * xx + yy * yy + zz * zz;
                            if (fabsf(r2 - ri2) < 1e-5f * ri2 || fabsf(r2 - ro2) < 1e-5f * ro2) {
                                // near the shell: decide in double from the accumulated position
                                const double X = Acc::to(Rx), Y = Acc::to(Ry), Z = Acc::to(Rz);
                                const double r1 = sqrt(X * X + Y * Y + Z * Z);
                                reborn = (r1 < r_in || r1 > r_out);
                            } else {
                                reborn = (r2 < ri2 || r2 > ro2);
                            }
                        }
                    }
                    if (reborn) {
                        // Sect. 3: reborn at the injection site with the initial velocity
                        const uint4 wd = draw(id, P.seed, event++);
                        if constexpr (sizeof(T) == 8) {
                            Rx = E.R0[0];
                            Ry = E.R0[1];
                            Rz = E.R0[2];
                            S = -lambda * log(u53(wd.z, wd.w));
                        } else {
                            Rx = df{E.R0_hi[0], E.R0_lo[0]};
                            Ry = df{E.R0_hi[1], E.R0_lo[1]};
                            Rz = df{E.R0_hi[2], E.R0_lo[2]};
                            S = df{lambda_f * neg_log_u(u31(wd.z)), 0.0f};
                        }
                        U = Acc::from(P.st.u_inj[i]);
                        mub = (T)P.st.mub_inj[i];
                        ncoll = 0;
                        t_birth = step_time(t0, (long long)(P.kbase + k + 1), P.dt);
                        ++n_reb;
                        n_phase = 4;
                    } else if (collide) {
                        // inertial-frame elastic collision: |p| kept, B at R^{n+1}; new pitch
                        // cosine from Eq. 10 (mu = 1 - 2a) or Eq. 12 (mu = +-sqrt(a))
                        const uint4 wd = draw(id, P.seed, event++);
                        if constexpr (sizeof(T) == 8) {
                            const double a = u53(wd.x, wd.y);
                            const double mu_new = (scatter_law == 0) ? 1.0 - 2.0 * a
                                                                     : ((wd.x & 1u) ? -sqrt(a) : sqrt(a));
                            const double Bm = (double)ax.Bm;
                            const double uu = Acc::to(U);
                            const double pm2 = uu * uu + 2.0 * (double)mub * Bm / P.m;
                            const double pm = sqrt(pm2);
                            U = mu_new * pm;
                            mub = (1.0 - mu_new * mu_new) * pm2 * P.m / (2.0 * Bm);
                            if (P.collision_form == 0)
                                S = -lambda * log(u53(wd.z, wd.w));
                        } else {
                            // sin^2 of the new pitch angle without cancellation: 4 a (1 - a)
                            // for Eq. 10 (mu = (1 - a) - a), 1 - a for Eq. 12 (mu^2 = a)
                            const UPair ua = u31(wd.x);
                            float mu_new, sin2;
                            if (scatter_law == 0) {
                                mu_new = ua.ub - ua.u;
                                sin2 = 4.0f * ua.u * ua.ub;
                            } else {
                                mu_new = (wd.x & 1u) ? -sqrtf(ua.u) : sqrtf(ua.u);
                                sin2 = ua.ub;
                            }
                            const float Bm = (float)ax.Bm;
                            const float uu = (float)Acc::val(U);
                            const float pm2 = uu * uu + 2.0f * (float)mub * Bm * (float)ph.inv_m;
                            U = df{mu_new * sqrtf(pm2), 0.0f};
                            mub = (T)(sin2 * pm2 * 0.5f / (Bm * (float)ph.inv_m));
                            if (P.collision_form == 0)
                                S = df{lambda_f * neg_log_u(u31(wd.z)), 0.0f};
                        }
                        ++ncoll;
                        ++n_coll;
                        n_phase = 4;
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            F1[c] = F0[c];
                            F0[c] = Fo[c];
                        }
                        vpar0 = ax.vpar;
                        Bm0 = ax.Bm;
                    }
                } else if (phase == 2) {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        F0[c] = Fo[c];
                    vpar0 = ax.vpar;
                    Bm0 = ax.Bm;
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        F1[c] = Fo[c];
                }
            }
            hprev = dtT;
            if (!(m_finite(Acc::val(Rx)) && m_finite(Acc::val(U)) && m_finite(F0[0])))
                flags |= FLAG_NONFINITE;

            if (k == next_tally) {
                next_tally += P.tally.cadence;
                const double t_new = step_time(t0, (long long)(P.kbase + k + 1), P.dt);
                tally_sample<T>(P.tally, P, ph, e, Acc::val(Rx), Acc::val(Ry), Acc::val(Rz), Acc::val(U),
                                mub, Bm0, t_new - t_birth, ncoll,
                                t_birth >= P.tally.t_start && (int)e < P.tally.n_ens);
            }
        }

        P.st.x[i] = Acc::to(Rx);
        P.st.y[i] = Acc::to(Ry);
        P.st.z[i] = Acc::to(Rz);
        P.st.u[i] = Acc::to(U);
        P.st.s_rem[i] = Acc::to(S);
        P.st.mub[i] = (double)mub;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            P.st.F0[c * cap + i] = (double)F0[c];
            P.st.F1[c * cap + i] = (double)F1[c];
        }
        P.st.vpar[i] = (double)vpar0;
        P.st.h_prev[i] = (double)hprev;
        P.st.t_birth[i] = t_birth;
        P.st.event[i] = event;
        P.st.ncoll[i] = ncoll;
        if (flags != P.st.flags[i]) {
            P.st.flags[i] = flags;
            atomicOr(P.gflags, flags);
        }
    }
    // counters: one atomic per warp
    const unsigned mask = __activemask();
    const unsigned c_sum = __reduce_add_sync(mask, n_coll);
    const unsigned r_sum = __reduce_add_sync(mask, n_reb);
    if ((threadIdx.x & 31u) == (unsigned)(__ffs(mask) - 1)) {
        if (c_sum) atomicAdd(P.counters + 0, (unsigned long long)c_sum);
        if (r_sum) atomicAdd(P.counters + 1, (unsigned long long)r_sum);
    }
}

// ----------------------------------------------------------------------------------------
// Injection (Sect. 3): site, mu0 and energy draws (Philox events 0 and 1), start-up history.
template <typename T>
__global__ void __launch_bounds__(256) inject_kernel(const GridMeta<T> gm, const Phys<T> ph,
                                                     const InjectParams P)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.count)
        return;
    const int64_t i = P.slot0 + j;
    int e = 0;
    while (e + 1 < P.n_ens && j >= P.ens[e + 1].first - P.slot0)
        ++e;
    const EnsDev &E = P.ens[e];
    const uint32_t id = P.id0 + (uint32_t)j;
    const uint4 w0 = draw(id, P.seed, 0u);
    const uint4 w1 = draw(id, P.seed, 1u);
    const double mu0 = (E.mu_law == 1) ? 1.0 : u53(w0.x, w0.y);
    double Ek = E.E0;
    if (E.energy_law == 1) {
        const double a = 1.0 - E.E_index;
        const double uu = u53(w1.x, w1.y);
        Ek = pow(pow(E.E_lo, a) + uu * (pow(E.E_hi, a) - pow(E.E_lo, a)), 1.0 / a);
    }
    const double mc2 = P.m * P.c2;
    const double gam = 1.0 + Ek / mc2;
    const double pm = sqrt(P.c2) * sqrt(gam * gam - 1.0);
    Sample<T> s;
    gather(gm, (T)E.R0[0], (T)E.R0[1], (T)E.R0[2], s);
    const double Bm = (double)m_sqrt(dot3(s.B, s.B));
    const double u = mu0 * pm;
    const double mub = (1.0 - mu0 * mu0) * pm * pm * P.m / (2.0 * Bm);
    T F0[4], F1[4];
    Aux<T> a0x, a1x;
    const T x = (T)E.R0[0], y = (T)E.R0[1], z = (T)E.R0[2], uT = (T)u, mubT = (T)mub;
    const T dt = (T)P.dt_init;
    uint32_t flags = s.flags;
    flags |= eval_F(gm, ph, x, y, z, uT, mubT, F0, a0x);
    flags |= eval_F(gm, ph, x - dt * F0[0], y - dt * F0[1], z - dt * F0[2], uT - dt * F0[3], mubT,
                    F1, a1x);
    const int64_t cap = P.st.cap;
    P.st.x[i] = E.R0[0];
    P.st.y[i] = E.R0[1];
    P.st.z[i] = E.R0[2];
    P.st.u[i] = u;
    P.st.mub[i] = mub;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        P.st.F0[c * cap + i] = (double)F0[c];
        P.st.F1[c * cap + i] = (double)F1[c];
    }
    P.st.vpar[i] = (double)a0x.vpar;
    P.st.s_rem[i] = -E.lambda * log(u53(w0.z, w0.w));
    P.st.h_prev[i] = P.dt_init;
    P.st.t_birth[i] = P.t;
    P.st.u_inj[i] = u;
    P.st.mub_inj[i] = mub;
    P.st.id[i] = id;
    P.st.ens[i] = (uint32_t)(P.ens_base + e);
    P.st.event[i] = 2u;
    P.st.ncoll[i] = 0u;
    P.st.flags[i] = flags;
    if (flags)
        atomicOr(P.gflags, flags);
}

// ----------------------------------------------------------------------------------------
template <typename T>
static GridMeta<T> make_meta(const GridHost &g)
{
    GridMeta<T> m;
    m.nodes = static_cast<const T *>(g.nodes);
    m.n_r = g.n_r;
    m.n_th = g.n_th;
    m.n_ph = g.n_ph;
    m.ideal = g.ideal;
    m.r_min = (T)g.r_min;
    m.inv_dr = (T)(1.0 / g.dr);
    m.inv_dth = (T)(1.0 / g.dth);
    m.inv_dph = (T)(1.0 / g.dph);
    return m;
}

template <typename T>
static Phys<T> make_phys(const PhysHost &p)
{
    Phys<T> q;
    q.qm = (T)p.qm;
    q.inv_qm = (T)(1.0 / p.qm);
    q.inv_m = (T)p.inv_m;
    q.inv_c2 = (T)p.inv_c2;
    q.mc2 = (T)(1.0 / (p.inv_m * p.inv_c2));
    q.drift_mask = p.drift_mask;
    return q;
}

cudaError_t launch_push(int precision, const GridHost &g, const PhysHost &ph, const PushParams &p,
                        int block, int grid, cudaStream_t s)
{
    cudaGetLastError(); // report this launch only
    if (precision == 0)
        push_kernel<double><<<grid, block, 0, s>>>(make_meta<double>(g), make_phys<double>(ph), p);
    else
        push_kernel<float><<<grid, block, 0, s>>>(make_meta<float>(g), make_phys<float>(ph), p);
    return cudaGetLastError();
}

cudaError_t launch_inject(int precision, const GridHost &g, const PhysHost &ph,
                          const InjectParams &p, cudaStream_t s)
{
    const int block = 128;
    const int grid = (int)((p.count + block - 1) / block);
    if (grid == 0)
        return cudaSuccess;
    if (precision == 0)
        inject_kernel<double><<<grid, block, 0, s>>>(make_meta<double>(g), make_phys<double>(ph), p);
    else
        inject_kernel<float><<<grid, block, 0, s>>>(make_meta<float>(g), make_phys<float>(ph), p);
    return cudaGetLastError();
}

cudaError_t preload_kernels()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, push_kernel<float>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, push_kernel<double>);
    return e;
}

int push_max_blocks_per_sm(int precision, int block)
{
    int nb = 0;
    if (precision == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, push_kernel<double>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, push_kernel<float>, block, 0);
    return nb;
}

} // namespace gcp
