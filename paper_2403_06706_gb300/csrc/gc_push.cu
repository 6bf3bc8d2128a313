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
// double-float pairs; mu_B is a double-float too (the right-hand side takes its float
// part), and the rare collision and rebirth updates of gamma v_par and mu_B run in double.
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

// The same draw as a double pair (a, 1 - a): the member below 1/2 is taken from the float
// that holds it without cancellation and the other is 1 minus it, so the two sum to 1 to
// double rounding (the two floats of a UPair sum to 1 only to float rounding).
struct UPairD {
    double a, b;
};

__device__ __forceinline__ UPairD u31_d(UPair p)
{
    if (p.u < 0.5f) {
        const double a = (double)p.u;
        return {a, 1.0 - a};
    }
    const double b = (double)p.ub;
    return {1.0 - b, b};
}

// FP64 reciprocal and square root by Newton's method from the float estimates, without the
// FP64 division and square-root sequences (GB300's FP64 pipe runs at 1/64 of the FP32 rate,
// and a warp with one colliding lane waits for them). For 0 < x < 3e38: the float estimate
// has a relative error e0 < 2^-21, each Newton step squares it (y <- y + y (1 - x y) for 1/x,
// y <- y + y (1 - x y^2) / 2 for 1/sqrt(x)), so two steps leave e0^4 < 2^-84 and the result
// carries only the FP64 roundings of the steps, a few ulp.
__device__ __forceinline__ double rcp_newton(double x)
{
    double y = (double)__frcp_rn((float)x);
    y = fma(y, fma(-x, y, 1.0), y);
    return fma(y, fma(-x, y, 1.0), y);
}

__device__ __forceinline__ double rsqrt_newton(double x)
{
    double y = (double)rsqrtf((float)x);
    y = fma(0.5 * y, fma(-x * y, y, 1.0), y);
    return fma(0.5 * y, fma(-x * y, y, 1.0), y);
}

__device__ __forceinline__ double sqrt_newton(double x) { return x > 0.0 ? x * rsqrt_newton(x) : 0.0; }

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
// Out of line: it runs once every cadence steps, and inlined its FP64 bin arithmetic would
// hold registers the step loop needs.
template <typename T>
__device__ __noinline__ void tally_sample(const TallyDev &T_, const PushParams &P, const Phys<T> &ph,
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
// mu_B of the FP32 path is a double-float: the float the right-hand side takes (in the
// particle state) and a low part that only the collision bookkeeping and the launch's load
// and store touch, kept in a per-thread shared-memory slot instead of a register the step
// loop would carry. Blocks of the push kernels have at most kMaxPushBlock threads.
constexpr int kMaxPushBlock = 128;
__shared__ float s_mub_lo[kMaxPushBlock];

template <typename T>
__device__ __forceinline__ void mub_lo_set(double d, T hi)
{
    if constexpr (sizeof(T) == 4)
        s_mub_lo[threadIdx.x] = (float)(d - (double)hi);
}

template <typename T>
__device__ __forceinline__ double mub_value(T hi)
{
    if constexpr (sizeof(T) == 4)
        return (double)hi + (double)s_mub_lo[threadIdx.x];
    else
        return (double)hi;
}

// ----------------------------------------------------------------------------------------
// Per-particle state and the four evaluation phases of a step, shared by the fused push
// (field evaluated inline) and the split-step push (field samples from a buffer).
//   phase 0  F* at the predictor point (Eq. 5), then the corrector (Eq. 6)
//   phase 1  F^{n+1} at the corrector point, then free path, rebirth and collision tests
//   phase 2  F^n of the new state after a rebirth or collision (start-up, Sect. 2.2)
//   phase 3  F^{n-1} at X^n - dt F^n
// Phases 2-3 run only for the particles that restart.
template <typename T>
struct PState {
    using A = typename AccOf<T>::A;
    A Rx, Ry, Rz, U, S;
    T mub, F0[4], F1[4], vpar0, hprev, Bm0;
    double t_birth;
    uint32_t event, ncoll, flags;
};

// constants of one particle that the step loop reads every step; the rest of its ensemble's
// constants are read from the table where an event needs them
struct PConst {
    float ri2, ro2; // squared shell radii moved 1e-5 inward: beyond them a rebirth is decided in double
    uint32_t e;
};

__device__ __forceinline__ double lambda_of(const PushParams &P, const EnsDev &E)
{
    return P.lambda_override > 0.0 ? P.lambda_override : E.lambda;
}
__device__ __forceinline__ float lambda_f_of(const PushParams &P, const EnsDev &E)
{
    return P.lambda_override > 0.0 ? (float)P.lambda_override : E.lambda_f;
}

// predictor / corrector weights of one step
template <typename T>
struct StepW {
    T a0, a1, c0, cs, c1;
};

template <typename T>
__device__ __forceinline__ void load_particle(const PushParams &P, int64_t i, PConst &c, PState<T> &s)
{
    using Acc = AccOf<T>;
    const int64_t cap = P.st.cap;
    c.e = P.st.ens[i];
    c.ri2 = P.ens[c.e].r_in2 * (1.0f + 1e-5f);
    c.ro2 = P.ens[c.e].r_out2 * (1.0f - 1e-5f);
    s.Rx = Acc::from(P.st.x[i]);
    s.Ry = Acc::from(P.st.y[i]);
    s.Rz = Acc::from(P.st.z[i]);
    s.U = Acc::from(P.st.u[i]);
    s.S = Acc::from(P.st.s_rem[i]);
    s.mub = (T)P.st.mub[i];
    mub_lo_set<T>(P.st.mub[i], s.mub);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        s.F0[k] = (T)P.st.F0[k * cap + i];
        s.F1[k] = (T)P.st.F1[k * cap + i];
    }
    s.vpar0 = (T)P.st.vpar[i];
    s.hprev = (T)P.st.h_prev[i];
    s.t_birth = P.st.t_birth[i];
    s.event = P.st.event[i];
    s.ncoll = P.st.ncoll[i];
    s.flags = P.st.flags[i];
    s.Bm0 = T(0);
}

template <typename T>
__device__ __forceinline__ void store_particle(const PushParams &P, int64_t i, const PState<T> &s)
{
    using Acc = AccOf<T>;
    const int64_t cap = P.st.cap;
    P.st.x[i] = Acc::to(s.Rx);
    P.st.y[i] = Acc::to(s.Ry);
    P.st.z[i] = Acc::to(s.Rz);
    P.st.u[i] = Acc::to(s.U);
    P.st.s_rem[i] = Acc::to(s.S);
    P.st.mub[i] = mub_value<T>(s.mub);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        P.st.F0[k * cap + i] = (double)s.F0[k];
        P.st.F1[k * cap + i] = (double)s.F1[k];
    }
    P.st.vpar[i] = (double)s.vpar0;
    P.st.h_prev[i] = (double)s.hprev;
    P.st.t_birth[i] = s.t_birth;
    P.st.event[i] = s.event;
    P.st.ncoll[i] = s.ncoll;
    if (s.flags != P.st.flags[i]) {
        P.st.flags[i] = s.flags;
        atomicOr(P.gflags, s.flags);
    }
}

// partial stores of the split-step kernels: only what a phase changed, so that the stored
// doubles of untouched fields keep every bit
__device__ __forceinline__ void store_flags(const PushParams &P, int64_t i, uint32_t flags)
{
    if (flags != P.st.flags[i]) {
        P.st.flags[i] = flags;
        atomicOr(P.gflags, flags);
    }
}

template <typename T>
__device__ __forceinline__ void store_RU(const PushParams &P, int64_t i, const PState<T> &s)
{
    using Acc = AccOf<T>;
    P.st.x[i] = Acc::to(s.Rx);
    P.st.y[i] = Acc::to(s.Ry);
    P.st.z[i] = Acc::to(s.Rz);
    P.st.u[i] = Acc::to(s.U);
    store_flags(P, i, s.flags);
}

template <typename T>
__device__ __forceinline__ void store_F(const PushParams &P, int64_t i, const PState<T> &s, int which)
{
    const int64_t cap = P.st.cap;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (which == 0)
            P.st.F0[k * cap + i] = (double)s.F0[k];
        else
            P.st.F1[k * cap + i] = (double)s.F1[k];
    }
    if (which == 0) P.st.vpar[i] = (double)s.vpar0;
    store_flags(P, i, s.flags);
}

template <typename T>
__device__ __forceinline__ StepW<T> step_weights(const StepW<T> &w1, T dtT, T hprev)
{
    StepW<T> w = w1;
    if (hprev != dtT) {
        // variable step: tau = dt^n / dt^{n-1}; weights (3+tau)/6,
        // (3+2 tau)/(6(1+tau)), -tau^2/(6(1+tau)) of Eq. 6
        const T tau = dtT / hprev;
        w.a0 = dtT * (T(1) + T(0.5) * tau);
        w.a1 = -dtT * T(0.5) * tau;
        const T q = dtT / (T(6) * (T(1) + tau));
        w.c0 = dtT * (T(3) + tau) / T(6);
        w.cs = q * (T(3) + T(2) * tau);
        w.c1 = -q * tau * tau;
    }
    return w;
}

// the point (R, gamma v_par) at which phase `phase` evaluates the field
template <typename T>
__device__ __forceinline__ void phase_point(int phase, const PState<T> &s, const StepW<T> &w, T dtT, T &px,
                                            T &py, T &pz, T &pu)
{
    using Acc = AccOf<T>;
    px = Acc::val(s.Rx);
    py = Acc::val(s.Ry);
    pz = Acc::val(s.Rz);
    pu = Acc::val(s.U);
    if (phase == 0) {
        px += w.a0 * s.F0[0] + w.a1 * s.F1[0];
        py += w.a0 * s.F0[1] + w.a1 * s.F1[1];
        pz += w.a0 * s.F0[2] + w.a1 * s.F1[2];
        pu += w.a0 * s.F0[3] + w.a1 * s.F1[3];
    } else if (phase == 3) {
        px -= dtT * s.F0[0];
        py -= dtT * s.F0[1];
        pz -= dtT * s.F0[2];
        pu -= dtT * s.F0[3];
    }
}

// Use the field evaluation Fo (with ax) of phase `phase` for particle slot i; after phase 1
// a rebirth or a collision sets n_phase = 4. kk: index of the step's end time (t_birth on
// rebirth).
// The state a rebirth or a collision changes.
template <typename T>
struct RareState {
    typename AccOf<T>::A Rx, Ry, Rz, U, S;
    T mub;
    double t_birth;
    uint32_t event, ncoll;
};

// A rebirth (Sect. 3) or, if not reborn, a collision (Sect. 2.3) of particle slot i, with B
// magnitude Bm_ and direction (b0, b1, b2) at the new position. Out of line: events are rare,
// and inlined, their FP64 and Philox arithmetic holds registers the step loop needs (the
// ensemble's constants are read from its table here for the same reason).
template <typename T>
__device__ __noinline__ RareState<T> rare_event(const PushParams &P, const Phys<T> &ph, int64_t i, bool reborn,
                                                RareState<T> s, T Bm_, T b0, T b1, T b2, double t0,
                                                long long kk)
{
    using Acc = AccOf<T>;
    const EnsDev &E = P.ens[P.st.ens[i]];
    const uint32_t id = P.st.id[i];
    if (reborn) {
        // Sect. 3: reborn at the injection site with the initial velocity
        const uint4 wd = draw(id, P.seed, s.event++);
        if constexpr (sizeof(T) == 8) {
            s.Rx = E.R0[0];
            s.Ry = E.R0[1];
            s.Rz = E.R0[2];
            s.S = -lambda_of(P, E) * log(u53(wd.z, wd.w));
        } else {
            s.Rx = df{E.R0_hi[0], E.R0_lo[0]};
            s.Ry = df{E.R0_hi[1], E.R0_lo[1]};
            s.Rz = df{E.R0_hi[2], E.R0_lo[2]};
            s.S = df{lambda_f_of(P, E) * neg_log_u(u31(wd.z)), 0.0f};
        }
        s.U = Acc::from(P.st.u_inj[i]);
        s.mub = (T)P.st.mub_inj[i];
        mub_lo_set<T>(P.st.mub_inj[i], s.mub);
        s.ncoll = 0;
        s.t_birth = step_time(t0, kk, P.dt);
    } else {
        // inertial-frame elastic collision: |p| kept, B at R^{n+1}; new pitch
        // cosine from Eq. 10 (mu = 1 - 2a) or Eq. 12 (mu = +-sqrt(a))
        const uint4 wd = draw(id, P.seed, s.event++);
        if constexpr (sizeof(T) == 8) {
            const double a = u53(wd.x, wd.y);
            const double mu_new = (E.scatter_law == 0) ? 1.0 - 2.0 * a : ((wd.x & 1u) ? -sqrt(a) : sqrt(a));
            const double Bm = (double)Bm_;
            const double uu = Acc::to(s.U);
            if (P.wind_u > 0.0) {
                // Sect. 3.2: elastic in the frame of the wind u = wind_u R/r; the guiding
                // centre drifts with u_perp already, so the frame change is a boost along
                // b by V = u.b (p_perp unchanged): u~ = gV (u - V gamma), back with -V
                const double X = Acc::to(s.Rx), Y = Acc::to(s.Ry), Z = Acc::to(s.Rz);
                const double V = P.wind_u * (X * b0 + Y * b1 + Z * b2) /
                                 sqrt(X * X + Y * Y + Z * Z);
                const double gV = 1.0 / sqrt(1.0 - V * V / P.c2);
                const double pp2 = 2.0 * (double)s.mub * Bm / P.m;
                const double gam = sqrt(1.0 + (uu * uu + pp2) / P.c2);
                const double ut = gV * (uu - V * gam);
                const double pt2 = ut * ut + pp2;
                const double gt = sqrt(1.0 + pt2 / P.c2);
                s.U = gV * (mu_new * sqrt(pt2) + V * gt);
                s.mub = (1.0 - mu_new * mu_new) * pt2 * P.m / (2.0 * Bm);
            } else {
                const double pm2 = uu * uu + 2.0 * (double)s.mub * Bm / P.m;
                const double pm = sqrt(pm2);
                s.U = mu_new * pm;
                s.mub = (1.0 - mu_new * mu_new) * pm2 * P.m / (2.0 * Bm);
            }
            if (P.collision_form == 0)
                s.S = -lambda_of(P, E) * log(u53(wd.z, wd.w));
        } else {
            // FP32 path: the pitch is drawn from float uniforms, the momentum bookkeeping
            // runs in FP64 on the double-float gamma v_par and mu_B, so |p| (|p~| in the wind
            // frame) is kept to double-float rounding (~1e-14), not FP32's; mu^2 + sin^2 = 1
            // to FP64 rounding (u31_d), and 1/x, sqrt(x) come from Newton steps.
            const UPairD ua = u31_d(u31(wd.x));
            double mu_new, sin2;
            if (E.scatter_law == 0) {
                mu_new = ua.b - ua.a; // Eq. 10: mu = (1 - a) - a
                sin2 = 4.0 * ua.a * ua.b;
            } else {
                const double su = sqrt_newton(ua.a); // Eq. 12: mu^2 = a
                mu_new = (wd.x & 1u) ? -su : su;
                sin2 = ua.b;
            }
            const double K = (double)Bm_ * P.two_over_m; // (p_perp / m)^2 = mu_B K
            const double uu = Acc::to(s.U);
            const double pp2 = mub_value<T>(s.mub) * K;
            double pm2 = uu * uu + pp2, un;
            if (P.wind_u > 0.0) {
                // the wind-frame collision of the FP64 branch above
                const double X = Acc::to(s.Rx), Y = Acc::to(s.Ry), Z = Acc::to(s.Rz);
                const double V = P.wind_u * (X * (double)b0 + Y * (double)b1 + Z * (double)b2) *
                                 rsqrt_newton(X * X + Y * Y + Z * Z);
                const double gV = rsqrt_newton(1.0 - V * V * P.inv_c2);
                const double gam = sqrt_newton(1.0 + pm2 * P.inv_c2);
                const double ut = gV * (uu - V * gam);
                pm2 = ut * ut + pp2;
                const double gt = sqrt_newton(1.0 + pm2 * P.inv_c2);
                un = gV * (mu_new * sqrt_newton(pm2) + V * gt);
            } else {
                un = mu_new * sqrt_newton(pm2);
            }
            const double mub_new = sin2 * pm2 * rcp_newton(K);
            s.U = Acc::from(un);
            s.mub = (T)mub_new;
            mub_lo_set<T>(mub_new, s.mub);
            if (P.collision_form == 0)
                s.S = df{lambda_f_of(P, E) * neg_log_u(u31(wd.z)), 0.0f};
        }
        ++s.ncoll;
    }
    return s;
}

template <typename T>
__device__ __forceinline__ void phase_consume(int phase, int &n_phase, int64_t i, PState<T> &s, const PConst &c,
                                              const T Fo[4],
                                              const Aux<T> &ax, const StepW<T> &w, const PushParams &P,
                                              const Phys<T> &ph, T dtT, double t0, long long kk,
                                              unsigned &n_coll, unsigned &n_reb)
{
    using Acc = AccOf<T>;
    if (phase == 0) {
        s.Rx = Acc::add(s.Rx, w.c0 * s.F0[0] + w.cs * Fo[0] + w.c1 * s.F1[0]);
        s.Ry = Acc::add(s.Ry, w.c0 * s.F0[1] + w.cs * Fo[1] + w.c1 * s.F1[1]);
        s.Rz = Acc::add(s.Rz, w.c0 * s.F0[2] + w.cs * Fo[2] + w.c1 * s.F1[2]);
        s.U = Acc::add(s.U, w.c0 * s.F0[3] + w.cs * Fo[3] + w.c1 * s.F1[3]);
    } else if (phase == 1) {
        const T px = Acc::val(s.Rx), py = Acc::val(s.Ry), pz = Acc::val(s.Rz);
        // Sect. 2.3: path length along B in this step
        const T ds = dtT * (fabs(s.vpar0) + fabs(ax.vpar)) * T(0.5);
        bool collide = false;
        if (!P.no_scatter) {
            if (P.collision_form == 0) {
                s.S = Acc::add(s.S, -ds);
                collide = Acc::nonpos(s.S);
            } else {
                // the per-step draw of Eq. 9: collide if a < 1 - exp(-ds / lambda)
                const uint4 wd = draw(P.st.id[i], P.seed, s.event++);
                if constexpr (sizeof(T) == 8)
                    collide = u53(wd.x, wd.y) < 1.0 - exp(-(double)ds / lambda_of(P, P.ens[c.e]));
                else
                    collide = u31(wd.x).u < -expm1f(-(float)ds / lambda_f_of(P, P.ens[c.e]));
            }
        }
        bool reborn = false;
        if (!P.no_rebirth) {
            if (sizeof(T) == 8) {
                const double xx = Acc::to(s.Rx), yy = Acc::to(s.Ry), zz = Acc::to(s.Rz);
                const double r1 = sqrt(xx * xx + yy * yy + zz * zz);
                reborn = (r1 < P.ens[c.e].r_in || r1 > P.ens[c.e].r_out);
            } else {
                const float xx = (float)px, yy = (float)py, zz = (float)pz;
                const float r2 = xx * xx + yy * yy + zz * zz;
                if (r2 < c.ri2 || r2 > c.ro2) {
                    // near or beyond the shell: decide in double from the accumulated position
                    const double X = Acc::to(s.Rx), Y = Acc::to(s.Ry), Z = Acc::to(s.Rz);
                    const double r1 = sqrt(X * X + Y * Y + Z * Z);
                    reborn = (r1 < P.ens[c.e].r_in || r1 > P.ens[c.e].r_out);
                }
            }
        }
        if (reborn || collide) {
            RareState<T> o{s.Rx, s.Ry, s.Rz, s.U, s.S, s.mub, s.t_birth, s.event, s.ncoll};
            o = rare_event<T>(P, ph, i, reborn, o, ax.Bm, ax.b[0], ax.b[1], ax.b[2], t0, kk);
            s.Rx = o.Rx; s.Ry = o.Ry; s.Rz = o.Rz; s.U = o.U; s.S = o.S;
            s.mub = o.mub; s.t_birth = o.t_birth; s.event = o.event; s.ncoll = o.ncoll;
            if (reborn)
                ++n_reb;
            else
                ++n_coll;
            n_phase = 4;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                s.F1[k] = s.F0[k];
                s.F0[k] = Fo[k];
            }
            s.vpar0 = ax.vpar;
            s.Bm0 = ax.Bm;
        }
    } else if (phase == 2) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            s.F0[k] = Fo[k];
        s.vpar0 = ax.vpar;
        s.Bm0 = ax.Bm;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            s.F1[k] = Fo[k];
    }
}
// The start-up history after a rebirth or a collision (phases 2 and 3 of the fused push):
// F^n at the new state and F^{n-1} at X^n - dt F^n. Out of line, like the events themselves,
// so that the step loop carries only the two phases every step has.
template <typename T>
struct Restart {
    T F0[4], F1[4], vpar0, Bm0;
    uint32_t flags;
};

template <typename T, bool TD, int POT>
__device__ __noinline__ Restart<T> restart_history(const GridMeta<T> &gm, const Phys<T> &ph, T x, T y, T z,
                                                   T u, T mub, T dtT, T t_end)
{
    Restart<T> o;
    Aux<T> ax;
    o.flags = eval_F<T, TD, POT>(gm, ph, x, y, z, u, mub, o.F0, ax, t_end);
    o.vpar0 = ax.vpar;
    o.Bm0 = ax.Bm;
    o.flags |= eval_F<T, TD, POT>(gm, ph, x - dtT * o.F0[0], y - dtT * o.F0[1], z - dtT * o.F0[2],
                                  u - dtT * o.F0[3], mub, o.F1, ax, t_end - dtT);
    return o;
}

// ----------------------------------------------------------------------------------------
// Resident CTAs of 128 threads per SM the FP32 push is compiled for (register budget:
// 65536 / (128 x blocks) per thread); the time-dependent variant carries more state.
#ifndef GC_PUSH_F32_MIN_BLOCKS
#define GC_PUSH_F32_MIN_BLOCKS 4
#endif
constexpr int kMinBlocksF32 = GC_PUSH_F32_MIN_BLOCKS;
// Time-dependent fields: 3 (4 spilled 172 bytes and measured 6 % slower). Potential channel:
// 4 like the steady kernel (3 measured 5 % slower).
#ifndef GC_PUSH_F32_TD_MIN_BLOCKS
#define GC_PUSH_F32_TD_MIN_BLOCKS 3
#endif
constexpr int kMinBlocksF32TD = GC_PUSH_F32_TD_MIN_BLOCKS;
#ifndef GC_PUSH_F32_POT_MIN_BLOCKS
#define GC_PUSH_F32_POT_MIN_BLOCKS GC_PUSH_F32_MIN_BLOCKS
#endif
constexpr int kMinBlocksF32Pot = GC_PUSH_F32_POT_MIN_BLOCKS;
// FP64: 2 (3 and 4 spill and measured 0.4 % and 1.7 % slower: the FP64 pipe, not
// latency, bounds that kernel)
#ifndef GC_PUSH_F64_MIN_BLOCKS
#define GC_PUSH_F64_MIN_BLOCKS 2
#endif
constexpr int kMinBlocksF64 = GC_PUSH_F64_MIN_BLOCKS;

// Fused push: one thread owns a particle for all the steps of a launch and evaluates the
// grid field inline.
template <typename T, bool TD, int POT>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? (TD ? kMinBlocksF32TD : (POT == POT_ON ? kMinBlocksF32Pot : kMinBlocksF32)) : kMinBlocksF64) push_kernel(const __grid_constant__ GridMeta<T> gm, const __grid_constant__ Phys<T> ph,
                                                   const __grid_constant__ PushParams P)
{
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
    const StepW<T> w1 = {dtT * T(1.5), dtT * T(-0.5), dtT * T(2.0 / 3.0), dtT * T(5.0 / 12.0),
                         dtT * T(-1.0 / 12.0)};
    // time-dependent fields: time of the call's start after the first snapshot
    const T tr0 = TD ? (T)(t0 - gm.t_snap0) : T(0);
    // the two phases of a step as straight-line code (each with its own copy of the field
    // evaluation) in the steady-field kernels; the time-dependent ones keep one copy in a
    // loop over the phases (unrolled, they spill)
    constexpr bool kUnrollPhases = !TD;

    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.st.n; i += stride) {
        PConst c;
        PState<T> s;
        load_particle(P, i, c, s);
        int next_tally = -1;
        if (P.tally_on) {
            const int64_t K = P.tally.cadence;
            next_tally = (int)((K - 1 - (step0 % K)) % K);
        }

        for (int k = 0; k < P.n_steps; ++k) {
            const StepW<T> w = step_weights(w1, dtT, s.hprev);
            // the predictor, corrector and restart evaluations are at the step's end time,
            // the start-up's F^{n-1} one step earlier
            const T t_end = TD ? tr0 + (T)(P.kbase + k + 1) * dtT : T(0);
            int n_phase = 2;
            // phase 0: predictor point and corrector; phase 1: F^{n+1}, free path, events;
            // after an event, phases 2-3 restart the history out of line
            auto run_phase = [&](int phase) {
                T px, py, pz, pu;
                phase_point(phase, s, w, dtT, px, py, pz, pu);
                T Fo[4];
                Aux<T> ax;
                s.flags |= eval_F<T, TD, POT>(gm, ph, px, py, pz, pu, s.mub, Fo, ax,
                                              phase == 3 ? t_end - dtT : t_end);
                phase_consume(phase, n_phase, i, s, c, Fo, ax, w, P, ph, dtT, t0, (long long)(P.kbase + k + 1),
                              n_coll, n_reb);
            };
            if constexpr (kUnrollPhases) {
#pragma unroll
                for (int phase = 0; phase < 2; ++phase)
                    run_phase(phase);
            } else {
#pragma unroll 1
                for (int phase = 0; phase < 2; ++phase)
                    run_phase(phase);
            }
            if (n_phase == 4) {
                using Acc = AccOf<T>;
                const Restart<T> o = restart_history<T, TD, POT>(gm, ph, Acc::val(s.Rx), Acc::val(s.Ry),
                                                                 Acc::val(s.Rz), Acc::val(s.U), s.mub, dtT, t_end);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    s.F0[q] = o.F0[q];
                    s.F1[q] = o.F1[q];
                }
                s.vpar0 = o.vpar0;
                s.Bm0 = o.Bm0;
                s.flags |= o.flags;
            }
            s.hprev = dtT;

            if (k == next_tally) {
                next_tally += P.tally.cadence;
                const double t_new = step_time(t0, (long long)(P.kbase + k + 1), P.dt);
                tally_sample<T>(P.tally, P, ph, c.e, AccOf<T>::val(s.Rx), AccOf<T>::val(s.Ry), AccOf<T>::val(s.Rz),
                                AccOf<T>::val(s.U), s.mub, s.Bm0, t_new - s.t_birth, s.ncoll,
                                s.t_birth >= P.tally.t_start && (int)c.e < P.tally.n_ens);
            }
        }
        // a non-finite position is flagged by the gather at the next evaluation; what the last
        // step leaves is checked here
        if (!(m_finite(AccOf<T>::val(s.Rx)) && m_finite(AccOf<T>::val(s.U)) && m_finite(s.F0[0])))
            s.flags |= FLAG_NONFINITE;
        store_particle(P, i, s);
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
struct InjDraw {
    double mu0, pm; // pitch cosine and momentum magnitude |p| / m = gamma v
    uint4 w0;       // event 0 (mu0 and the first free path)
};

__device__ __forceinline__ InjDraw inj_draw(const EnsDev &E, uint32_t id, uint32_t seed, double m, double c2)
{
    InjDraw d;
    d.w0 = draw(id, seed, 0u);
    const uint4 w1 = draw(id, seed, 1u);
    d.mu0 = (E.mu_law == 1) ? 1.0 : u53(d.w0.x, d.w0.y);
    double Ek = E.E0;
    if (E.energy_law == 1) {
        const double a = 1.0 - E.E_index;
        const double uu = u53(w1.x, w1.y);
        Ek = pow(pow(E.E_lo, a) + uu * (pow(E.E_hi, a) - pow(E.E_lo, a)), 1.0 / a);
    }
    const double mc2 = m * c2;
    const double gam = 1.0 + Ek / mc2;
    d.pm = sqrt(c2) * sqrt(gam * gam - 1.0);
    return d;
}

template <typename T, bool TD, int POT>
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
    const InjDraw d = inj_draw(E, id, P.seed, P.m, P.c2);
    const double mu0 = d.mu0, pm = d.pm;
    const uint4 w0 = d.w0;
    Sample<T> s;
    if constexpr (TD)
        gather_td<T, POT>(gm, (T)E.R0[0], (T)E.R0[1], (T)E.R0[2], (T)(P.t - gm.t_snap0), s);
    else
        gather<T, POT>(gm, (T)E.R0[0], (T)E.R0[1], (T)E.R0[2], s);
    const double Bm = (double)m_sqrt(dot3(s.B, s.B));
    const double u = mu0 * pm;
    const double mub = (1.0 - mu0 * mu0) * pm * pm * P.m / (2.0 * Bm);
    T F0[4], F1[4];
    Aux<T> a0x, a1x;
    const T x = (T)E.R0[0], y = (T)E.R0[1], z = (T)E.R0[2], uT = (T)u, mubT = (T)mub;
    const T dt = (T)P.dt_init;
    uint32_t flags = s.flags;
    const T t_inj = TD ? (T)(P.t - gm.t_snap0) : T(0);
    flags |= eval_F<T, TD, POT>(gm, ph, x, y, z, uT, mubT, F0, a0x, t_inj);
    flags |= eval_F<T, TD, POT>(gm, ph, x - dt * F0[0], y - dt * F0[1], z - dt * F0[2], uT - dt * F0[3],
                                mubT, F1, a1x, t_inj - dt);
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
// Split-step push (FP32 path). Each kernel advances every particle (or every entry of the
// restart list) by one evaluation phase, using the field samples of its request points.
__device__ __forceinline__ void load_sample(const float *__restrict__ S, int64_t k, int g_in, Sample<float> &s)
{
    const float4 *q = reinterpret_cast<const float4 *>(S + k * kSampleStride);
    float v[40];
#pragma unroll
    for (int j = 0; j < 10; ++j) {
        const float4 t = __ldg(q + j);
        v[4 * j] = t.x;
        v[4 * j + 1] = t.y;
        v[4 * j + 2] = t.z;
        v[4 * j + 3] = t.w;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s.B[c] = v[c];
        s.E[c] = v[3 + c];
        s.dPhi[c] = v[34 + c];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            s.dB[d][c] = v[6 + 3 * d + c];
            s.dE[d][c] = v[15 + 3 * d + c];
            s.g[d][c] = g_in ? v[24 + 3 * d + c] : (d == c ? 1.0f : 0.0f);
        }
    s.flags = g_in ? __float_as_uint(v[33]) : 0u;
}

__device__ __forceinline__ void put_point(float *R, int64_t k, float x, float y, float z)
{
    R[3 * k] = x;
    R[3 * k + 1] = y;
    R[3 * k + 2] = z;
}

__device__ __forceinline__ void flush_counters(const PushParams &P, unsigned n_coll, unsigned n_reb)
{
    const unsigned mask = __activemask();
    const unsigned c_sum = __reduce_add_sync(mask, n_coll);
    const unsigned r_sum = __reduce_add_sync(mask, n_reb);
    if ((threadIdx.x & 31u) == (unsigned)(__ffs(mask) - 1)) {
        if (c_sum) atomicAdd(P.counters + 0, (unsigned long long)c_sum);
        if (r_sum) atomicAdd(P.counters + 1, (unsigned long long)r_sum);
    }
}

template <int KIND>
__global__ void __launch_bounds__(128) split_kernel(const __grid_constant__ Phys<float> ph, const __grid_constant__ SplitParams Q)
{
    using Acc = AccOf<float>;
    const PushParams &P = Q.P;
    const float dtT = (float)P.dt;
    const StepW<float> w1 = {dtT * 1.5f, dtT * -0.5f, dtT * (float)(2.0 / 3.0), dtT * (float)(5.0 / 12.0),
                             dtT * (float)(-1.0 / 12.0)};
    const bool on_list = (KIND == SPLIT_R2 || KIND == SPLIT_R3);
    int64_t n = P.st.n;
    if (on_list) n = *Q.count;
    if (KIND == SPLIT_INJ_REQ || KIND == SPLIT_INJ_FIX) n = Q.n_new;
    unsigned n_coll = 0, n_reb = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        if constexpr (KIND == SPLIT_INJ_REQ) {
            const EnsDev &E = P.ens[P.st.ens[Q.slot0 + k]];
            put_point(Q.req, k, (float)E.R0[0], (float)E.R0[1], (float)E.R0[2]);
            continue;
        }
        const int64_t i = on_list ? (int64_t)Q.list[k] : (KIND == SPLIT_INJ_FIX ? Q.slot0 + k : k);
        PConst c;
        PState<float> s;
        load_particle(P, i, c, s);
        const StepW<float> w = step_weights(w1, dtT, s.hprev);
        Sample<float> smp;
        float Fo[4];
        Aux<float> ax;
        float px, py, pz, pu;
        int n_phase = 2;
        if constexpr (KIND == SPLIT_PRED) {
            phase_point(0, s, w, dtT, px, py, pz, pu);
            put_point(Q.req, i, px, py, pz);
            continue;
        } else if constexpr (KIND == SPLIT_CORR) {
            phase_point(0, s, w, dtT, px, py, pz, pu);
            load_sample(Q.S, i, Q.g_in_sample, smp);
            s.flags |= smp.flags;
            rhs(smp, ph, Q.ideal, pu, s.mub, Fo, ax);
            phase_consume(0, n_phase, i, s, c, Fo, ax, w, P, ph, dtT, P.t0, Q.kk, n_coll, n_reb);
            put_point(Q.req, i, Acc::val(s.Rx), Acc::val(s.Ry), Acc::val(s.Rz));
            store_RU(P, i, s);
        } else if constexpr (KIND == SPLIT_POST) {
            phase_point(1, s, w, dtT, px, py, pz, pu);
            load_sample(Q.S, i, Q.g_in_sample, smp);
            s.flags |= smp.flags;
            rhs(smp, ph, Q.ideal, pu, s.mub, Fo, ax);
            phase_consume(1, n_phase, i, s, c, Fo, ax, w, P, ph, dtT, P.t0, Q.kk, n_coll, n_reb);
            s.hprev = dtT;
            if (n_phase == 4) {
                const int32_t slot = atomicAdd(Q.count, 1);
                Q.list[slot] = (int32_t)i;
                put_point(Q.reqR, slot, Acc::val(s.Rx), Acc::val(s.Ry), Acc::val(s.Rz));
            } else {
                if (!(m_finite(Acc::val(s.Rx)) && m_finite(Acc::val(s.U)) && m_finite(s.F0[0])))
                    s.flags |= FLAG_NONFINITE;
                if (Q.tally_now) {
                    const double t_new = step_time(P.t0, Q.kk, P.dt);
                    tally_sample<float>(P.tally, P, ph, c.e, Acc::val(s.Rx), Acc::val(s.Ry), Acc::val(s.Rz),
                                        Acc::val(s.U), s.mub, s.Bm0, t_new - s.t_birth, s.ncoll,
                                        s.t_birth >= P.tally.t_start && (int)c.e < P.tally.n_ens);
                }
            }
            store_particle(P, i, s);
        } else if constexpr (KIND == SPLIT_R2) {
            phase_point(2, s, w, dtT, px, py, pz, pu);
            load_sample(Q.SR, k, Q.g_in_sample, smp);
            s.flags |= smp.flags;
            rhs(smp, ph, Q.ideal, pu, s.mub, Fo, ax);
            phase_consume(2, n_phase, i, s, c, Fo, ax, w, P, ph, dtT, P.t0, Q.kk, n_coll, n_reb);
            if (Q.tally_now) {
                const double t_new = step_time(P.t0, Q.kk, P.dt);
                tally_sample<float>(P.tally, P, ph, c.e, Acc::val(s.Rx), Acc::val(s.Ry), Acc::val(s.Rz),
                                    Acc::val(s.U), s.mub, s.Bm0, t_new - s.t_birth, s.ncoll,
                                    s.t_birth >= P.tally.t_start && (int)c.e < P.tally.n_ens);
            }
            phase_point(3, s, w, dtT, px, py, pz, pu);
            put_point(Q.reqR, k, px, py, pz);
            store_F(P, i, s, 0);
        } else if constexpr (KIND == SPLIT_R3) {
            phase_point(3, s, w, dtT, px, py, pz, pu);
            load_sample(Q.SR, k, Q.g_in_sample, smp);
            s.flags |= smp.flags;
            rhs(smp, ph, Q.ideal, pu, s.mub, Fo, ax);
            phase_consume(3, n_phase, i, s, c, Fo, ax, w, P, ph, dtT, P.t0, Q.kk, n_coll, n_reb);
            if (!(m_finite(Acc::val(s.Rx)) && m_finite(Acc::val(s.U)) && m_finite(s.F0[0])))
                s.flags |= FLAG_NONFINITE;
            store_F(P, i, s, 1);
        } else if constexpr (KIND == SPLIT_INJ_FIX) {
            // the injection's field-dependent part with this source: mu_B from |B| at the
            // site, F^n there, and the F^{n-1} request at X^n - dt F^n (Sect. 2.2)
            const InjDraw d = inj_draw(P.ens[c.e], P.st.id[i], P.seed, P.m, P.c2);
            load_sample(Q.S, k, Q.g_in_sample, smp);
            s.flags |= smp.flags;
            const double Bm = (double)m_sqrt(dot3(smp.B, smp.B));
            const double u = d.mu0 * d.pm;
            const double mub = (1.0 - d.mu0 * d.mu0) * d.pm * d.pm * P.m / (2.0 * Bm);
            s.U = Acc::from(u);
            s.mub = (float)mub;
            mub_lo_set<float>(mub, s.mub);
            rhs(smp, ph, Q.ideal, (float)u, (float)mub, Fo, ax);
            phase_consume(2, n_phase, i, s, c, Fo, ax, w, P, ph, dtT, P.t0, Q.kk, n_coll, n_reb);
            Q.list[k] = (int32_t)i;
            phase_point(3, s, w, dtT, px, py, pz, pu);
            put_point(Q.reqR, k, px, py, pz);
            P.st.u[i] = u;
            P.st.mub[i] = mub;
            P.st.u_inj[i] = u;
            P.st.mub_inj[i] = mub;
            store_F(P, i, s, 0);
        }
    }
    if (KIND == SPLIT_POST) flush_counters(P, n_coll, n_reb);
}

// grid samples in the split-step layout (Sample fields, index-space derivatives with g)
__global__ void __launch_bounds__(128) grid_sample_kernel(const GridMeta<float> gm, const float *__restrict__ R,
                                                          int64_t cap, const int32_t *n_dev, float *__restrict__ S)
{
    int64_t n = cap;
    if (n_dev) n = *n_dev < cap ? *n_dev : cap;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        Sample<float> s;
        gather(gm, R[3 * k], R[3 * k + 1], R[3 * k + 2], s);
        float v[40];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[c] = s.B[c];
            v[3 + c] = s.E[c];
        }
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[6 + 3 * d + c] = s.dB[d][c];
                v[15 + 3 * d + c] = s.dE[d][c];
                v[24 + 3 * d + c] = s.g[d][c];
            }
        v[33] = __uint_as_float(s.flags);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            v[34 + c] = s.dPhi[c];
        v[37] = v[38] = v[39] = 0.f;
        float4 *q = reinterpret_cast<float4 *>(S + k * kSampleStride);
#pragma unroll
        for (int j = 0; j < 10; ++j)
            q[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
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
    m.nodes1 = static_cast<const T *>(g.nodes1);
    m.span = g.nodes1 ? (T)(g.t_snap1 - g.t_snap0) : T(1);
    m.inv_span = g.nodes1 ? (T)(1.0 / (g.t_snap1 - g.t_snap0)) : T(0);
    m.t_snap0 = g.t_snap0;
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

// The fused push and injection come in one variant per field mode: steady or time
// dependent (two snapshots), with or without the potential channel (two-fluid E_par).
template <typename T>
using PushFn = void (*)(const GridMeta<T>, const Phys<T>, const PushParams);
template <typename T>
using InjectFn = void (*)(const GridMeta<T>, const Phys<T>, const InjectParams);

// ideal: the grid's mode is 1 (E_par = 0), which has a variant of its own
template <typename T>
PushFn<T> push_fn(bool td, bool pot, bool ideal)
{
    if (td)
        return pot ? push_kernel<T, true, POT_ON> : (ideal ? push_kernel<T, true, POT_IDEAL> : push_kernel<T, true, POT_NONE>);
    return pot ? push_kernel<T, false, POT_ON> : (ideal ? push_kernel<T, false, POT_IDEAL> : push_kernel<T, false, POT_NONE>);
}

template <typename T>
InjectFn<T> inject_fn(bool td, bool pot)
{
    if (td)
        return pot ? inject_kernel<T, true, POT_ON> : inject_kernel<T, true, POT_NONE>;
    return pot ? inject_kernel<T, false, POT_ON> : inject_kernel<T, false, POT_NONE>;
}

cudaError_t launch_push(int precision, const GridHost &g, const PhysHost &ph, const PushParams &p,
                        int block, int grid, cudaStream_t s)
{
    if (block < 1 || block > kMaxPushBlock)
        return cudaErrorInvalidConfiguration;
    cudaGetLastError(); // report this launch only
    const bool td = g.nodes1 != nullptr, pot = g.ideal == 2, ideal = g.ideal == 1;
    if (precision == 0)
        push_fn<double>(td, pot, ideal)<<<grid, block, 0, s>>>(make_meta<double>(g), make_phys<double>(ph), p);
    else
        push_fn<float>(td, pot, ideal)<<<grid, block, 0, s>>>(make_meta<float>(g), make_phys<float>(ph), p);
    return cudaGetLastError();
}

cudaError_t launch_inject(int precision, const GridHost &g, const PhysHost &ph,
                          const InjectParams &p, cudaStream_t s)
{
    const int block = 128;
    const int grid = (int)((p.count + block - 1) / block);
    if (grid == 0)
        return cudaSuccess;
    const bool td = g.nodes1 != nullptr, pot = g.ideal == 2;
    if (precision == 0)
        inject_fn<double>(td, pot)<<<grid, block, 0, s>>>(make_meta<double>(g), make_phys<double>(ph), p);
    else
        inject_fn<float>(td, pot)<<<grid, block, 0, s>>>(make_meta<float>(g), make_phys<float>(ph), p);
    return cudaGetLastError();
}

cudaError_t launch_split(int kind, const PhysHost &ph, const SplitParams &p, cudaStream_t s)
{
    const Phys<float> q = make_phys<float>(ph);
    const int block = 128;
    int64_t n = p.P.st.n;
    if (kind == SPLIT_R2 || kind == SPLIT_R3) n = p.P.st.n; // list length known on the device only
    if (kind == SPLIT_INJ_REQ || kind == SPLIT_INJ_FIX) n = p.n_new;
    int64_t blocks = (n + block - 1) / block;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    cudaGetLastError();
    switch (kind) {
    case SPLIT_PRED: split_kernel<SPLIT_PRED><<<(int)blocks, block, 0, s>>>(q, p); break;
    case SPLIT_CORR: split_kernel<SPLIT_CORR><<<(int)blocks, block, 0, s>>>(q, p); break;
    case SPLIT_POST: split_kernel<SPLIT_POST><<<(int)blocks, block, 0, s>>>(q, p); break;
    case SPLIT_R2: split_kernel<SPLIT_R2><<<(int)blocks, block, 0, s>>>(q, p); break;
    case SPLIT_R3: split_kernel<SPLIT_R3><<<(int)blocks, block, 0, s>>>(q, p); break;
    case SPLIT_INJ_REQ: split_kernel<SPLIT_INJ_REQ><<<(int)blocks, block, 0, s>>>(q, p); break;
    case SPLIT_INJ_FIX: split_kernel<SPLIT_INJ_FIX><<<(int)blocks, block, 0, s>>>(q, p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_grid_samples(const GridHost &g, const float *R, int64_t cap, const int32_t *n_dev, float *S,
                                cudaStream_t s)
{
    int64_t blocks = (cap + 127) / 128;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    cudaGetLastError();
    grid_sample_kernel<<<(int)blocks, 128, 0, s>>>(make_meta<float>(g), R, cap, n_dev, S);
    return cudaGetLastError();
}

cudaError_t preload_kernels()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < 8 && e == cudaSuccess; ++v) {
        e = cudaFuncGetAttributes(&a, push_fn<float>(v & 1, v & 2, v & 4));
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, push_fn<double>(v & 1, v & 2, v & 4));
    }
    return e;
}

int push_max_blocks_per_sm(int precision, int block, bool time_dependent, bool potential)
{
    int nb = 0;
    if (precision == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, push_fn<double>(time_dependent, potential, !potential), block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, push_fn<float>(time_dependent, potential, !potential), block, 0);
    return nb;
}

} // namespace gcp
