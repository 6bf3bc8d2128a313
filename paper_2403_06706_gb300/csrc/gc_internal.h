// gc_internal.h -- structures shared by the host side and the kernels of libgcpush.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gcp {

// One ensemble on the device (SI units). Injection parameters are only read by the
// injection kernel; the push reads the site, lambda and the shell.
struct EnsDev {
    double R0[3];
    double lambda;       // m
    double r_in, r_out;  // m
    double E0, E_lo, E_hi, E_index; // J
    int64_t first, count; // slot range of the ensemble's particles at injection
    int32_t energy_law, mu_law, scatter_law, pad;
    // FP32-path copies, precomputed on the host: R0 as double-float pairs, r_in^2, r_out^2
    float R0_hi[3], R0_lo[3];
    float r_in2, r_out2, lambda_f, pad_f;
};

// Device structure-of-arrays particle state; F0/F1 rows have stride `cap`.
struct StateDev {
    double *x, *y, *z, *u, *mub, *F0, *F1, *vpar, *s_rem, *h_prev, *t_birth, *u_inj, *mub_inj;
    uint32_t *id, *ens, *event, *ncoll, *flags;
    int64_t n, cap;
};

struct TallyDev {
    int32_t cadence, n_mu, n_E, n_r, n_age, n_ens;
    double t_start, E_lo, log_E_ratio, r_lo, r_span, age_max, rwin_lo, rwin_hi, age_young;
    // FP32-path forms: 1/E_lo, n_E/ln(E_hi/E_lo), r_lo, n_r/span, n_age/age_max, window, age
    float inv_E_lo_f, E_scale_f, r_lo_f, r_scale_f, age_scale_f, rwin_lo_f, rwin_hi_f, age_young_f;
    uint32_t *h_mer, *h_age, *h_pad;
    unsigned long long *m_cnt, *m_sin2, *n_seen;
};

struct PushParams {
    StateDev st;
    const EnsDev *ens;
    double dt, t0;       // t_new = t0 + (kbase + k + 1) dt for local step k
    int64_t step0;       // global step index of local step 0
    int64_t kbase;
    int32_t n_steps;
    int32_t collision_form, no_scatter, no_rebirth;
    double lambda_override; // m, > 0 overrides the ensembles
    double wind_u;          // m/s, > 0: collisions in the frame of the radial wind (Sect. 3.2)
    uint32_t seed;
    int32_t tally_on;
    double m, c2;           // rest mass (kg), c^2
    double two_over_m, inv_c2; // 2 / m and 1 / c^2 (the FP32 path's collision bookkeeping)
    TallyDev tally;
    uint32_t *gflags;              // OR of particle flags raised in this launch
    unsigned long long *counters;  // [0] collisions, [1] rebirths
    // optional clock in device memory ([0] time, [1] global step of the call's start); when
    // set it replaces t0 and step0 - kbase, so a captured graph replays at any time
    const double *clock;
};

struct InjectParams {
    StateDev st;
    const EnsDev *ens;
    int32_t n_ens;        // ensembles of this call (ens points at the first of them)
    int32_t ens_base;     // global index of ens[0]
    int64_t slot0, count; // inject slots [slot0, slot0 + count)
    uint32_t id0;
    uint32_t seed;
    double t, dt_init, m, c2;
    uint32_t *gflags;
};

// Split-step push: the state machine of the fused push cut at each field evaluation, for
// field sources that evaluate many points at once (the neural field). Per step:
//   PRED (all) -> samples -> CORR (all) -> samples -> POST (all; restarts join a list)
//   -> samples (list) -> R2 (list) -> samples (list) -> R3 (list).
// INJ_REQ / INJ_FIX redo the field-dependent part of the injection with the samples.
constexpr int kSampleStride = 40; // B, E, dB, dE (24), g (9), flags (1), dPhi (3), pad (3)
enum SplitKind { SPLIT_PRED = 0, SPLIT_CORR, SPLIT_POST, SPLIT_R2, SPLIT_R3, SPLIT_INJ_REQ, SPLIT_INJ_FIX };

struct SplitParams {
    PushParams P;          // state, ensembles, physics switches, tallies, counters; P.dt, P.t0
    float *req;            // [cap][3] request points (m), one per particle slot
    const float *S;        // [cap][kSampleStride] field samples at req
    float *reqR;           // [cap][3] requests of the restart list
    const float *SR;       // samples at reqR
    int32_t *list;         // slots of the restart list
    int32_t *count;        // entries in the list (device)
    int32_t g_in_sample;   // 1: index-space derivatives and g in the sample (grid), 0: Cartesian
    int32_t tally_now;     // this step ends on a tally sample
    int32_t ideal;         // drop E_par (ideal MHD field)
    int32_t pad;
    long long kk;          // t_new = t0 + kk dt for this step
    int64_t slot0, n_new;  // injection fix-up: slots [slot0, slot0 + n_new)
};

} // namespace gcp

// launchers (gc_push.cu)
namespace gcp {
struct GridHost {
    const void *nodes;
    int n_r, n_th, n_ph, ideal, is_f64;
    double r_min, dr, dth, dph;
    // time-dependent fields: a second snapshot (null: steady) and the snapshot times (s)
    const void *nodes1;
    double t_snap0, t_snap1;
};
struct PhysHost {
    double qm, inv_m, inv_c2;
    int drift_mask;
};
cudaError_t launch_push(int precision, const GridHost &g, const PhysHost &ph, const PushParams &p,
                        int block, int grid, cudaStream_t s);
cudaError_t launch_inject(int precision, const GridHost &g, const PhysHost &ph,
                          const InjectParams &p, cudaStream_t s);
int push_max_blocks_per_sm(int precision, int block, bool time_dependent = false, bool potential = false);
// one split-step kernel (FP32 path)
cudaError_t launch_split(int kind, const PhysHost &ph, const SplitParams &p, cudaStream_t s);
// grid field samples (FP32 grid) at R (cap x 3, m; count on the device or cap)
cudaError_t launch_grid_samples(const GridHost &g, const float *R, int64_t cap, const int32_t *n_dev, float *S,
                                cudaStream_t s);
// load the push kernels now (a launch inside a stream capture must not trigger loading)
cudaError_t preload_kernels();
// message returned by gc_last_error() on the calling thread (gc_api.cu)
void set_last_error(const char *msg);
} // namespace gcp
