/*
 * gcpush.h -- C ABI of libgcpush, a GB300 (sm_103a) implementation of the
 * guiding-centre transport of solar energetic electrons of Houeibib,
 * Pantellini & Griton, "Dynamics of energetic electrons scattered in the solar
 * wind" (A&A, arXiv:2403.06706).
 *
 * Conventions for every entry point
 *   - All functions return an int status: GC_OK (0) or a negative GC_ERR_*.
 *     gc_last_error() returns a message for the calling thread's last error.
 *     Errors never abort the process and never trap the GPU: device-side
 *     anomalies (non-finite state, positions far outside the grid) set flags
 *     that gc_advance reports as GC_ERR_DEVICE_ANOMALY after its work is done.
 *   - Host pointers are caller-owned and are only read or written during the
 *     call. Device copies of the field and of the particle state are owned by
 *     the context and freed by gc_destroy.
 *   - Units at the boundary: descriptors use AU, keV, degrees and seconds;
 *     particle state and grid values are SI (m, m/s, J/T, T, V/m).
 *   - Work is issued on the context's CUDA stream (gc_options.stream). Calls
 *     that return data to the host synchronise that stream before returning.
 *   - A context is not thread-safe; use one context per host thread. Contexts on the
 *     same device, each on its own stream and driven by its own thread, run
 *     concurrently (one context's host copies overlap another's kernels); a
 *     population split into such shards evolves exactly as in one context when
 *     each shard keeps its particle ids (gc_options.id_base).
 */
#ifndef GCPUSH_H
#define GCPUSH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gc_ctx gc_ctx;

enum {
    GC_OK = 0,
    GC_ERR_INVALID = -1,        /* bad argument, size or descriptor */
    GC_ERR_CUDA = -2,           /* a CUDA runtime call failed (message has the detail) */
    GC_ERR_NOMEM = -3,          /* device or pinned host allocation failed */
    GC_ERR_STATE = -4,          /* call out of order (e.g. advance before field_load) */
    GC_ERR_DEVICE_ANOMALY = -5, /* particles were flagged during the call (see gc_stats) */
    GC_ERR_UNSUPPORTED = -6     /* feature not available for this field source or precision */
};

/* precision of the push */
enum {
    GC_PREC_FP64 = 0,      /* all arithmetic in FP64 */
    GC_PREC_FP32_MIXED = 1 /* FP32 field and right-hand side; position, gamma v_par and the
                              free path accumulated in double-float (two FP32 words) */
};

/* grid node value type */
enum { GC_DTYPE_F64 = 0, GC_DTYPE_F32 = 1 };

/* per-particle flag bits */
enum { GC_FLAG_OUT_OF_GRID = 1, GC_FLAG_AXIS = 2, GC_FLAG_NONFINITE = 4 };

typedef struct {
    int32_t precision;      /* GC_PREC_* */
    int32_t device;         /* CUDA device ordinal */
    void *stream;           /* cudaStream_t used for all work; NULL = legacy default stream */
    uint32_t seed;          /* Philox key word 1 (word 0 is the particle id) */
    int32_t collision_form; /* 0: exponential free path (default); 1: per-step draw of Eq. 9 */
    int32_t drift_mask;     /* 0: full Eqs. 1-2; 1: dR/dt = v_par b only */
    int32_t no_scatter;     /* 1: collisions off */
    int32_t no_rebirth;     /* 1: rebirth off */
    uint32_t id_base;       /* id of the first injected particle (shards of one run use
                               disjoint id ranges, so their Philox streams differ) */
    double charge;          /* particle charge, C (0 selects the electron, -e) */
    double mass;            /* rest mass, kg (0 selects the electron mass) */
    double dt_init;         /* step (s) used to build the start-up history at injection */
    double wind_u;          /* 0: collisions in the fixed frame, elastic there (default);
                               > 0: in the frame of a radial solar wind of this speed (m/s),
                               elastic there (Sect. 3.2, adiabatic cooling): a boost along b
                               by u.b, the pitch redraw, and the boost back */
} gc_options;

/* Spherical grid of node values, Sect. 2.2 (trilinear interpolation of the field at the
 * particle position). Node (i_r, i_theta, i_phi) sits at r = r_min + i_r dr
 * (dr = (r_max - r_min)/(n_r - 1)), theta = i_theta pi/(n_th - 1) (poles included),
 * phi = 2 pi i_phi / n_ph (periodic). Layout: [n_ph][n_th][n_r][8] with channels
 * Bx, By, Bz (T), Ex, Ey, Ez (V/m), |B| (T), Phi (V, used by two-fluid fields only); vector
 * components are Cartesian. */
typedef struct {
    int32_t n_r, n_th, n_ph;
    int32_t dtype;          /* GC_DTYPE_*; FP32_MIXED contexts convert F64 data to F32 */
    double r_min_au, r_max_au;
    int32_t ideal;          /* 1: E_par := 0 after interpolation (ideal Ohm's law);
                               0: E_par = E.b of the interpolated E;
                               2: two-fluid Ohm's law, E = -u x B - grad(p)/(e n) with
                               p = p(n) (Sect. 2.2): E_par = -b.grad(Phi) from the potential
                               channel's interpolant (the E channels carry -u x B) */
    int32_t pad0;
} gc_grid_desc;

/* One ensemble (Sect. 3): count electrons injected at one site, all with one energy or a
 * power-law spectrum; mu0 and the spectrum draws come from each particle's Philox stream.
 * Particles are reborn at the site with their initial momentum when they leave
 * [r_in, r_out]. Ids are assigned contiguously across ensembles in call order. */
typedef struct {
    int64_t count;
    double r0_au, lat_deg, lon_deg; /* injection site */
    double E0_keV;                  /* mono-energetic kinetic energy */
    double E_lo_keV, E_hi_keV, E_index; /* spectrum dN/dE ~ E^-index on [E_lo, E_hi] */
    double lambda_au;               /* field-aligned mean free path (Sect. 2.3) */
    double r_in_au, r_out_au;       /* shell; r_in <= 0 selects r0 */
    int32_t energy_law;             /* 0: mono, 1: power law */
    int32_t mu_law;                 /* 0: mu0 uniform on (0, 1]; 1: mu0 = 1 */
    int32_t scatter_law;            /* 0: mu = 1 - 2a (Eq. 10); 1: mu = +-sqrt(a) (Eq. 12) */
    int32_t pad0;
} gc_ensemble_desc;

/* Snapshot tallies (Sect. 3): every `cadence` steps of the global step counter, each
 * particle born at t >= t_start adds one sample. */
typedef struct {
    int32_t cadence, n_mu, n_E, n_r, n_age, pad0;
    double t_start_s;
    double E_lo_keV, E_hi_keV; /* log-spaced energy bins */
    double r_lo_au, r_hi_au;   /* linear radial bins */
    double age_max_s;          /* linear age bins on [0, age_max) */
    double rwin_lo_au, rwin_hi_au; /* window of the age-energy and young-PAD tallies */
    double age_young_s;        /* young-PAD: age < age_young and >= 1 collision */
} gc_tally_desc;

/* Host buffers for gc_tally (caller-owned; sizes follow the armed descriptor, n_ens is
 * the number of ensembles injected so far). */
typedef struct {
    uint32_t *h_mer;  /* [n_ens][n_mu][n_E][n_r] counts */
    uint32_t *h_age;  /* [n_ens][n_age][n_E] counts in the radial window */
    uint32_t *h_pad;  /* [n_ens][n_mu] young particles with >= 1 collision in the window */
    uint64_t *m_cnt;  /* [n_ens][n_r] samples per radial bin */
    uint64_t *m_sin2; /* [n_ens][n_r] sum of sin^2(alpha) in units of 2^-32 */
    uint64_t *n_seen; /* [2] samples taken, samples outside the mu-E-r ranges */
} gc_tally_out;

/* Structure-of-arrays particle state (host, caller-owned, n entries each; F0/F1 are
 * [4][n]: dR/dt (3) and d(gamma v_par)/dt of F^n and F^{n-1}). */
typedef struct {
    int64_t n;
    double *x, *y, *z;  /* guiding-centre position, m */
    double *u;          /* gamma v_par, m/s */
    double *mub;        /* magnetic moment, J/T */
    double *F0, *F1;    /* [4][n] */
    double *vpar;       /* v_par at the current state, m/s */
    double *s_rem;      /* remaining free path, m */
    double *h_prev;     /* step that separates X^{n-1} from X^n, s */
    double *t_birth;    /* time of (re)birth, s */
    double *u_inj, *mub_inj; /* injection momentum, restored at rebirth */
    uint32_t *id, *ens, *event, *ncoll, *flags;
} gc_particle_soa;

typedef struct {
    int64_t n_particles;
    int64_t step;           /* global step counter */
    double t;               /* simulated time, s */
    uint64_t particle_steps;
    uint64_t collisions;
    uint64_t rebirths;
    uint32_t flags_or;      /* OR of all particle flags seen */
    uint32_t pad0;
    uint64_t kernel_launches; /* kernels this context launched */
    uint64_t push_launches;   /* launches of the push kernel */
    double push_ms;           /* summed device time of those launches (CUDA events) */
    uint64_t sorts;           /* cell sorts performed */
    double sort_ms;           /* summed device time of the sorts */
    uint64_t field_evals;     /* field samples of the split-step push (points) */
    double field_ms;          /* summed device time of those sample launches */
} gc_stats_out;

/* Create a context on opt->device. *out receives the handle. */
int gc_create(gc_ctx **out, const gc_options *opt);
void gc_destroy(gc_ctx *ctx);
/* Message of the calling thread's last error ("" if none). Valid until the next call. */
const char *gc_last_error(void);

/* Copy the field grid into context-owned device memory. data points to
 * n_ph*n_th*n_r*8 values of g->dtype, on the host, or on this device if
 * data_on_device != 0 (then read on the context's stream). */
int gc_field_load(gc_ctx *ctx, const gc_grid_desc *g, const void *data, int data_on_device);

/* Make the loaded field time dependent (Eqs. 1-2 keep their time-derivative terms, Sect. 2):
 * data is a second snapshot on the same grid, with the same layout, dtype and descriptor as
 * the last gc_field_load, and [t0_s, t1_s] the simulated times of the two snapshots. Every
 * field evaluation then blends the two linearly in time, and the derivatives dB/dt and dE/dt
 * are the snapshots' difference over (t1_s - t0_s). Outside the window the field holds the
 * nearer snapshot and its time derivatives are zero. The context copies the data (and converts it to its precision); a later
 * gc_field_load makes the field steady again. GC_ERR_STATE without a first snapshot,
 * GC_ERR_INVALID unless t0_s < t1_s are finite, GC_ERR_UNSUPPORTED while a split-step field
 * source (gc_field_select) is selected. */
int gc_field_load_next(gc_ctx *ctx, const void *data, int data_on_device, double t0_s, double t1_s);

/* Inject the ensembles (Sect. 3) at the current time; needs a loaded field. Each
 * particle's mu0 (and energy for a spectrum) comes from Philox events 0 and 1 of its
 * stream; its free path is drawn, and the start-up history is built with dt_init. */
int gc_particles_inject(gc_ctx *ctx, const gc_ensemble_desc *e, int n_ens);

/* Advance every particle by n_steps steps of dt seconds (Eqs. 1-6), with scattering
 * (Eqs. 9-10/12), rebirth and the armed tallies. lambda_au > 0 overrides every
 * ensemble's mean free path for this call; <= 0 uses the per-ensemble values.
 * Synchronises the stream; GC_ERR_DEVICE_ANOMALY if any particle was flagged. */
int gc_advance(gc_ctx *ctx, double dt, int64_t n_steps, double lambda_au);

/* Snapshot tallies (Sect. 3: every `cadence` steps, the particles (re)born at or after
 * t_start_s are binned by pitch cosine, kinetic energy and r; by age and energy inside the
 * [rwin_lo, rwin_hi) window at 1 AU; young pitch distributions; sin^2 alpha per r bin). If
 * out != NULL the current counts are copied to the host first; then, if arm != NULL, the
 * tallies are (re)armed with that descriptor and zeroed. */
int gc_tally(gc_ctx *ctx, const gc_tally_desc *arm, gc_tally_out *out);

/* Copy the particle state to / from host arrays (in id order of the last set/inject;
 * the library may reorder particles internally, get returns them in that order).
 * Every array of the gc_particle_soa holds out_host->n / in_host->n entries (F0 and F1
 * as [4][n]); pinned host memory makes the copies fastest. get: n must equal the
 * context's particle count (GC_ERR_INVALID otherwise); a NULL array is skipped. set:
 * replaces the whole state (every array required; ensemble ids must name injected
 * ensembles, else GC_ERR_INVALID and the old state is kept); the next gc_advance treats
 * the state as unsorted. Both synchronise the context's stream before returning. Used for
 * checkpoints (with gc_set_clock) and for host-side analysis. */
int gc_particles_get(gc_ctx *ctx, gc_particle_soa *out_host);
int gc_particles_set(gc_ctx *ctx, const gc_particle_soa *in_host);

/* Counters and time. */
int gc_stats(gc_ctx *ctx, gc_stats_out *out);

/* Set the simulated time (s) and the global step counter, e.g. when resuming from a
 * checkpoint written with gc_particles_get; tally cadence and birth times follow them. */
int gc_set_clock(gc_ctx *ctx, double t, int64_t step);

/* Launch shape: threads per block (multiple of 32 up to 128; 0 = keep), steps per kernel
 * launch (0 = keep), the period of the cell sort in steps (0 = never), and the grid in
 * resident waves of blocks (k >= 1: k x SMs x resident blocks per SM, each thread walking
 * several particles; 0: one thread per particle). */
int gc_set_launch(gc_ctx *ctx, int block, int steps_per_launch, int sort_every, int grid_waves);

/* Replay gc_advance from CUDA graphs (enable != 0). The first call of a given pattern
 * (dt, n_steps, lambda, launch shape, tallies, buffers) captures its sorts and push
 * launches into a graph on an internal stream; later calls with the same pattern replay
 * it on the context's stream with the clock read from device memory. Results are those of
 * the direct path. A context caches up to four graphs; reallocation drops them. */
int gc_set_graph(gc_ctx *ctx, int enable);

/* Result of gc_autotune. */
typedef struct {
    int32_t block, grid_waves, steps_per_launch, sort_every;
    double particle_steps_per_s; /* measured rate of the chosen shape */
    int32_t trials, pad0;
} gc_launch_choice;

/* Time trial_steps steps of dt for each launch shape of a small search space (block size,
 * grid waves, cell-sort period) from a snapshot of the current state, keep the fastest
 * with gc_set_launch, and restore the state, clock, counters and tallies as they were. */
int gc_autotune(gc_ctx *ctx, double dt, int64_t trial_steps, gc_launch_choice *best);

/* Sort the particles by grid cell now (results are unchanged: every random draw is keyed
 * by particle id and every tally is an integer sum). */
int gc_sort(gc_ctx *ctx);

/* Library version (major * 10000 + minor * 100 + patch). */
int gc_version(void);

/* Measured fused multiply-add throughput of GPU `device`, in TFLOP/s (an FMA counts as two
 * flops): *fp32_tflops for float, *fp64_tflops for double. These are the peaks the push
 * kernels are measured against (no counterpart in the paper). Each rate is the best of ten
 * launches of about 10 ms of independent FMA chains on every SM, timed with CUDA events on a
 * stream of its own, which is created, synchronised and destroyed inside the call; the
 * current device is restored. GC_ERR_INVALID for a missing device or a null pointer,
 * GC_ERR_CUDA if a launch fails. */
int gc_fma_peak(int device, double *fp32_tflops, double *fp64_tflops);

/* BF16 tensor-core GEMM used by the neural-field training: C = A B^T with A (M x K) and
 * B (N x K) bf16 row-major on the device (K contiguous, 16-byte aligned), FP32 accumulate,
 * C (M x N) FP32 row-major on the device (16-byte aligned). accumulate != 0 adds into C
 * with atomics, which split_k > 1 requires (K is then split over split_k CTAs per tile).
 * M and N must be multiples of 128 and K of 64. Runs on stream and synchronises it. */
int gc_gemm_bf16_tn(const void *A, const void *B, float *C, int M, int N, int K, int split_k, int accumulate,
                    void *stream);

/* The same GEMM with either operand stored MN-major: a_mn = 1 means A is given as its
 * transpose (row-major K x M, M contiguous), b_mn = 1 that B is row-major K x N. This is how
 * the training's backward products read activations and gradients without transposing
 * them: dW = dZ^T H (both MN-major) and dH = dZ W (B MN-major). Same rules and errors as
 * gc_gemm_bf16_tn, plus GC_ERR_INVALID for a_mn or b_mn outside {0, 1}. */
int gc_gemm_bf16(const void *A, int a_mn, const void *B, int b_mn, float *C, int M, int N, int K, int split_k,
                 int accumulate, void *stream);

/* ---------------------------------------------------------------------------------------
 * Neural field (north of the grid: an alternative field source). A SIREN (sine-activated
 * MLP, Sitzmann et al. 2020) 3 -> 256 -> 256 -> 256 -> 256 -> 8 maps x = R / r_max to the
 * grid's eight channels [B, E, |B|, Phi] scaled to O(1):
 *   y_B = B (r / 1 AU)^2 / B_scale, y_E = E (r / 1 AU) / E_scale,
 *   y_|B| = |B| (r / 1 AU)^2 / B_scale, y_Phi = Phi / (E_scale 1 AU).
 * Layers: z1 = w0 (W1 x + b1), h_k = sin z_k, z_k = W_k h_{k-1} + b_k, y = W5 h4 + b5.
 * Parameters are FP32 (GC_SIREN_NPARAMS floats, in this order: W1 [256][3], b1 [256],
 * W2 [256][256] ([out][in]), b2, W3, b3, W4, b4, W5 [8][256], b5 [8]). Evaluation and
 * training use BF16 copies of W2..W5 and BF16 activations with FP32 accumulation on the
 * tensor cores; W1 and the biases stay FP32. The field's derivatives come from the
 * network's exact Jacobian (three forward-mode tangents). */
#define GC_SIREN_NPARAMS 200456
/* field sources of gc_advance: the grid gathered inside the fused push (default), the
 * neural field, or the grid evaluated through the split-step push's sample buffers (the
 * neural path's machinery with the grid field: it reproduces GC_FIELD_GRID) */
enum { GC_FIELD_GRID = 0, GC_FIELD_SIREN = 1, GC_FIELD_GRID_SAMPLED = 2 };

typedef struct {
    double omega0;   /* frequency of the first layer's sine (30 in Sitzmann et al.) */
    double r_max_au; /* input scaling x = R / r_max */
    double B_scale;  /* T */
    double E_scale;  /* V/m */
} gc_siren_desc;

/* Define the network and load its parameters (host or device FP32 array of
 * GC_SIREN_NPARAMS); resets the Adam moments. */
int gc_siren_set(gc_ctx *ctx, const gc_siren_desc *d, const float *params, int params_on_device);

/* Copy the current FP32 parameters to a caller-owned host array of GC_SIREN_NPARAMS. */
int gc_siren_get(gc_ctx *ctx, float *params_host);

/* Raw network outputs at n points: x_dev (n x 3 FP32, device, already scaled), y_dev
 * (n x 8) and, if J_dev is not NULL, J_dev (n x 8 x 3, dy_o / dx_j). Device buffers are the
 * caller's. GC_ERR_STATE before gc_siren_set. */
int gc_siren_eval(gc_ctx *ctx, const float *x_dev, int64_t n, float *y_dev, float *J_dev);

/* The physical field the push uses at n points x_dev (scaled positions): field_dev
 * (n x 24 FP32, device) = B (T, 3), E (V/m, 3), dB[d][c] = dB_c/dR_d (T/m, 9),
 * dE[d][c] (V/m^2, 9), from the network's outputs and Jacobian by the product rule. */
int gc_siren_field(gc_ctx *ctx, const float *x_dev, int64_t n, float *field_dev);

/* Training targets: the loaded grid's trilinear interpolant of all eight channels at n
 * scaled points x_dev, scaled as the network's outputs, into t_dev (n x 8, device). Needs
 * gc_field_load and gc_siren_set (for the scaling). */
int gc_field_targets(gc_ctx *ctx, const float *x_dev, int64_t n, float *t_dev);

/* Mean squared error over n samples (n a multiple of 128) and all eight outputs, and its
 * gradient with respect to the parameters (grad_dev: GC_SIREN_NPARAMS FP32, device, or NULL
 * to keep it internal), computed by the training's forward and backward passes.
 * x_dev: n x 3, t_dev: n x 8 (device). loss_out: host, may be NULL. */
int gc_siren_loss_grad(gc_ctx *ctx, const float *x_dev, const float *t_dev, int64_t n, float *grad_dev,
                       double *loss_out);

typedef struct {
    const float *samples;      /* n_samples x 3 scaled positions (x = R / r_max) */
    int32_t samples_on_device; /* 1: device pointer, 0: host */
    int32_t pad;
    int64_t batch;             /* samples per Adam step, a multiple of 128 */
    double lr, beta1, beta2, eps; /* Adam (Kingma & Ba 2015) */
} gc_fit_desc;

/* Fit the loaded network to the loaded grid field: targets from gc_field_targets at the
 * samples, then n_epochs passes over the samples in order, one Adam step per batch (a last
 * partial batch is dropped). loss_out (host, n_epochs floats, may be NULL) receives each
 * epoch's mean batch loss measured before the batch's update. */
int gc_field_fit(gc_ctx *ctx, const gc_fit_desc *f, int64_t n_samples, int n_epochs, float *loss_out);

/* Field source of gc_advance and of later injections: GC_FIELD_GRID (default), or one of
 * the split-step sources (FP32_MIXED precision only): GC_FIELD_SIREN (needs gc_siren_set)
 * or GC_FIELD_GRID_SAMPLED. The split-step push advances all particles one evaluation phase
 * per launch (predictor, corrector, post-step tests, then the start-up of the restarted
 * particles, Sect. 2.2) with the field sampled in between; it has no cell sort and no graph
 * replay. Injections under a split-step source take mu_B and the start-up history from that
 * source. */
int gc_field_select(gc_ctx *ctx, int source);

/* Device memory gc_advance_noalloc keeps for its own use on every GPU that loads the
 * library (held until the process exits), and the most ensembles it accepts. */
#define GC_NOALLOC_SCRATCH_BYTES 40960
#define GC_NOALLOC_MAX_ENSEMBLES 256

/* gc_advance_noalloc: advance a particle state that lives in the caller's own device
 * memory, without this library allocating any device memory. The paper has no
 * counterpart; this is an embedding aid. It is meant for callers that cannot let a
 * library call cudaMalloc: a simulation code that reserves the GPU's memory for its own
 * pool and hands out views of its buffers, or a stepping loop that must not pay the
 * device-wide synchronisation an allocation can cause.
 *
 * It runs the push kernel of gc_advance (with scattering and rebirth; no tallies and no
 * cell sort) on:
 *   opt       precision, device, stream, seed and the physics switches (dt_init and
 *             id_base are not used);
 *   g, grid_dev   the field grid already on the device, in the precision's type (F64 for
 *             GC_PREC_FP64, F32 for GC_PREC_FP32_MIXED; there is no conversion);
 *   ens, n_ens    the ensembles the particles were injected with (1..GC_NOALLOC_MAX_
 *             ENSEMBLES; `count` is ignored); every particle's ens id must be < n_ens;
 *   state_dev a gc_particle_soa whose pointers are DEVICE addresses (F0/F1 as [4][n]),
 *             advanced in place, e.g. a copy of what gc_particles_get returned;
 *   t0, step0 the clock of that state (as gc_stats reports it), then dt, n_steps and
 *             lambda_au as for gc_advance;
 *   stats_out optional: collisions, rebirths and flags of this call.
 * The ensemble table, the anomaly flag and the event counters live in one file-scope
 * device array of GC_NOALLOC_SCRATCH_BYTES. The first call on a device (and the first after
 * its context was reset) looks up that array's device address; make that first call before
 * any stream capture on the device.
 * Every call overwrites the array (the status words are cleared at the start of each
 * call), so calls whose work overlaps on the GPU race on it: serialise them. Returns
 * GC_ERR_INVALID for more ensembles than the maximum, a wrong grid type or an ens id out
 * of range (checked on the device before the push reads the table), and
 * GC_ERR_DEVICE_ANOMALY if particles were flagged. It synchronises opt->stream. */
int gc_advance_noalloc(const gc_options *opt, const gc_grid_desc *g, const void *grid_dev,
                       const gc_ensemble_desc *ens, int n_ens, const gc_particle_soa *state_dev,
                       double t0, int64_t step0, double dt, int64_t n_steps, double lambda_au,
                       gc_stats_out *stats_out);

#ifdef __cplusplus
}
#endif

#endif /* GCPUSH_H */
