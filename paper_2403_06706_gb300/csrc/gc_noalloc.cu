// gc_noalloc.cu -- gc_advance_noalloc: the push on caller-owned device memory with no
// device allocation by this library.
//
// Some callers cannot let a library call cudaMalloc: a simulation code that reserves the
// device memory for its own pool and hands out views of it, or a time-stepping loop that
// must not pay the device-wide synchronisation an allocation can cause. This entry point
// runs the same push kernel as gc_advance, but everything the launch needs beyond the
// caller's grid and particle arrays (the ensemble table, the anomaly flag word and the
// event counters) lives in one fixed file-scope device array.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h> // CUcontext and cuCtxGetCurrent's type only; the function comes from the runtime
#include <cuda_runtime.h>

#include "../../include/gcpush.h"
#include "gc_internal.h"

namespace {

// Layout of the scratch: [ensemble table | status block].
constexpr size_t kTableBytes = (size_t)GC_NOALLOC_MAX_ENSEMBLES * sizeof(gcp::EnsDev);
constexpr size_t kStatusOff = (kTableBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kStatusOff + 256; // flags (u32), bad-id flag (u32), 2 x u64
static_assert(kScratchBytes <= GC_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

// The scratch itself. Every call on a device shares it and overwrites it; calls whose
// work overlaps on the GPU (other streams, other host threads) race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

constexpr double kAU = 1.495978707e11;
constexpr double kKeV = 1.602176634e-16;
constexpr double kC = 299792458.0;
constexpr double kQe = -1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kPi = 3.14159265358979323846;

int nfail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    gcp::set_last_error(buf); // reported by gc_last_error()
    return code;
}

// The current CUDA context (the device's primary context once the runtime has used it), or
// nullptr if the driver cannot be asked; cuCtxGetCurrent is looked up through the runtime.
CUcontext current_context()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    static const GetCurrent fn = []() -> GetCurrent {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<GetCurrent>(p);
    }();
    CUcontext c = nullptr;
    return (fn && fn(&c) == CUDA_SUCCESS) ? c : nullptr;
}

// Device address of the scratch on `device` (which must be current). The first call on a
// device looks the symbol up, and so does the first call after that device's context was
// replaced (cudaDeviceReset), since the address belongs to the context; other calls reuse
// the cached address.
int scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices)
        return nfail(GC_ERR_INVALID, "gc_advance_noalloc: device %d out of range", device);
    const CUcontext ctx = current_context();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[device] || !ctx || ctx != g_scratch_ctx[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return nfail(GC_ERR_CUDA, "gc_advance_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_addr[device] = p;
        g_scratch_ctx[device] = ctx;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[device]);
    return GC_OK;
}

// Sets *bad if any particle names an ensemble outside [0, n_ens).
__global__ void check_ensembles(const uint32_t *__restrict__ ens, int64_t n, uint32_t n_ens, uint32_t *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (ens[i] >= n_ens)
            atomicOr(bad, 1u);
}

} // namespace

extern "C" int gc_advance_noalloc(const gc_options *opt, const gc_grid_desc *g, const void *grid_dev,
                                  const gc_ensemble_desc *ens, int n_ens, const gc_particle_soa *sd,
                                  double t0, int64_t step0, double dt, int64_t n_steps,
                                  double lambda_au, gc_stats_out *stats_out)
{
    if (!opt || !g || !grid_dev || !sd || (!ens && n_ens > 0))
        return nfail(GC_ERR_INVALID, "gc_advance_noalloc: null argument");
    if (n_ens < 1 || n_ens > GC_NOALLOC_MAX_ENSEMBLES)
        return nfail(GC_ERR_INVALID, "gc_advance_noalloc: %d ensembles; this entry point takes 1 to %d",
                     n_ens, GC_NOALLOC_MAX_ENSEMBLES);
    if (opt->precision != GC_PREC_FP64 && opt->precision != GC_PREC_FP32_MIXED)
        return nfail(GC_ERR_INVALID, "gc_advance_noalloc: unknown precision %d", opt->precision);
    const int want_dtype = opt->precision == GC_PREC_FP64 ? GC_DTYPE_F64 : GC_DTYPE_F32;
    if (g->dtype != want_dtype)
        return nfail(GC_ERR_INVALID, "gc_advance_noalloc: grid dtype must be %s for this precision "
                     "(no conversion without scratch)", want_dtype == GC_DTYPE_F64 ? "F64" : "F32");
    if (g->n_r < 2 || g->n_th < 2 || g->n_ph < 2 || !(g->r_min_au > 0.0) || !(g->r_max_au > g->r_min_au) ||
        g->ideal < 0 || g->ideal > 2)
        return nfail(GC_ERR_INVALID, "gc_advance_noalloc: bad grid descriptor");
    if ((size_t)g->n_r * g->n_th * g->n_ph * 8 >= ((size_t)1 << 32))
        return nfail(GC_ERR_INVALID, "gc_advance_noalloc: grid exceeds the 2^32 index range");
    if (!(dt > 0.0) || !std::isfinite(dt) || n_steps < 0 || sd->n < 0 || step0 < 0)
        return nfail(GC_ERR_INVALID, "gc_advance_noalloc: need dt > 0, n_steps >= 0, n >= 0");
    const void *ptrs[] = {sd->x, sd->y, sd->z, sd->u, sd->mub, sd->F0, sd->F1, sd->vpar, sd->s_rem,
                          sd->h_prev, sd->t_birth, sd->u_inj, sd->mub_inj, sd->id, sd->ens,
                          sd->event, sd->ncoll, sd->flags};
    for (const void *p : ptrs)
        if (!p && sd->n > 0)
            return nfail(GC_ERR_INVALID, "gc_advance_noalloc: every state array is required");
    for (int k = 0; k < n_ens; ++k)
        if (!(ens[k].lambda_au > 0.0) || !(ens[k].r0_au > 0.0) || ens[k].scatter_law < 0 || ens[k].scatter_law > 1)
            return nfail(GC_ERR_INVALID, "gc_advance_noalloc: bad ensemble descriptor %d", k);

    cudaError_t e = cudaSetDevice(opt->device);
    if (e != cudaSuccess)
        return nfail(GC_ERR_CUDA, "gc_advance_noalloc: cudaSetDevice: %s", cudaGetErrorString(e));
    unsigned char *scr = nullptr;
    int rc = scratch_address(opt->device, &scr);
    if (rc != GC_OK)
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(opt->stream);

    // ensemble table (the same conversion as the context path) into the scratch
    gcp::EnsDev table[GC_NOALLOC_MAX_ENSEMBLES];
    for (int k = 0; k < n_ens; ++k) {
        const gc_ensemble_desc &d = ens[k];
        gcp::EnsDev E{};
        const double r0 = d.r0_au * kAU;
        const double lat = d.lat_deg * (kPi / 180.0);
        const double lon = d.lon_deg * (kPi / 180.0);
        E.R0[0] = r0 * cos(lat) * cos(lon);
        E.R0[1] = r0 * cos(lat) * sin(lon);
        E.R0[2] = r0 * sin(lat);
        E.lambda = d.lambda_au * kAU;
        E.r_in = (d.r_in_au > 0.0 ? d.r_in_au : d.r0_au) * kAU;
        E.r_out = d.r_out_au * kAU;
        E.E0 = d.E0_keV * kKeV;
        E.E_lo = d.E_lo_keV * kKeV;
        E.E_hi = d.E_hi_keV * kKeV;
        E.E_index = d.E_index;
        E.energy_law = d.energy_law;
        E.mu_law = d.mu_law;
        E.scatter_law = d.scatter_law;
        for (int a = 0; a < 3; ++a) {
            E.R0_hi[a] = (float)E.R0[a];
            E.R0_lo[a] = (float)(E.R0[a] - (double)E.R0_hi[a]);
        }
        E.r_in2 = (float)(E.r_in * E.r_in);
        E.r_out2 = (float)(E.r_out * E.r_out);
        E.lambda_f = (float)E.lambda;
        table[k] = E;
    }
    gcp::EnsDev *d_table = reinterpret_cast<gcp::EnsDev *>(scr);
    uint32_t *d_flags = reinterpret_cast<uint32_t *>(scr + kStatusOff);
    uint32_t *d_bad = d_flags + 1;
    unsigned long long *d_counters = reinterpret_cast<unsigned long long *>(scr + kStatusOff + 8);
    // the status block must start at zero on every call
    if ((e = cudaMemsetAsync(scr + kStatusOff, 0, 256, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_table, table, (size_t)n_ens * sizeof(gcp::EnsDev), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return nfail(GC_ERR_CUDA, "gc_advance_noalloc: %s", cudaGetErrorString(e));

    // every particle must name an ensemble of the table before the push reads it
    if (sd->n > 0) {
        const int grid = (int)std::min<int64_t>((sd->n + 255) / 256, 152 * 8);
        check_ensembles<<<grid, 256, 0, s>>>(sd->ens, sd->n, (uint32_t)n_ens, d_bad);
        uint32_t bad = 0;
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return nfail(GC_ERR_CUDA, "gc_advance_noalloc: %s", cudaGetErrorString(e));
        if (bad)
            return nfail(GC_ERR_INVALID, "gc_advance_noalloc: a particle names an ensemble >= %d", n_ens);
    }

    gcp::GridHost gh{};
    gh.nodes = grid_dev;
    gh.n_r = g->n_r;
    gh.n_th = g->n_th;
    gh.n_ph = g->n_ph;
    gh.ideal = g->ideal;
    gh.is_f64 = opt->precision == GC_PREC_FP64;
    gh.r_min = g->r_min_au * kAU;
    gh.dr = (g->r_max_au * kAU - g->r_min_au * kAU) / (double)(g->n_r - 1);
    gh.dth = kPi / (double)(g->n_th - 1);
    gh.dph = 2.0 * kPi / (double)g->n_ph;
    const double charge = opt->charge == 0.0 ? kQe : opt->charge;
    const double mass = opt->mass > 0.0 ? opt->mass : kMe;
    gcp::PhysHost ph{};
    ph.qm = charge / mass;
    ph.inv_m = 1.0 / mass;
    ph.inv_c2 = 1.0 / (kC * kC);
    ph.drift_mask = opt->drift_mask;

    gcp::PushParams P{};
    P.st.x = sd->x; P.st.y = sd->y; P.st.z = sd->z; P.st.u = sd->u; P.st.mub = sd->mub;
    P.st.F0 = sd->F0; P.st.F1 = sd->F1; P.st.vpar = sd->vpar; P.st.s_rem = sd->s_rem;
    P.st.h_prev = sd->h_prev; P.st.t_birth = sd->t_birth; P.st.u_inj = sd->u_inj;
    P.st.mub_inj = sd->mub_inj; P.st.id = sd->id; P.st.ens = sd->ens; P.st.event = sd->event;
    P.st.ncoll = sd->ncoll; P.st.flags = sd->flags;
    P.st.n = sd->n;
    P.st.cap = sd->n; // F0/F1 rows are [4][n] in the caller's arrays
    P.ens = d_table;
    P.dt = dt;
    P.t0 = t0;
    P.collision_form = opt->collision_form;
    P.no_scatter = opt->no_scatter;
    P.no_rebirth = opt->no_rebirth;
    P.lambda_override = lambda_au > 0.0 ? lambda_au * kAU : 0.0;
    P.wind_u = opt->wind_u;
    P.seed = opt->seed;
    P.m = mass;
    P.c2 = kC * kC;
    P.two_over_m = 2.0 / mass;
    P.inv_c2 = 1.0 / (kC * kC);
    P.tally_on = 0;
    P.gflags = d_flags;
    P.counters = d_counters;

    const int block = 128;
    int nb = gcp::push_max_blocks_per_sm(opt->precision, block, false, g->ideal == 2);
    cudaGetLastError(); // the occupancy query's status is not this call's
    if (nb < 1) nb = 1;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, opt->device);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((sd->n + block - 1) / block, (int64_t)sms * nb));
    int64_t done = 0;
    while (sd->n > 0 && done < n_steps) {
        const int64_t chunk = std::min<int64_t>(n_steps - done, 2000);
        P.step0 = step0 + done;
        P.kbase = done;
        P.n_steps = (int32_t)chunk;
        if ((e = gcp::launch_push(opt->precision, gh, ph, P, block, grid, s)) != cudaSuccess)
            return nfail(GC_ERR_CUDA, "gc_advance_noalloc: launch: %s", cudaGetErrorString(e));
        done += chunk;
    }
    uint32_t flags = 0;
    unsigned long long counters[2] = {0, 0};
    if ((e = cudaMemcpyAsync(&flags, d_flags, sizeof(flags), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(counters, d_counters, sizeof(counters), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return nfail(GC_ERR_CUDA, "gc_advance_noalloc: %s", cudaGetErrorString(e));
    if (stats_out) {
        *stats_out = gc_stats_out{};
        stats_out->n_particles = sd->n;
        stats_out->step = step0 + n_steps;
        stats_out->t = t0 + (double)n_steps * dt;
        stats_out->particle_steps = (uint64_t)sd->n * (uint64_t)n_steps;
        stats_out->collisions = counters[0];
        stats_out->rebirths = counters[1];
        stats_out->flags_or = flags;
    }
    if (flags)
        return nfail(GC_ERR_DEVICE_ANOMALY, "gc_advance_noalloc: particles flagged (0x%x)", flags);
    return GC_OK;
}
