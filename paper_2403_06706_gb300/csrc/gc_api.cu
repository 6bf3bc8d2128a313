// gc_api.cu -- C ABI of libgcpush (see include/gcpush.h).
//
// Host side only: context, device memory ownership, argument checks, launch loop.
// Every computation on particles runs in the kernels of gc_push.cu / gc_sort.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gcpush.h"
#include "gc_internal.h"
#include "gc_neural.h"
#include "gc_sort.h"

namespace {

constexpr double kAU = 1.495978707e11;      // m
constexpr double kKeV = 1.602176634e-16;    // J
constexpr double kC = 299792458.0;          // m/s
constexpr double kQe = -1.602176634e-19;    // electron charge, C
constexpr double kMe = 9.1093837015e-31;    // electron mass, kg
constexpr double kPi = 3.14159265358979323846;

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? GC_ERR_NOMEM : GC_ERR_CUDA,          \
                        "%s: %s", #expr, cudaGetErrorString(e_));                              \
    } while (0)

#define TRY(expr)                                                                              \
    do {                                                                                       \
        int r_ = (expr);                                                                       \
        if (r_ != GC_OK)                                                                       \
            return r_;                                                                         \
    } while (0)

// convert node arrays between precisions on the device
__global__ void convert_nodes(const double *src, float *dst, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}
__global__ void convert_nodes(const float *src, double *dst, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

const int kF64Fields = 13; // x y z u mub vpar s_rem h_prev t_birth u_inj mub_inj + F0, F1 rows
const int kU32Fields = 5;

// one timed interval (a push launch or a sort) bracketed by two events
struct Timed {
    cudaEvent_t a, b;
    int kind; // 0 push, 1 sort
};

struct LaunchCounts {
    uint64_t kernels = 0, pushes = 0, sorts = 0;
};

// A captured advance: valid for one call pattern and one pair of state buffers.
struct GraphKey {
    double dt, lambda_au;
    int64_t n_steps, n, cap, steps_since_sort, n_ens;
    int block, grid_waves, steps_per_launch, sort_every, tally_on;
    const void *st_x, *alt_x, *tally, *grid, *ens;
    bool operator==(const GraphKey &o) const
    {
        return dt == o.dt && lambda_au == o.lambda_au && n_steps == o.n_steps && n == o.n && cap == o.cap &&
               steps_since_sort == o.steps_since_sort && n_ens == o.n_ens && block == o.block &&
               grid_waves == o.grid_waves && steps_per_launch == o.steps_per_launch &&
               sort_every == o.sort_every && tally_on == o.tally_on && st_x == o.st_x && alt_x == o.alt_x &&
               tally == o.tally && grid == o.grid && ens == o.ens;
    }
};

struct GraphEntry {
    GraphKey key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<Timed> timed; // events owned by this entry
    LaunchCounts counts;
    gcp::StateDev st_after{}, alt_after{};
    int64_t steps_since_sort_after = 0;
};

} // namespace

void gcp::set_last_error(const char *msg) { g_err = msg; }

struct gc_ctx {
    gc_options opt{};
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;

    // field (d_grid1: the second snapshot of a time-dependent field)
    void *d_grid = nullptr;
    void *d_grid1 = nullptr;
    gc_grid_desc grid{};
    gcp::GridHost gh{};
    bool has_field = false;

    // particles (structure of arrays; F0/F1 are [4][cap])
    gcp::StateDev st{};
    int64_t n = 0, cap = 0;
    std::vector<gcp::EnsDev> ens;
    gcp::EnsDev *d_ens = nullptr;
    int64_t ens_cap = 0;
    uint32_t next_id = 0;

    // time
    double t = 0.0;
    int64_t step = 0;

    // tallies
    bool tally_on = false;
    gc_tally_desc tdesc{};
    gcp::TallyDev tdev{};
    void *d_tally = nullptr;
    size_t tally_bytes = 0;
    size_t off_age = 0, off_pad = 0, off_cnt = 0, off_sin2 = 0, off_seen = 0;

    // status
    uint32_t *d_flags = nullptr;          // [1]
    unsigned long long *d_counters = nullptr; // [2]
    uint32_t *h_flags = nullptr;          // pinned mirror
    unsigned long long *h_counters = nullptr;
    uint64_t collisions = 0, rebirths = 0, particle_steps = 0;
    uint32_t flags_or = 0;

    // instrumentation: CUDA events around push launches and sorts
    std::vector<cudaEvent_t> ev_pool;
    std::vector<Timed> pending; // intervals recorded since the last harvest (pool events)
    size_t ev_next = 0;
    uint64_t kernel_launches = 0, push_launches = 0, sorts = 0;
    double push_ms = 0.0, sort_ms = 0.0;

    // graph replay: clock words read by the push kernel, captured graphs
    bool use_graph = false;
    cudaStream_t cap_stream = nullptr;
    double *d_clock = nullptr, *h_clock = nullptr;
    std::vector<GraphEntry *> graphs;

    // order of the particle slots
    bool in_id_order = true; // slot k holds the k-th smallest id
    bool ids_dense = true;   // ids are a permutation of [id_lo, id_lo + n)
    uint32_t id_lo = 0;

    // neural field (SIREN) and the field source of gc_advance
    gcn::Neural nn;
    int field_source = GC_FIELD_GRID;

    // split-step push buffers (sources other than the inline grid gather)
    int64_t split_cap = 0;
    float *d_req = nullptr, *d_reqR = nullptr, *d_S = nullptr, *d_SR = nullptr;
    int32_t *d_list = nullptr, *d_count = nullptr;
    uint64_t field_evals = 0;
    double field_ms = 0.0;

    // launch shape
    int block = 128;
    int grid_waves = 1;      // resident waves of blocks (0: one thread per particle)
    int blocks_per_sm[5] = {0, 0, 0, 0, 0}; // occupancy per block size / 32, cached
    int steps_per_launch = 2000;
    int sort_every = 0;
    int64_t steps_since_sort = 0;
    gcp::SortWork sortw{};

    gcp::PhysHost phys() const
    {
        gcp::PhysHost p;
        p.qm = opt.charge / opt.mass;
        p.inv_m = 1.0 / opt.mass;
        p.inv_c2 = 1.0 / (kC * kC);
        p.drift_mask = opt.drift_mask;
        return p;
    }
};

namespace {

int set_device(gc_ctx *c)
{
    CUDA_TRY(cudaSetDevice(c->device));
    return GC_OK;
}

void free_state(gcp::StateDev &s)
{
    double **d[] = {&s.x, &s.y, &s.z, &s.u, &s.mub, &s.vpar, &s.s_rem, &s.h_prev, &s.t_birth,
                    &s.u_inj, &s.mub_inj, &s.F0, &s.F1};
    for (double **p : d) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    uint32_t **u[] = {&s.id, &s.ens, &s.event, &s.ncoll, &s.flags};
    for (uint32_t **p : u) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
}

// Grow the particle arrays to hold `need` particles, keeping the first c->n.
void drop_graphs(gc_ctx *c);

int reserve(gc_ctx *c, int64_t need)
{
    if (need <= c->cap)
        return GC_OK;
    drop_graphs(c); // captured graphs hold the old buffers
    int64_t cap = std::max<int64_t>(need, c->cap + c->cap / 2);
    gcp::StateDev ns{};
    double **dd[] = {&ns.x, &ns.y, &ns.z, &ns.u, &ns.mub, &ns.vpar, &ns.s_rem, &ns.h_prev,
                     &ns.t_birth, &ns.u_inj, &ns.mub_inj};
    double *const od[] = {c->st.x, c->st.y, c->st.z, c->st.u, c->st.mub, c->st.vpar, c->st.s_rem,
                          c->st.h_prev, c->st.t_birth, c->st.u_inj, c->st.mub_inj};
    for (int k = 0; k < 11; ++k) {
        cudaError_t e = cudaMalloc(dd[k], (size_t)cap * sizeof(double));
        if (e != cudaSuccess) {
            free_state(ns);
            return fail(GC_ERR_NOMEM, "cudaMalloc(%lld particles): %s", (long long)cap, cudaGetErrorString(e));
        }
        if (c->n)
            CUDA_TRY(cudaMemcpyAsync(*dd[k], od[k], (size_t)c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    }
    double **ff[] = {&ns.F0, &ns.F1};
    double *const of[] = {c->st.F0, c->st.F1};
    for (int k = 0; k < 2; ++k) {
        cudaError_t e = cudaMalloc(ff[k], (size_t)cap * 4 * sizeof(double));
        if (e != cudaSuccess) {
            free_state(ns);
            return fail(GC_ERR_NOMEM, "cudaMalloc(F rows): %s", cudaGetErrorString(e));
        }
        if (c->n)
            CUDA_TRY(cudaMemcpy2DAsync(*ff[k], (size_t)cap * sizeof(double), of[k], (size_t)c->cap * sizeof(double),
                                       (size_t)c->n * sizeof(double), 4, cudaMemcpyDeviceToDevice, c->stream));
    }
    uint32_t **uu[] = {&ns.id, &ns.ens, &ns.event, &ns.ncoll, &ns.flags};
    uint32_t *const ou[] = {c->st.id, c->st.ens, c->st.event, c->st.ncoll, c->st.flags};
    for (int k = 0; k < kU32Fields; ++k) {
        cudaError_t e = cudaMalloc(uu[k], (size_t)cap * sizeof(uint32_t));
        if (e != cudaSuccess) {
            free_state(ns);
            return fail(GC_ERR_NOMEM, "cudaMalloc(u32 state): %s", cudaGetErrorString(e));
        }
        if (c->n)
            CUDA_TRY(cudaMemcpyAsync(*uu[k], ou[k], (size_t)c->n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    free_state(c->st);
    ns.n = c->n;
    ns.cap = cap;
    c->st = ns;
    c->cap = cap;
    (void)kF64Fields;
    return GC_OK;
}

int upload_ensembles(gc_ctx *c)
{
    drop_graphs(c);
    if ((int64_t)c->ens.size() > c->ens_cap) {
        if (c->d_ens) cudaFree(c->d_ens);
        c->d_ens = nullptr;
        c->ens_cap = std::max<int64_t>(64, (int64_t)c->ens.size() * 2);
        CUDA_TRY(cudaMalloc(&c->d_ens, (size_t)c->ens_cap * sizeof(gcp::EnsDev)));
    }
    CUDA_TRY(cudaMemcpyAsync(c->d_ens, c->ens.data(), c->ens.size() * sizeof(gcp::EnsDev),
                             cudaMemcpyHostToDevice, c->stream));
    return GC_OK;
}

// sum the device times of recorded intervals (their stream must be synchronised)
void harvest(gc_ctx *c, const std::vector<Timed> &tl)
{
    for (const Timed &t : tl) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess)
            (t.kind == 0 ? c->push_ms : (t.kind == 1 ? c->sort_ms : c->field_ms)) += ms;
    }
    cudaGetLastError(); // a timing that could not be read is not an error of the next call
}

// read back the status words of the last launches (synchronises the stream)
int collect_status(gc_ctx *c, bool *anomaly)
{
    CUDA_TRY(cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->h_counters, c->d_counters, 2 * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    harvest(c, c->pending);
    c->pending.clear();
    c->ev_next = 0;
    const uint32_t f = *c->h_flags;
    c->flags_or |= f;
    c->collisions += c->h_counters[0];
    c->rebirths += c->h_counters[1];
    CUDA_TRY(cudaMemsetAsync(c->d_flags, 0, sizeof(uint32_t), c->stream));
    CUDA_TRY(cudaMemsetAsync(c->d_counters, 0, 2 * sizeof(unsigned long long), c->stream));
    if (anomaly)
        *anomaly = (f != 0);
    return GC_OK;
}

// Two events for one interval: from the context's pool (owned == nullptr, harvested by
// collect_status) or created for, and owned by, a captured graph.
int new_interval(gc_ctx *c, int kind, std::vector<Timed> *owned, Timed *out)
{
    out->kind = kind;
    if (owned) {
        CUDA_TRY(cudaEventCreate(&out->a));
        CUDA_TRY(cudaEventCreate(&out->b));
        owned->push_back(*out);
        return GC_OK;
    }
    while (c->ev_pool.size() < c->ev_next + 2) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        c->ev_pool.push_back(e);
    }
    out->a = c->ev_pool[c->ev_next];
    out->b = c->ev_pool[c->ev_next + 1];
    c->ev_next += 2;
    c->pending.push_back(*out);
    return GC_OK;
}

int do_sort(gc_ctx *c, cudaStream_t s, std::vector<Timed> *owned, LaunchCounts *lc)
{
    Timed t;
    TRY(new_interval(c, 1, owned, &t));
    CUDA_TRY(cudaEventRecord(t.a, s));
    cudaError_t e = gcp::sort_by_cell(c->sortw, c->st, c->gh, (int)c->ens.size(), s);
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? GC_ERR_NOMEM : GC_ERR_CUDA, "cell sort: %s",
                    cudaGetErrorString(e));
    CUDA_TRY(cudaEventRecord(t.b, s));
    lc->kernels += gcp::kSortKernels;
    lc->sorts += 1;
    c->steps_since_sort = 0;
    c->in_id_order = false;
    return GC_OK;
}

int push_grid(gc_ctx *c)
{
    int &nb = c->blocks_per_sm[c->block / 32];
    if (nb <= 0) {
        nb = gcp::push_max_blocks_per_sm(c->opt.precision, c->block, c->gh.nodes1 != nullptr,
                                        c->gh.ideal == 2);
        cudaGetLastError(); // an occupancy query failure only means "one block"
        if (nb < 1) nb = 1;
    }
    const int64_t want = (c->n + c->block - 1) / c->block;
    if (c->grid_waves <= 0)
        return (int)std::min<int64_t>(want, 0x7FFFFFFF);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c->grid_waves * c->sm_count * nb));
}

// Enqueue the launches of one advance on stream s: cell sorts on schedule and push
// launches of at most steps_per_launch steps. clock_dev != nullptr makes the kernels take
// the clock from device memory (graph capture).
int enqueue_advance(gc_ctx *c, cudaStream_t s, double dt, int64_t n_steps, double lambda_au,
                    const double *clock_dev, std::vector<Timed> *owned, LaunchCounts *lc)
{
    const int grid = push_grid(c);
    gcp::PushParams P{};
    P.st = c->st;
    P.ens = c->d_ens;
    P.dt = dt;
    P.t0 = c->t;
    P.collision_form = c->opt.collision_form;
    P.no_scatter = c->opt.no_scatter;
    P.no_rebirth = c->opt.no_rebirth;
    P.lambda_override = lambda_au > 0.0 ? lambda_au * kAU : 0.0;
    P.wind_u = c->opt.wind_u;
    P.seed = c->opt.seed;
    P.m = c->opt.mass;
    P.c2 = kC * kC;
    P.two_over_m = 2.0 / c->opt.mass;
    P.inv_c2 = 1.0 / (kC * kC);
    P.tally_on = c->tally_on ? 1 : 0;
    P.tally = c->tdev;
    P.gflags = c->d_flags;
    P.counters = c->d_counters;
    P.clock = clock_dev;
    const gcp::PhysHost ph = c->phys();

    int64_t done = 0;
    while (done < n_steps) {
        if (c->sort_every > 0 && c->steps_since_sort >= c->sort_every) {
            TRY(do_sort(c, s, owned, lc));
            P.st = c->st;
        }
        int64_t chunk = std::min<int64_t>(n_steps - done, c->steps_per_launch);
        if (c->sort_every > 0)
            chunk = std::min<int64_t>(chunk, std::max<int64_t>(1, c->sort_every - c->steps_since_sort));
        P.step0 = c->step + done;
        P.kbase = done;
        P.n_steps = (int32_t)chunk;
        Timed t;
        TRY(new_interval(c, 0, owned, &t));
        CUDA_TRY(cudaEventRecord(t.a, s));
        CUDA_TRY(gcp::launch_push(c->opt.precision, c->gh, ph, P, c->block, grid, s));
        CUDA_TRY(cudaEventRecord(t.b, s));
        lc->kernels += 1;
        lc->pushes += 1;
        done += chunk;
        c->steps_since_sort += chunk;
    }
    return GC_OK;
}

void add_counts(gc_ctx *c, const LaunchCounts &lc)
{
    c->kernel_launches += lc.kernels;
    c->push_launches += lc.pushes;
    c->sorts += lc.sorts;
}

void free_graph(GraphEntry *g)
{
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    for (const Timed &t : g->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    delete g;
}

void drop_graphs(gc_ctx *c)
{
    for (GraphEntry *g : c->graphs)
        free_graph(g);
    c->graphs.clear();
}

GraphKey graph_key(gc_ctx *c, double dt, int64_t n_steps, double lambda_au)
{
    GraphKey k{};
    k.dt = dt;
    k.lambda_au = lambda_au;
    k.n_steps = n_steps;
    k.n = c->n;
    k.cap = c->cap;
    k.steps_since_sort = c->steps_since_sort;
    k.n_ens = (int64_t)c->ens.size();
    k.block = c->block;
    k.grid_waves = c->grid_waves;
    k.steps_per_launch = c->steps_per_launch;
    k.sort_every = c->sort_every;
    k.tally_on = c->tally_on ? 1 : 0;
    k.st_x = c->st.x;
    k.alt_x = c->sortw.alt.x;
    k.tally = c->d_tally;
    k.grid = c->d_grid;
    k.ens = c->d_ens;
    return k;
}

// Capture the advance for this call pattern into a graph (once), then replay it. The
// graph resets the status words, copies the clock from a pinned host word, runs the sorts
// and push launches, and copies the status words back.
int advance_graph(gc_ctx *c, double dt, int64_t n_steps, double lambda_au, bool *anomaly)
{
    const GraphKey key = graph_key(c, dt, n_steps, lambda_au);
    GraphEntry *G = nullptr;
    for (GraphEntry *g : c->graphs)
        if (g->key == key) G = g;
    if (!G) {
        if (!c->cap_stream)
            CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        if (!c->d_clock) {
            CUDA_TRY(cudaMalloc(&c->d_clock, 2 * sizeof(double)));
            CUDA_TRY(cudaMallocHost(&c->h_clock, 2 * sizeof(double)));
        }
        if (c->sort_every > 0) {
            cudaError_t e = gcp::sort_reserve(c->sortw, c->st, c->gh);
            if (e != cudaSuccess)
                return fail(GC_ERR_NOMEM, "gc_advance: sort buffers: %s", cudaGetErrorString(e));
        }
        CUDA_TRY(gcp::preload_kernels());
        CUDA_TRY(gcp::sort_preload());
        push_grid(c); // occupancy query outside the capture
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        cudaGetLastError(); // start the capture with no stale error
        G = new GraphEntry();
        G->key = graph_key(c, dt, n_steps, lambda_au);
        const gcp::StateDev st0 = c->st, alt0 = c->sortw.alt;
        const int64_t ss0 = c->steps_since_sort;
        const bool order0 = c->in_id_order;
        cudaStream_t s = c->cap_stream;
        int rc = GC_OK;
        const char *what = "cudaStreamBeginCapture";
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            what = "status reset";
            e = cudaMemsetAsync(c->d_flags, 0, sizeof(uint32_t), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counters, 0, 2 * sizeof(unsigned long long), s);
            if (e == cudaSuccess) {
                what = "clock copy";
                e = cudaMemcpyAsync(c->d_clock, c->h_clock, 2 * sizeof(double), cudaMemcpyHostToDevice, s);
            }
            if (e == cudaSuccess) {
                what = "launches";
                rc = enqueue_advance(c, s, dt, n_steps, lambda_au, c->d_clock, &G->timed, &G->counts);
            }
            if (e == cudaSuccess && rc == GC_OK) {
                what = "status copy";
                e = cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(c->h_counters, c->d_counters, 2 * sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, s);
            }
            const cudaError_t e2 = cudaStreamEndCapture(s, &G->graph);
            if (e == cudaSuccess && rc == GC_OK && e2 != cudaSuccess) {
                e = e2;
                what = "cudaStreamEndCapture";
            }
        }
        G->st_after = c->st;
        G->alt_after = c->sortw.alt;
        G->steps_since_sort_after = c->steps_since_sort;
        c->st = st0; // capture ran no work: the state is where it was
        c->sortw.alt = alt0;
        c->steps_since_sort = ss0;
        c->in_id_order = order0;
        if (e == cudaSuccess && rc == GC_OK) {
            what = "cudaGraphInstantiate";
            e = cudaGraphInstantiate(&G->exec, G->graph, 0);
        }
        if (e != cudaSuccess || rc != GC_OK) {
            free_graph(G);
            cudaGetLastError();
            if (rc != GC_OK) return rc;
            return fail(GC_ERR_CUDA, "gc_advance: graph capture (%s): %s", what, cudaGetErrorString(e));
        }
        if (c->graphs.size() >= 4) {
            free_graph(c->graphs.front());
            c->graphs.erase(c->graphs.begin());
        }
        c->graphs.push_back(G);
    }
    c->h_clock[0] = c->t;
    c->h_clock[1] = (double)c->step;
    CUDA_TRY(cudaGraphLaunch(G->exec, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    harvest(c, G->timed);
    add_counts(c, G->counts);
    c->st = G->st_after;
    c->sortw.alt = G->alt_after;
    c->steps_since_sort = G->steps_since_sort_after;
    if (G->counts.sorts) c->in_id_order = false;
    const uint32_t f = *c->h_flags;
    c->flags_or |= f;
    c->collisions += c->h_counters[0];
    c->rebirths += c->h_counters[1];
    *anomaly = (f != 0);
    return GC_OK;
}

// ----------------------------------------------------------------------------------------
// Split-step push: for field sources evaluated on many points at once (the neural field),
// and for the grid evaluated through the same sample buffers (GC_FIELD_GRID_SAMPLED).
void free_split(gc_ctx *c)
{
    void *p[] = {c->d_req, c->d_reqR, c->d_S, c->d_SR, c->d_list, c->d_count};
    for (void *q : p)
        if (q) cudaFree(q);
    c->d_req = c->d_reqR = c->d_S = c->d_SR = nullptr;
    c->d_list = c->d_count = nullptr;
    c->split_cap = 0;
}

int ensure_split(gc_ctx *c)
{
    if (c->split_cap >= c->cap && c->d_count) return GC_OK;
    free_split(c);
    const size_t n = (size_t)std::max<int64_t>(c->cap, 1);
    CUDA_TRY(cudaMalloc(&c->d_req, n * 3 * sizeof(float)));
    CUDA_TRY(cudaMalloc(&c->d_reqR, n * 3 * sizeof(float)));
    CUDA_TRY(cudaMalloc(&c->d_S, n * gcp::kSampleStride * sizeof(float)));
    CUDA_TRY(cudaMalloc(&c->d_SR, n * gcp::kSampleStride * sizeof(float)));
    CUDA_TRY(cudaMalloc(&c->d_list, n * sizeof(int32_t)));
    CUDA_TRY(cudaMalloc(&c->d_count, sizeof(int32_t)));
    c->split_cap = (int64_t)n;
    return GC_OK;
}

// field samples at R (cap points; the count on the device when n_dev is set)
int field_samples(gc_ctx *c, const float *R, int64_t cap, const int32_t *n_dev, float *S, LaunchCounts *lc)
{
    Timed t;
    TRY(new_interval(c, 2, nullptr, &t));
    CUDA_TRY(cudaEventRecord(t.a, c->stream));
    if (c->field_source == GC_FIELD_SIREN)
        CUDA_TRY(gcn::neural_field_at(c->nn, R, cap, n_dev, S, gcp::kSampleStride, c->stream));
    else
        CUDA_TRY(gcp::launch_grid_samples(c->gh, R, cap, n_dev, S, c->stream));
    CUDA_TRY(cudaEventRecord(t.b, c->stream));
    lc->kernels += 1;
    return GC_OK;
}

gcp::SplitParams split_params(gc_ctx *c, double dt, double lambda_au)
{
    gcp::SplitParams Q{};
    gcp::PushParams &P = Q.P;
    P.st = c->st;
    P.ens = c->d_ens;
    P.dt = dt;
    P.t0 = c->t;
    P.collision_form = c->opt.collision_form;
    P.no_scatter = c->opt.no_scatter;
    P.no_rebirth = c->opt.no_rebirth;
    P.lambda_override = lambda_au > 0.0 ? lambda_au * kAU : 0.0;
    P.wind_u = c->opt.wind_u;
    P.seed = c->opt.seed;
    P.m = c->opt.mass;
    P.c2 = kC * kC;
    P.two_over_m = 2.0 / c->opt.mass;
    P.inv_c2 = 1.0 / (kC * kC);
    P.tally_on = c->tally_on ? 1 : 0;
    P.tally = c->tdev;
    P.gflags = c->d_flags;
    P.counters = c->d_counters;
    Q.req = c->d_req;
    Q.S = c->d_S;
    Q.reqR = c->d_reqR;
    Q.SR = c->d_SR;
    Q.list = c->d_list;
    Q.count = c->d_count;
    Q.g_in_sample = c->field_source == GC_FIELD_SIREN ? 0 : 1;
    Q.ideal = c->gh.ideal;
    return Q;
}

// n_steps steps of the split-step push: per step the predictor requests, two evaluations
// of all particles, and two evaluations of the restart list
int split_advance(gc_ctx *c, double dt, int64_t n_steps, double lambda_au, bool *anomaly)
{
    TRY(ensure_split(c));
    gcp::SplitParams Q = split_params(c, dt, lambda_au);
    const gcp::PhysHost ph = c->phys();
    cudaStream_t s = c->stream;
    LaunchCounts lc;
    const uint64_t coll0 = c->collisions, reb0 = c->rebirths;
    for (int64_t k = 0; k < n_steps; ++k) {
        Q.kk = (long long)(k + 1);
        Q.tally_now = (c->tally_on && ((c->step + k + 1) % c->tdev.cadence == 0)) ? 1 : 0;
        CUDA_TRY(cudaMemsetAsync(c->d_count, 0, sizeof(int32_t), s));
        CUDA_TRY(gcp::launch_split(gcp::SPLIT_PRED, ph, Q, s));
        TRY(field_samples(c, c->d_req, c->n, nullptr, c->d_S, &lc));
        CUDA_TRY(gcp::launch_split(gcp::SPLIT_CORR, ph, Q, s));
        TRY(field_samples(c, c->d_req, c->n, nullptr, c->d_S, &lc));
        CUDA_TRY(gcp::launch_split(gcp::SPLIT_POST, ph, Q, s));
        TRY(field_samples(c, c->d_reqR, c->n, c->d_count, c->d_SR, &lc));
        CUDA_TRY(gcp::launch_split(gcp::SPLIT_R2, ph, Q, s));
        TRY(field_samples(c, c->d_reqR, c->n, c->d_count, c->d_SR, &lc));
        CUDA_TRY(gcp::launch_split(gcp::SPLIT_R3, ph, Q, s));
        lc.kernels += 5;
    }
    add_counts(c, lc);
    TRY(collect_status(c, anomaly));
    c->field_evals += (uint64_t)(2 * c->n * n_steps) + 2 * ((c->collisions - coll0) + (c->rebirths - reb0));
    return GC_OK;
}

// redo the field-dependent part of an injection (slots [slot0, slot0 + n_new)) with the
// selected split-step source: mu_B from |B| at the site and the start-up history
int split_inject_fix(gc_ctx *c, int64_t slot0, int64_t n_new)
{
    TRY(ensure_split(c));
    gcp::SplitParams Q = split_params(c, c->opt.dt_init, 0.0);
    Q.slot0 = slot0;
    Q.n_new = n_new;
    const gcp::PhysHost ph = c->phys();
    cudaStream_t s = c->stream;
    LaunchCounts lc;
    const int32_t cnt = (int32_t)n_new;
    CUDA_TRY(gcp::launch_split(gcp::SPLIT_INJ_REQ, ph, Q, s));
    TRY(field_samples(c, c->d_req, n_new, nullptr, c->d_S, &lc));
    CUDA_TRY(gcp::launch_split(gcp::SPLIT_INJ_FIX, ph, Q, s));
    CUDA_TRY(cudaMemcpyAsync(c->d_count, &cnt, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    TRY(field_samples(c, c->d_reqR, n_new, c->d_count, c->d_SR, &lc));
    CUDA_TRY(gcp::launch_split(gcp::SPLIT_R3, ph, Q, s));
    CUDA_TRY(cudaStreamSynchronize(s)); // the host word cnt is read by the copy above
    lc.kernels += 3;
    add_counts(c, lc);
    c->field_evals += (uint64_t)(2 * n_new);
    return GC_OK;
}

// copy (and convert to the context's precision) node data into a new device array
int upload_nodes(gc_ctx *c, const gc_grid_desc *g, const void *data, int data_on_device, void **dst)
{
    const size_t nval = (size_t)g->n_r * g->n_th * g->n_ph * 8;
    const bool want64 = (c->opt.precision == GC_PREC_FP64);
    const size_t esz = want64 ? sizeof(double) : sizeof(float);
    const size_t in_esz = (g->dtype == GC_DTYPE_F64) ? sizeof(double) : sizeof(float);
    CUDA_TRY(cudaMalloc(dst, nval * esz));
    const bool same = (want64 == (g->dtype == GC_DTYPE_F64));
    const cudaMemcpyKind kind = data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (same) {
        CUDA_TRY(cudaMemcpyAsync(*dst, data, nval * esz, kind, c->stream));
    } else {
        void *tmp = nullptr;
        CUDA_TRY(cudaMalloc(&tmp, nval * in_esz));
        cudaError_t e = cudaMemcpyAsync(tmp, data, nval * in_esz, kind, c->stream);
        if (e == cudaSuccess) {
            if (want64)
                convert_nodes<<<1024, 256, 0, c->stream>>>((const float *)tmp, (double *)*dst, nval);
            else
                convert_nodes<<<1024, 256, 0, c->stream>>>((const double *)tmp, (float *)*dst, nval);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
        if (e != cudaSuccess)
            return fail(GC_ERR_CUDA, "node upload: %s", cudaGetErrorString(e));
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GC_OK;
}

void free_tally(gc_ctx *c)
{
    if (c->d_tally) cudaFree(c->d_tally);
    c->d_tally = nullptr;
    c->tally_on = false;
    c->tally_bytes = 0;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

} // namespace

extern "C" {

int gc_version(void) { return 100; }

const char *gc_last_error(void) { return g_err.c_str(); }

int gc_create(gc_ctx **out, const gc_options *opt)
{
    if (!out || !opt)
        return fail(GC_ERR_INVALID, "gc_create: null argument");
    *out = nullptr;
    if (opt->precision != GC_PREC_FP64 && opt->precision != GC_PREC_FP32_MIXED)
        return fail(GC_ERR_INVALID, "gc_create: unknown precision %d", opt->precision);
    if (opt->collision_form < 0 || opt->collision_form > 1 || opt->drift_mask < 0 || opt->drift_mask > 1)
        return fail(GC_ERR_INVALID, "gc_create: bad collision_form/drift_mask");
    if (!(opt->wind_u >= 0.0) || !(opt->wind_u < 0.01 * kC))
        return fail(GC_ERR_INVALID, "gc_create: wind_u must be >= 0 and far below c");
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (opt->device < 0 || opt->device >= ndev)
        return fail(GC_ERR_INVALID, "gc_create: device %d not present (%d devices)", opt->device, ndev);
    gc_ctx *c = new gc_ctx();
    c->opt = *opt;
    if (c->opt.charge == 0.0) c->opt.charge = kQe;
    if (c->opt.mass <= 0.0) c->opt.mass = kMe;
    if (!(c->opt.dt_init > 0.0)) c->opt.dt_init = 0.5;
    c->device = opt->device;
    c->stream = static_cast<cudaStream_t>(opt->stream);
    c->next_id = opt->id_base;
    c->id_lo = opt->id_base;
    int rc = set_device(c);
    if (rc != GC_OK) { delete c; return rc; }
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (cudaMalloc(&c->d_flags, sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&c->d_counters, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&c->h_flags, sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&c->h_counters, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        gc_destroy(c);
        return fail(GC_ERR_NOMEM, "gc_create: status allocation failed");
    }
    cudaMemsetAsync(c->d_flags, 0, sizeof(uint32_t), c->stream);
    cudaMemsetAsync(c->d_counters, 0, 2 * sizeof(unsigned long long), c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        gc_destroy(c);
        return fail(GC_ERR_CUDA, "gc_create: stream not usable");
    }
    *out = c;
    return GC_OK;
}

void gc_destroy(gc_ctx *c)
{
    if (!c)
        return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->d_grid) cudaFree(c->d_grid);
    if (c->d_grid1) cudaFree(c->d_grid1);
    free_state(c->st);
    if (c->d_ens) cudaFree(c->d_ens);
    free_tally(c);
    if (c->d_flags) cudaFree(c->d_flags);
    if (c->d_counters) cudaFree(c->d_counters);
    if (c->h_flags) cudaFreeHost(c->h_flags);
    if (c->h_counters) cudaFreeHost(c->h_counters);
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->d_clock) cudaFree(c->d_clock);
    if (c->h_clock) cudaFreeHost(c->h_clock);
    gcp::sort_free(c->sortw);
    gcn::neural_free(c->nn);
    free_split(c);
    for (cudaEvent_t e : c->ev_pool)
        cudaEventDestroy(e);
    delete c;
}

int gc_field_load(gc_ctx *c, const gc_grid_desc *g, const void *data, int data_on_device)
{
    if (!c || !g || !data)
        return fail(GC_ERR_INVALID, "gc_field_load: null argument");
    if (g->n_r < 2 || g->n_th < 2 || g->n_ph < 2)
        return fail(GC_ERR_INVALID, "gc_field_load: need n_r, n_th, n_ph >= 2");
    if (g->dtype != GC_DTYPE_F64 && g->dtype != GC_DTYPE_F32)
        return fail(GC_ERR_INVALID, "gc_field_load: unknown dtype %d", g->dtype);
    if (g->ideal < 0 || g->ideal > 2)
        return fail(GC_ERR_INVALID, "gc_field_load: ideal must be 0, 1 or 2");
    if (!(g->r_min_au > 0.0) || !(g->r_max_au > g->r_min_au))
        return fail(GC_ERR_INVALID, "gc_field_load: need 0 < r_min < r_max");
    const size_t nodes = (size_t)g->n_r * g->n_th * g->n_ph;
    const size_t nval = nodes * 8;
    if (nval >= (size_t)1 << 32)
        return fail(GC_ERR_INVALID, "gc_field_load: %zu node values exceed the 2^32 index range", nval);
    TRY(set_device(c));
    const bool want64 = (c->opt.precision == GC_PREC_FP64);
    drop_graphs(c);
    if (c->d_grid) {
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        cudaFree(c->d_grid);
        c->d_grid = nullptr;
        c->has_field = false;
    }
    TRY(upload_nodes(c, g, data, data_on_device, &c->d_grid));
    if (c->d_grid1) {
        cudaFree(c->d_grid1);
        c->d_grid1 = nullptr;
    }
    c->gh.nodes1 = nullptr;
    for (int &nb : c->blocks_per_sm) nb = 0;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->grid = *g;
    c->gh.nodes = c->d_grid;
    c->gh.n_r = g->n_r;
    c->gh.n_th = g->n_th;
    c->gh.n_ph = g->n_ph;
    c->gh.ideal = g->ideal;
    c->gh.is_f64 = want64 ? 1 : 0;
    c->gh.r_min = g->r_min_au * kAU;
    c->gh.dr = (g->r_max_au * kAU - g->r_min_au * kAU) / (double)(g->n_r - 1);
    c->gh.dth = kPi / (double)(g->n_th - 1);
    c->gh.dph = 2.0 * kPi / (double)g->n_ph;
    c->has_field = true;
    return GC_OK;
}

int gc_field_load_next(gc_ctx *c, const void *data, int data_on_device, double t0_s, double t1_s)
{
    if (!c || !data)
        return fail(GC_ERR_INVALID, "gc_field_load_next: null argument");
    if (!c->has_field)
        return fail(GC_ERR_STATE, "gc_field_load_next: load the first snapshot with gc_field_load first");
    if (!(t1_s > t0_s) || !std::isfinite(t0_s) || !std::isfinite(t1_s))
        return fail(GC_ERR_INVALID, "gc_field_load_next: need finite t0 < t1");
    if (c->field_source != GC_FIELD_GRID)
        return fail(GC_ERR_UNSUPPORTED, "gc_field_load_next: time-dependent fields run with GC_FIELD_GRID");
    TRY(set_device(c));
    drop_graphs(c);
    if (c->d_grid1) {
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        cudaFree(c->d_grid1);
        c->d_grid1 = nullptr;
        c->gh.nodes1 = nullptr;
    }
    TRY(upload_nodes(c, &c->grid, data, data_on_device, &c->d_grid1));
    c->gh.nodes1 = c->d_grid1;
    c->gh.t_snap0 = t0_s;
    c->gh.t_snap1 = t1_s;
    for (int &nb : c->blocks_per_sm) nb = 0;
    return GC_OK;
}

int gc_particles_inject(gc_ctx *c, const gc_ensemble_desc *e, int n_ens)
{
    if (!c || (!e && n_ens > 0) || n_ens < 0)
        return fail(GC_ERR_INVALID, "gc_particles_inject: bad arguments");
    if (!c->has_field)
        return fail(GC_ERR_STATE, "gc_particles_inject: no field loaded");
    if (c->ens.size() + (size_t)n_ens > 65535)
        return fail(GC_ERR_INVALID, "gc_particles_inject: more than 65535 ensembles");
    int64_t total = 0;
    for (int k = 0; k < n_ens; ++k) {
        const gc_ensemble_desc &d = e[k];
        if (d.count < 0 || !(d.r0_au > 0.0) || !(d.lambda_au > 0.0) || !(d.r_out_au > 0.0) ||
            d.energy_law < 0 || d.energy_law > 1 || d.mu_law < 0 || d.mu_law > 1 ||
            d.scatter_law < 0 || d.scatter_law > 1)
            return fail(GC_ERR_INVALID, "gc_particles_inject: bad descriptor %d", k);
        if (d.energy_law == 0 && !(d.E0_keV > 0.0))
            return fail(GC_ERR_INVALID, "gc_particles_inject: E0 must be > 0 (descriptor %d)", k);
        if (d.energy_law == 1 && (!(d.E_lo_keV > 0.0) || !(d.E_hi_keV > d.E_lo_keV) || d.E_index == 1.0))
            return fail(GC_ERR_INVALID, "gc_particles_inject: bad spectrum (descriptor %d)", k);
        total += d.count;
    }
    if ((uint64_t)c->next_id + (uint64_t)total > 0xFFFFFFFFull)
        return fail(GC_ERR_INVALID, "gc_particles_inject: particle ids exceed 32 bits");
    TRY(set_device(c));
    TRY(reserve(c, c->n + total));
    const int ens_base = (int)c->ens.size();
    int64_t first = c->n;
    for (int k = 0; k < n_ens; ++k) {
        const gc_ensemble_desc &d = e[k];
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
        E.first = first;
        E.count = d.count;
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
        c->ens.push_back(E);
        first += d.count;
    }
    TRY(upload_ensembles(c));
    if (total > 0) {
        gcp::InjectParams P{};
        P.st = c->st;
        P.ens = c->d_ens + ens_base;
        P.n_ens = n_ens;
        P.ens_base = ens_base;
        P.slot0 = c->n;
        P.count = total;
        P.id0 = c->next_id;
        P.seed = c->opt.seed;
        P.t = c->t;
        P.dt_init = c->opt.dt_init;
        P.m = c->opt.mass;
        P.c2 = kC * kC;
        P.gflags = c->d_flags;
        CUDA_TRY(gcp::launch_inject(c->opt.precision, c->gh, c->phys(), P, c->stream));
        c->kernel_launches += 1;
    }
    if (c->n == 0) {
        c->id_lo = c->next_id;
        c->ids_dense = true;
        c->in_id_order = true;
    } else if (c->ids_dense && c->next_id != c->id_lo + (uint32_t)c->n) {
        c->ids_dense = false; // appended ids do not continue the existing range
    }
    const int64_t slot0 = c->n;
    c->n += total;
    c->st.n = c->n;
    c->next_id += (uint32_t)total;
    if (total > 0 && c->field_source != GC_FIELD_GRID)
        TRY(split_inject_fix(c, slot0, total));
    bool anomaly = false;
    TRY(collect_status(c, &anomaly));
    if (anomaly)
        return fail(GC_ERR_DEVICE_ANOMALY, "gc_particles_inject: particles flagged (0x%x)", c->flags_or);
    return GC_OK;
}

int gc_set_launch(gc_ctx *c, int block, int steps_per_launch, int sort_every, int grid_waves)
{
    if (!c)
        return fail(GC_ERR_INVALID, "gc_set_launch: null context");
    if (block != 0 && (block < 32 || block > 128 || block % 32 != 0))
        return fail(GC_ERR_INVALID, "gc_set_launch: block must be a multiple of 32 in [32, 128]");
    if (steps_per_launch < 0 || sort_every < 0 || grid_waves < 0)
        return fail(GC_ERR_INVALID, "gc_set_launch: negative argument");
    if (block) c->block = block;
    if (steps_per_launch) c->steps_per_launch = steps_per_launch;
    c->sort_every = sort_every;
    c->grid_waves = grid_waves;
    return GC_OK;
}

int gc_sort(gc_ctx *c)
{
    if (!c)
        return fail(GC_ERR_INVALID, "gc_sort: null context");
    if (!c->has_field)
        return fail(GC_ERR_STATE, "gc_sort: no field loaded");
    TRY(set_device(c));
    if (c->n < 2)
        return GC_OK;
    LaunchCounts lc;
    TRY(do_sort(c, c->stream, nullptr, &lc));
    add_counts(c, lc);
    bool anomaly = false;
    return collect_status(c, &anomaly);
}

int gc_advance(gc_ctx *c, double dt, int64_t n_steps, double lambda_au)
{
    if (!c)
        return fail(GC_ERR_INVALID, "gc_advance: null context");
    if (!(dt > 0.0) || !std::isfinite(dt) || n_steps < 0)
        return fail(GC_ERR_INVALID, "gc_advance: need dt > 0 and n_steps >= 0");
    if (!c->has_field)
        return fail(GC_ERR_STATE, "gc_advance: no field loaded");
    TRY(set_device(c));
    if (c->n == 0 || n_steps == 0) {
        c->t += (double)n_steps * dt;
        c->step += n_steps;
        return GC_OK;
    }
    bool anomaly = false;
    if (c->field_source != GC_FIELD_GRID) {
        TRY(split_advance(c, dt, n_steps, lambda_au, &anomaly));
    } else if (c->use_graph) {
        TRY(advance_graph(c, dt, n_steps, lambda_au, &anomaly));
    } else {
        LaunchCounts lc;
        TRY(enqueue_advance(c, c->stream, dt, n_steps, lambda_au, nullptr, nullptr, &lc));
        add_counts(c, lc);
        TRY(collect_status(c, &anomaly));
    }
    c->t += (double)n_steps * dt;
    c->step += n_steps;
    c->particle_steps += (uint64_t)c->n * (uint64_t)n_steps;
    if (anomaly)
        return fail(GC_ERR_DEVICE_ANOMALY, "gc_advance: particles flagged (0x%x)", c->flags_or);
    return GC_OK;
}

int gc_set_graph(gc_ctx *c, int enable)
{
    if (!c)
        return fail(GC_ERR_INVALID, "gc_set_graph: null context");
    TRY(set_device(c));
    c->use_graph = enable != 0;
    if (!c->use_graph) {
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        drop_graphs(c);
    }
    return GC_OK;
}

namespace {

// D2D copy of n particles between two state buffers of equal capacity
int copy_state(const gcp::StateDev &dst, const gcp::StateDev &src, int64_t n, int64_t cap, cudaStream_t s)
{
    double *const dd[] = {dst.x, dst.y, dst.z, dst.u, dst.mub, dst.vpar, dst.s_rem, dst.h_prev,
                          dst.t_birth, dst.u_inj, dst.mub_inj};
    const double *const sd[] = {src.x, src.y, src.z, src.u, src.mub, src.vpar, src.s_rem, src.h_prev,
                                src.t_birth, src.u_inj, src.mub_inj};
    for (int k = 0; k < 11; ++k)
        CUDA_TRY(cudaMemcpyAsync(dd[k], sd[k], (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(dst.F0, src.F0, (size_t)cap * 32, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(dst.F1, src.F1, (size_t)cap * 32, cudaMemcpyDeviceToDevice, s));
    uint32_t *const du[] = {dst.id, dst.ens, dst.event, dst.ncoll, dst.flags};
    const uint32_t *const su[] = {src.id, src.ens, src.event, src.ncoll, src.flags};
    for (int k = 0; k < kU32Fields; ++k)
        CUDA_TRY(cudaMemcpyAsync(du[k], su[k], (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    return GC_OK;
}

} // namespace

int gc_autotune(gc_ctx *c, double dt, int64_t trial_steps, gc_launch_choice *best)
{
    if (!c || !(dt > 0.0) || trial_steps < 1)
        return fail(GC_ERR_INVALID, "gc_autotune: need a context, dt > 0 and trial_steps >= 1");
    if (!c->has_field || c->n == 0)
        return fail(GC_ERR_STATE, "gc_autotune: needs a field and particles");
    TRY(set_device(c));
    // snapshot of the state; every trial starts from it and the state is restored after
    gcp::StateDev bk{};
    {
        cudaError_t e = gcp::alloc_state(bk, c->cap);
        if (e != cudaSuccess) {
            gcp::free_state_arrays(bk);
            return fail(GC_ERR_NOMEM, "gc_autotune: snapshot: %s", cudaGetErrorString(e));
        }
    }
    int rc = copy_state(bk, c->st, c->n, c->cap, c->stream);
    const double t_sv = c->t;
    const int64_t step_sv = c->step, ss_sv = c->steps_since_sort;
    const uint64_t coll_sv = c->collisions, reb_sv = c->rebirths, ps_sv = c->particle_steps;
    const uint32_t flags_sv = c->flags_or;
    const bool tally_sv = c->tally_on, graph_sv = c->use_graph, order_sv = c->in_id_order;
    const int blk_sv = c->block, waves_sv = c->grid_waves, spl_sv = c->steps_per_launch, se_sv = c->sort_every;
    c->tally_on = false;
    c->use_graph = false;
    gc_launch_choice b{};
    b.particle_steps_per_s = -1.0;
    int trials = 0;
    const int blocks[] = {64, 128};
    const int waves[] = {1, 2, 4, 0};
    const int sorts[] = {0, 250, 1000};
    for (int blk : blocks) {
        for (int wv : waves) {
            for (int se : sorts) {
                if (rc != GC_OK) break;
                c->block = blk;
                c->grid_waves = wv;
                c->sort_every = se;
                c->steps_per_launch = (int)std::min<int64_t>(trial_steps, 2000);
                c->steps_since_sort = se; // a trial with sorting starts with one sort
                rc = copy_state(c->st, bk, c->n, c->cap, c->stream);
                if (rc != GC_OK) break;
                const double push0 = c->push_ms, sort0 = c->sort_ms;
                LaunchCounts lc;
                rc = enqueue_advance(c, c->stream, dt, trial_steps, 0.0, nullptr, nullptr, &lc);
                if (rc != GC_OK) break;
                add_counts(c, lc);
                bool an = false;
                rc = collect_status(c, &an);
                if (rc != GC_OK) break;
                const double push_s = (c->push_ms - push0) * 1e-3;
                const double sort_s = (c->sort_ms - sort0) * 1e-3;
                // a sort serves sort_every steps: charge its share to this trial
                const double per_step = push_s / trial_steps + (se > 0 ? sort_s / se : 0.0);
                const double rate = (double)c->n / per_step;
                ++trials;
                if (rate > b.particle_steps_per_s) {
                    b.block = blk;
                    b.grid_waves = wv;
                    b.sort_every = se;
                    b.steps_per_launch = 2000;
                    b.particle_steps_per_s = rate;
                }
            }
        }
    }
    if (rc == GC_OK)
        rc = copy_state(c->st, bk, c->n, c->cap, c->stream);
    cudaStreamSynchronize(c->stream);
    gcp::free_state_arrays(bk);
    c->t = t_sv;
    c->step = step_sv;
    c->steps_since_sort = ss_sv;
    c->collisions = coll_sv;
    c->rebirths = reb_sv;
    c->particle_steps = ps_sv;
    c->flags_or = flags_sv;
    c->tally_on = tally_sv;
    c->use_graph = graph_sv;
    c->in_id_order = order_sv;
    if (rc != GC_OK) {
        c->block = blk_sv;
        c->grid_waves = waves_sv;
        c->steps_per_launch = spl_sv;
        c->sort_every = se_sv;
        return rc;
    }
    c->block = b.block;
    c->grid_waves = b.grid_waves;
    c->steps_per_launch = b.steps_per_launch;
    c->sort_every = b.sort_every;
    b.trials = trials;
    if (best) *best = b;
    return GC_OK;
}

int gc_tally(gc_ctx *c, const gc_tally_desc *arm, gc_tally_out *out)
{
    if (!c)
        return fail(GC_ERR_INVALID, "gc_tally: null context");
    TRY(set_device(c));
    if (out) {
        if (!c->tally_on)
            return fail(GC_ERR_STATE, "gc_tally: tallies are not armed");
        const gc_tally_desc &t = c->tdesc;
        const size_t ne = (size_t)c->tdev.n_ens;
        struct Item { void *dst; size_t off, bytes; } items[] = {
            {out->h_mer, 0, ne * t.n_mu * t.n_E * t.n_r * 4},
            {out->h_age, c->off_age, ne * t.n_age * t.n_E * 4},
            {out->h_pad, c->off_pad, ne * t.n_mu * 4},
            {out->m_cnt, c->off_cnt, ne * t.n_r * 8},
            {out->m_sin2, c->off_sin2, ne * t.n_r * 8},
            {out->n_seen, c->off_seen, 2 * 8},
        };
        for (const Item &it : items) {
            if (!it.dst)
                continue;
            CUDA_TRY(cudaMemcpyAsync(it.dst, (char *)c->d_tally + it.off, it.bytes, cudaMemcpyDeviceToHost, c->stream));
        }
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    if (arm) {
        const gc_tally_desc &t = *arm;
        if (t.cadence < 1 || t.n_mu < 1 || t.n_E < 1 || t.n_r < 1 || t.n_age < 1 ||
            !(t.E_lo_keV > 0.0) || !(t.E_hi_keV > t.E_lo_keV) || !(t.r_hi_au > t.r_lo_au) ||
            !(t.age_max_s > 0.0))
            return fail(GC_ERR_INVALID, "gc_tally: bad descriptor");
        const size_t ne = std::max<size_t>(1, c->ens.size());
        const size_t b_mer = ne * t.n_mu * t.n_E * t.n_r * 4;
        const size_t b_age = ne * t.n_age * t.n_E * 4;
        const size_t b_pad = ne * t.n_mu * 4;
        const size_t b_r = ne * t.n_r * 8;
        if ((double)ne * t.n_mu * t.n_E * t.n_r >= 2147483647.0 || (double)ne * t.n_age * t.n_E >= 2147483647.0)
            return fail(GC_ERR_INVALID, "gc_tally: histogram larger than 2^31 bins");
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        drop_graphs(c);
        free_tally(c);
        c->off_age = align_up(b_mer, 256);
        c->off_pad = align_up(c->off_age + b_age, 256);
        c->off_cnt = align_up(c->off_pad + b_pad, 256);
        c->off_sin2 = align_up(c->off_cnt + b_r, 256);
        c->off_seen = align_up(c->off_sin2 + b_r, 256);
        c->tally_bytes = c->off_seen + 16;
        CUDA_TRY(cudaMalloc(&c->d_tally, c->tally_bytes));
        CUDA_TRY(cudaMemsetAsync(c->d_tally, 0, c->tally_bytes, c->stream));
        char *base = (char *)c->d_tally;
        gcp::TallyDev &d = c->tdev;
        d.cadence = t.cadence;
        d.n_mu = t.n_mu;
        d.n_E = t.n_E;
        d.n_r = t.n_r;
        d.n_age = t.n_age;
        d.n_ens = (int)ne;
        d.t_start = t.t_start_s;
        d.E_lo = t.E_lo_keV * kKeV;
        d.log_E_ratio = log((t.E_hi_keV * kKeV) / (t.E_lo_keV * kKeV));
        d.r_lo = t.r_lo_au * kAU;
        d.r_span = t.r_hi_au * kAU - t.r_lo_au * kAU;
        d.age_max = t.age_max_s;
        d.rwin_lo = t.rwin_lo_au * kAU;
        d.rwin_hi = t.rwin_hi_au * kAU;
        d.age_young = t.age_young_s;
        d.inv_E_lo_f = (float)(1.0 / d.E_lo);
        d.E_scale_f = (float)(t.n_E / d.log_E_ratio);
        d.r_lo_f = (float)d.r_lo;
        d.r_scale_f = (float)(t.n_r / d.r_span);
        d.age_scale_f = (float)(t.n_age / d.age_max);
        d.rwin_lo_f = (float)d.rwin_lo;
        d.rwin_hi_f = (float)d.rwin_hi;
        d.age_young_f = (float)d.age_young;
        d.h_mer = (uint32_t *)base;
        d.h_age = (uint32_t *)(base + c->off_age);
        d.h_pad = (uint32_t *)(base + c->off_pad);
        d.m_cnt = (unsigned long long *)(base + c->off_cnt);
        d.m_sin2 = (unsigned long long *)(base + c->off_sin2);
        d.n_seen = (unsigned long long *)(base + c->off_seen);
        c->tdesc = t;
        c->tally_on = true;
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    return GC_OK;
}

int gc_particles_get(gc_ctx *c, gc_particle_soa *o)
{
    if (!c || !o)
        return fail(GC_ERR_INVALID, "gc_particles_get: null argument");
    if (o->n != c->n)
        return fail(GC_ERR_INVALID, "gc_particles_get: buffer holds %lld particles, context %lld",
                    (long long)o->n, (long long)c->n);
    TRY(set_device(c));
    const int64_t n = c->n;
    if (n == 0)
        return GC_OK;
    // Source in ascending id order: the state itself, or its un-permuted copy in the
    // sort's alternate arrays; only an irregular id set falls back to a host reorder.
    const gcp::StateDev *src = &c->st;
    std::vector<int64_t> order;
    if (!c->in_id_order) {
        if (c->ids_dense) {
            cudaError_t e = gcp::unpermute_to_alt(c->sortw, c->st, c->id_lo, c->stream);
            if (e != cudaSuccess)
                return fail(GC_ERR_CUDA, "gc_particles_get: %s", cudaGetErrorString(e));
            c->kernel_launches += gcp::kUnpermuteKernels;
            src = &c->sortw.alt;
        } else {
            std::vector<uint32_t> id(n);
            CUDA_TRY(cudaMemcpyAsync(id.data(), c->st.id, n * 4, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            order.resize(n);
            std::iota(order.begin(), order.end(), 0);
            std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return id[a] < id[b]; });
        }
    }
    const int64_t scap = c->cap;
    std::vector<double> buf(order.empty() ? 0 : n);
    std::vector<uint32_t> ubuf(order.empty() ? 0 : n);
    auto getd = [&](const double *from, double *dst) -> int {
        if (!dst) return GC_OK;
        if (order.empty()) {
            CUDA_TRY(cudaMemcpyAsync(dst, from, n * 8, cudaMemcpyDeviceToHost, c->stream));
            return GC_OK;
        }
        CUDA_TRY(cudaMemcpyAsync(buf.data(), from, n * 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        for (int64_t k = 0; k < n; ++k) dst[k] = buf[order[k]];
        return GC_OK;
    };
    auto getu = [&](const uint32_t *from, uint32_t *dst) -> int {
        if (!dst) return GC_OK;
        if (order.empty()) {
            CUDA_TRY(cudaMemcpyAsync(dst, from, n * 4, cudaMemcpyDeviceToHost, c->stream));
            return GC_OK;
        }
        CUDA_TRY(cudaMemcpyAsync(ubuf.data(), from, n * 4, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        for (int64_t k = 0; k < n; ++k) dst[k] = ubuf[order[k]];
        return GC_OK;
    };
    TRY(getd(src->x, o->x)); TRY(getd(src->y, o->y)); TRY(getd(src->z, o->z));
    TRY(getd(src->u, o->u)); TRY(getd(src->mub, o->mub)); TRY(getd(src->vpar, o->vpar));
    TRY(getd(src->s_rem, o->s_rem)); TRY(getd(src->h_prev, o->h_prev));
    TRY(getd(src->t_birth, o->t_birth)); TRY(getd(src->u_inj, o->u_inj));
    TRY(getd(src->mub_inj, o->mub_inj));
    for (int r = 0; r < 4; ++r) {
        TRY(getd(src->F0 + r * scap, o->F0 ? o->F0 + r * n : nullptr));
        TRY(getd(src->F1 + r * scap, o->F1 ? o->F1 + r * n : nullptr));
    }
    TRY(getu(src->id, o->id)); TRY(getu(src->ens, o->ens)); TRY(getu(src->event, o->event));
    TRY(getu(src->ncoll, o->ncoll)); TRY(getu(src->flags, o->flags));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GC_OK;
}

int gc_particles_set(gc_ctx *c, const gc_particle_soa *in)
{
    if (!c || !in || in->n < 0)
        return fail(GC_ERR_INVALID, "gc_particles_set: bad argument");
    const double *const dsrc[] = {in->x, in->y, in->z, in->u, in->mub, in->vpar, in->s_rem,
                                  in->h_prev, in->t_birth, in->u_inj, in->mub_inj, in->F0, in->F1};
    const uint32_t *const usrc[] = {in->id, in->ens, in->event, in->ncoll, in->flags};
    for (const double *p : dsrc)
        if (!p && in->n) return fail(GC_ERR_INVALID, "gc_particles_set: every array is required");
    for (const uint32_t *p : usrc)
        if (!p && in->n) return fail(GC_ERR_INVALID, "gc_particles_set: every array is required");
    const int64_t n = in->n;
    bool ascending = true;
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (in->ens[k] >= c->ens.size())
            return fail(GC_ERR_INVALID, "gc_particles_set: particle %lld has unknown ensemble %u",
                        (long long)k, in->ens[k]);
        if (k && in->id[k] <= in->id[k - 1]) ascending = false;
        lo = std::min(lo, in->id[k]);
        hi = std::max(hi, in->id[k]);
    }
    bool dense = (n == 0) || ((int64_t)hi - (int64_t)lo + 1 == n);
    if (dense && !ascending) {
        std::vector<char> seen(n, 0);
        for (int64_t k = 0; k < n && dense; ++k) {
            char &f = seen[in->id[k] - lo];
            if (f) dense = false;
            f = 1;
        }
    }
    TRY(set_device(c));
    c->n = 0;
    c->st.n = 0;
    TRY(reserve(c, n));
    double *const ddst[] = {c->st.x, c->st.y, c->st.z, c->st.u, c->st.mub, c->st.vpar, c->st.s_rem,
                            c->st.h_prev, c->st.t_birth, c->st.u_inj, c->st.mub_inj};
    if (n) {
        for (int k = 0; k < 11; ++k)
            CUDA_TRY(cudaMemcpyAsync(ddst[k], dsrc[k], n * 8, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaMemcpy2DAsync(c->st.F0, c->cap * 8, in->F0, n * 8, n * 8, 4, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaMemcpy2DAsync(c->st.F1, c->cap * 8, in->F1, n * 8, n * 8, 4, cudaMemcpyHostToDevice, c->stream));
        uint32_t *const udst[] = {c->st.id, c->st.ens, c->st.event, c->st.ncoll, c->st.flags};
        for (int k = 0; k < kU32Fields; ++k)
            CUDA_TRY(cudaMemcpyAsync(udst[k], usrc[k], n * 4, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    c->n = n;
    c->st.n = n;
    // a state from the host is in id order, not in cell order: sort before the next push
    if (c->sort_every > 0)
        c->steps_since_sort = c->sort_every;
    c->in_id_order = ascending;
    c->ids_dense = dense;
    c->id_lo = n ? lo : c->next_id;
    if (n && hi >= c->next_id)
        c->next_id = hi + 1;
    return GC_OK;
}

int gc_stats(gc_ctx *c, gc_stats_out *o)
{
    if (!c || !o)
        return fail(GC_ERR_INVALID, "gc_stats: null argument");
    o->n_particles = c->n;
    o->step = c->step;
    o->t = c->t;
    o->particle_steps = c->particle_steps;
    o->collisions = c->collisions;
    o->rebirths = c->rebirths;
    o->flags_or = c->flags_or;
    o->pad0 = 0;
    o->kernel_launches = c->kernel_launches;
    o->push_launches = c->push_launches;
    o->push_ms = c->push_ms;
    o->sorts = c->sorts;
    o->sort_ms = c->sort_ms;
    o->field_evals = c->field_evals;
    o->field_ms = c->field_ms;
    return GC_OK;
}

int gc_set_clock(gc_ctx *c, double t, int64_t step)
{
    if (!c || !std::isfinite(t) || step < 0)
        return fail(GC_ERR_INVALID, "gc_set_clock: bad argument");
    c->t = t;
    c->step = step;
    return GC_OK;
}


// ----------------------------------------------------------------------------- neural field
static int nn_ready(gc_ctx *c, const char *who)
{
    if (!c) return fail(GC_ERR_INVALID, "%s: null context", who);
    if (!c->nn.ready) return fail(GC_ERR_STATE, "%s: no network (call gc_siren_set first)", who);
    return GC_OK;
}

static gcn::GridRef grid_ref(const gc_ctx *c)
{
    gcn::GridRef g;
    g.nodes = c->d_grid;
    g.is_f64 = c->gh.is_f64;
    g.n_r = c->gh.n_r;
    g.n_th = c->gh.n_th;
    g.n_ph = c->gh.n_ph;
    g.r_min = c->gh.r_min;
    g.dr = c->gh.dr;
    return g;
}

int gc_siren_set(gc_ctx *c, const gc_siren_desc *d, const float *params, int params_on_device)
{
    if (!c || !d || !params) return fail(GC_ERR_INVALID, "gc_siren_set: null argument");
    if (!(d->omega0 > 0.0) || !(d->r_max_au > 0.0) || !(d->B_scale > 0.0) || !(d->E_scale > 0.0))
        return fail(GC_ERR_INVALID, "gc_siren_set: omega0, r_max_au, B_scale and E_scale must be > 0");
    TRY(set_device(c));
    drop_graphs(c);
    cudaError_t e = gcn::neural_set(c->nn, params, params_on_device != 0, d->omega0, d->r_max_au * kAU, d->B_scale,
                                    d->E_scale, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? GC_ERR_NOMEM : GC_ERR_CUDA, "gc_siren_set: %s",
                    cudaGetErrorString(e));
    return GC_OK;
}

int gc_siren_get(gc_ctx *c, float *params_host)
{
    TRY(nn_ready(c, "gc_siren_get"));
    if (!params_host) return fail(GC_ERR_INVALID, "gc_siren_get: null output");
    TRY(set_device(c));
    CUDA_TRY(cudaMemcpyAsync(params_host, c->nn.P, (size_t)GC_SIREN_NPARAMS * sizeof(float), cudaMemcpyDeviceToHost,
                             c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GC_OK;
}

static int nn_check_tc(gc_ctx *c, const char *who)
{
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    int te = gcs::read_error(c->stream);
    if (!te) te = gcn::neural_read_error(c->nn, c->stream);
    if (te) return fail(GC_ERR_DEVICE_ANOMALY, "%s: a tensor-core pipeline wait ran out (code %d)", who, te);
    return GC_OK;
}

int gc_siren_eval(gc_ctx *c, const float *x_dev, int64_t n, float *y_dev, float *J_dev)
{
    TRY(nn_ready(c, "gc_siren_eval"));
    if (n < 0 || (n > 0 && (!x_dev || !y_dev))) return fail(GC_ERR_INVALID, "gc_siren_eval: bad arguments");
    TRY(set_device(c));
    CUDA_TRY(gcn::neural_eval(c->nn, x_dev, n, y_dev, J_dev, c->stream));
    return nn_check_tc(c, "gc_siren_eval");
}

int gc_siren_field(gc_ctx *c, const float *x_dev, int64_t n, float *field_dev)
{
    TRY(nn_ready(c, "gc_siren_field"));
    if (n < 0 || (n > 0 && (!x_dev || !field_dev))) return fail(GC_ERR_INVALID, "gc_siren_field: bad arguments");
    TRY(set_device(c));
    CUDA_TRY(gcn::neural_field(c->nn, x_dev, n, field_dev, c->stream));
    return nn_check_tc(c, "gc_siren_field");
}

int gc_field_targets(gc_ctx *c, const float *x_dev, int64_t n, float *t_dev)
{
    TRY(nn_ready(c, "gc_field_targets"));
    if (!c->has_field) return fail(GC_ERR_STATE, "gc_field_targets: no field loaded");
    if (n < 0 || (n > 0 && (!x_dev || !t_dev))) return fail(GC_ERR_INVALID, "gc_field_targets: bad arguments");
    TRY(set_device(c));
    CUDA_TRY(gcn::neural_targets(c->nn, grid_ref(c), x_dev, n, t_dev, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GC_OK;
}

int gc_siren_loss_grad(gc_ctx *c, const float *x_dev, const float *t_dev, int64_t n, float *grad_dev,
                       double *loss_out)
{
    TRY(nn_ready(c, "gc_siren_loss_grad"));
    if (!x_dev || !t_dev || n <= 0 || n % 128 != 0 || n > ((int64_t)1 << 30))
        return fail(GC_ERR_INVALID, "gc_siren_loss_grad: need device x and t and n a positive multiple of 128");
    TRY(set_device(c));
    double loss = 0.0;
    CUDA_TRY(gcn::neural_loss_grad(c->nn, x_dev, t_dev, n, grad_dev, &loss, c->stream));
    TRY(nn_check_tc(c, "gc_siren_loss_grad"));
    if (loss_out) *loss_out = loss;
    return GC_OK;
}

int gc_field_fit(gc_ctx *c, const gc_fit_desc *f, int64_t n_samples, int n_epochs, float *loss_out)
{
    TRY(nn_ready(c, "gc_field_fit"));
    if (!c->has_field) return fail(GC_ERR_STATE, "gc_field_fit: no field loaded");
    if (!f || !f->samples || n_epochs < 0 || f->batch <= 0 || f->batch % 128 != 0 || f->batch > ((int64_t)1 << 24) ||
        n_samples < f->batch)
        return fail(GC_ERR_INVALID, "gc_field_fit: need samples, batch a positive multiple of 128 (<= 2^24) "
                                    "and n_samples >= batch");
    if (!(f->lr > 0.0) || !(f->beta1 >= 0.0 && f->beta1 < 1.0) || !(f->beta2 >= 0.0 && f->beta2 < 1.0) ||
        !(f->eps > 0.0))
        return fail(GC_ERR_INVALID, "gc_field_fit: need lr > 0, 0 <= beta1, beta2 < 1, eps > 0");
    TRY(set_device(c));
    drop_graphs(c);
    CUDA_TRY(gcn::neural_fit(c->nn, grid_ref(c), f->samples, f->samples_on_device != 0, n_samples, f->batch,
                             n_epochs, f->lr, f->beta1, f->beta2, f->eps, loss_out, c->stream));
    return nn_check_tc(c, "gc_field_fit");
}

int gc_field_select(gc_ctx *c, int source)
{
    if (!c) return fail(GC_ERR_INVALID, "gc_field_select: null context");
    if (source != GC_FIELD_GRID && source != GC_FIELD_SIREN && source != GC_FIELD_GRID_SAMPLED)
        return fail(GC_ERR_INVALID, "gc_field_select: unknown source %d", source);
    if (source == GC_FIELD_SIREN) TRY(nn_ready(c, "gc_field_select"));
    if (source != GC_FIELD_GRID) {
        if (c->gh.nodes1)
            return fail(GC_ERR_UNSUPPORTED, "gc_field_select: time-dependent fields run with GC_FIELD_GRID");
        if (c->opt.precision != GC_PREC_FP32_MIXED)
            return fail(GC_ERR_UNSUPPORTED, "gc_field_select: the split-step push runs with GC_PREC_FP32_MIXED only");
        if (!c->has_field) return fail(GC_ERR_STATE, "gc_field_select: load the grid first");
    }
    drop_graphs(c);
    c->field_source = source;
    return GC_OK;
}

} // extern "C"
