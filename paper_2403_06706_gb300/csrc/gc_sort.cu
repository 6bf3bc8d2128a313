// gc_sort.cu -- counting sort of the particle structure-of-arrays by coarse grid cell.
//
// Particles that share grid cells then share warps, so the eight corner records of a
// field gather hit the same L1/L2 lines. The sort does not change any result: every
// random draw is keyed by the particle id and every tally is an integer sum.
//   1. key: coarse cell of each particle; rank: its slot in the bin (atomic counter)
//   2. exclusive scan of the bin counts (one block)
//   3. scatter of every state array to offset[key] + rank, then a pointer swap
#include <algorithm>

#include "gc_sort.h"

namespace gcp {

namespace {

struct KeyGeom {
    double r_min, inv_dr, inv_dth, inv_dph;
    int n_r, n_th, n_ph, shift;
    int nr_c, nth_c, nph_c;
};

__global__ void key_kernel(const double *__restrict__ x, const double *__restrict__ y,
                           const double *__restrict__ z, int64_t n, KeyGeom g, uint32_t *key,
                           uint32_t *rank, uint32_t *hist)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double X = x[i], Y = y[i], Z = z[i];
        const double rho = sqrt(X * X + Y * Y);
        const double r = sqrt(X * X + Y * Y + Z * Z);
        const double th = atan2(rho, Z);
        double ph = atan2(Y, X);
        if (ph < 0.0) ph += 6.283185307179586;
        double fi = (r - g.r_min) * g.inv_dr, fj = th * g.inv_dth, fk = ph * g.inv_dph;
        if (!(isfinite(fi) && isfinite(fj) && isfinite(fk))) { fi = 0; fj = 0; fk = 0; }
        const int i_ = (int)fmin(fmax(floor(fi), 0.0), (double)(g.n_r - 1));
        const int j_ = (int)fmin(fmax(floor(fj), 0.0), (double)(g.n_th - 1));
        const int k_ = (int)fmin(fmax(floor(fk), 0.0), (double)(g.n_ph - 1));
        const uint32_t kk = ((uint32_t)(k_ >> g.shift) * g.nth_c + (uint32_t)(j_ >> g.shift)) * g.nr_c +
                            (uint32_t)(i_ >> g.shift);
        key[i] = kk;
        rank[i] = atomicAdd(hist + kk, 1u);
    }
}

// exclusive scan of hist[0..nb) in place, one block of 1024 threads
__global__ void __launch_bounds__(1024) scan_kernel(uint32_t *hist, int nb)
{
    __shared__ uint32_t part[1024];
    const int per = (nb + 1023) / 1024;
    const int lo = threadIdx.x * per;
    const int hi = min(lo + per, nb);
    uint32_t sum = 0;
    for (int i = lo; i < hi; ++i) sum += hist[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = (threadIdx.x >= (unsigned)off) ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - sum; // exclusive prefix of this thread's chunk
    for (int i = lo; i < hi; ++i) {
        const uint32_t c = hist[i];
        hist[i] = run;
        run += c;
    }
}

// all 19 double rows (11 arrays + 4 rows each of F0, F1) and 5 uint32 arrays
struct Scatter {
    const double *src_d[19];
    double *dst_d[19];
    const uint32_t *src_u[5];
    uint32_t *dst_u[5];
};

__global__ void scatter_kernel(Scatter S, int64_t n, const uint32_t *__restrict__ key,
                               const uint32_t *__restrict__ rank, const uint32_t *__restrict__ off)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = (int64_t)off[key[i]] + rank[i];
#pragma unroll
        for (int a = 0; a < 19; ++a) S.dst_d[a][d] = S.src_d[a][i];
#pragma unroll
        for (int a = 0; a < 5; ++a) S.dst_u[a][d] = S.src_u[a][i];
    }
}

__global__ void unpermute_kernel(Scatter S, int64_t n, const uint32_t *__restrict__ id, uint32_t id_lo)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = (int64_t)(id[i] - id_lo);
#pragma unroll
        for (int a = 0; a < 19; ++a) S.dst_d[a][d] = S.src_d[a][i];
#pragma unroll
        for (int a = 0; a < 5; ++a) S.dst_u[a][d] = S.src_u[a][i];
    }
}

Scatter make_scatter(const StateDev &st, const StateDev &alt)
{
    Scatter S;
    const double *sd[11] = {st.x, st.y, st.z, st.u, st.mub, st.vpar, st.s_rem, st.h_prev,
                            st.t_birth, st.u_inj, st.mub_inj};
    double *dd[11] = {alt.x, alt.y, alt.z, alt.u, alt.mub, alt.vpar, alt.s_rem, alt.h_prev,
                      alt.t_birth, alt.u_inj, alt.mub_inj};
    for (int a = 0; a < 11; ++a) {
        S.src_d[a] = sd[a];
        S.dst_d[a] = dd[a];
    }
    for (int r = 0; r < 4; ++r) {
        S.src_d[11 + r] = st.F0 + r * st.cap;
        S.dst_d[11 + r] = alt.F0 + r * st.cap;
        S.src_d[15 + r] = st.F1 + r * st.cap;
        S.dst_d[15 + r] = alt.F1 + r * st.cap;
    }
    const uint32_t *su[5] = {st.id, st.ens, st.event, st.ncoll, st.flags};
    uint32_t *du[5] = {alt.id, alt.ens, alt.event, alt.ncoll, alt.flags};
    for (int a = 0; a < 5; ++a) {
        S.src_u[a] = su[a];
        S.dst_u[a] = du[a];
    }
    return S;
}

void free_alt(StateDev &s)
{
    double *d[] = {s.x, s.y, s.z, s.u, s.mub, s.vpar, s.s_rem, s.h_prev, s.t_birth, s.u_inj, s.mub_inj, s.F0, s.F1};
    for (double *p : d)
        if (p) cudaFree(p);
    uint32_t *u[] = {s.id, s.ens, s.event, s.ncoll, s.flags};
    for (uint32_t *p : u)
        if (p) cudaFree(p);
    s = StateDev{};
}

cudaError_t alloc_alt(StateDev &s, int64_t cap)
{
    double **d[] = {&s.x, &s.y, &s.z, &s.u, &s.mub, &s.vpar, &s.s_rem, &s.h_prev, &s.t_birth, &s.u_inj, &s.mub_inj};
    for (double **p : d) {
        const cudaError_t e = cudaMalloc(p, (size_t)cap * 8);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMalloc(&s.F0, (size_t)cap * 32);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&s.F1, (size_t)cap * 32);
    if (e != cudaSuccess) return e;
    uint32_t **u[] = {&s.id, &s.ens, &s.event, &s.ncoll, &s.flags};
    for (uint32_t **p : u) {
        e = cudaMalloc(p, (size_t)cap * 4);
        if (e != cudaSuccess) return e;
    }
    s.cap = cap;
    return cudaSuccess;
}

cudaError_t ensure_alt(SortWork &w, int64_t cap)
{
    if (w.cap == cap) return cudaSuccess;
    free_alt(w.alt);
    if (w.key) cudaFree(w.key);
    if (w.rank) cudaFree(w.rank);
    w.key = w.rank = nullptr;
    w.cap = 0;
    cudaError_t e;
    if ((e = alloc_alt(w.alt, cap)) != cudaSuccess) { free_alt(w.alt); return e; }
    if ((e = cudaMalloc(&w.key, (size_t)cap * 4)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.rank, (size_t)cap * 4)) != cudaSuccess) return e;
    w.cap = cap;
    return cudaSuccess;
}

int grid_for(int64_t n, int block) { return (int)std::min<int64_t>((n + block - 1) / block, 152 * 16); }

} // namespace

void sort_free(SortWork &w)
{
    free_alt(w.alt);
    if (w.key) cudaFree(w.key);
    if (w.rank) cudaFree(w.rank);
    if (w.hist) cudaFree(w.hist);
    w = SortWork{};
}

cudaError_t unpermute_to_alt(SortWork &w, const StateDev &st, uint32_t id_lo, cudaStream_t s)
{
    const int64_t n = st.n;
    if (n == 0) return cudaSuccess;
    cudaError_t e;
    if ((e = ensure_alt(w, st.cap)) != cudaSuccess) return e;
    unpermute_kernel<<<grid_for(n, 256), 256, 0, s>>>(make_scatter(st, w.alt), n, st.id, id_lo);
    return cudaGetLastError();
}

namespace {
KeyGeom key_geom(const GridHost &g, int64_t *nbins)
{
    KeyGeom kg;
    kg.r_min = g.r_min;
    kg.inv_dr = 1.0 / g.dr;
    kg.inv_dth = 1.0 / g.dth;
    kg.inv_dph = 1.0 / g.dph;
    kg.n_r = g.n_r;
    kg.n_th = g.n_th;
    kg.n_ph = g.n_ph;
    kg.shift = 0;
    auto bins = [&](int sh) {
        return (int64_t)(((g.n_r - 1) >> sh) + 1) * (((g.n_th - 1) >> sh) + 1) * (((g.n_ph - 1) >> sh) + 1);
    };
    while (bins(kg.shift) > (1 << 18)) ++kg.shift;
    kg.nr_c = ((g.n_r - 1) >> kg.shift) + 1;
    kg.nth_c = ((g.n_th - 1) >> kg.shift) + 1;
    kg.nph_c = ((g.n_ph - 1) >> kg.shift) + 1;
    *nbins = bins(kg.shift);
    return kg;
}

cudaError_t ensure_hist(SortWork &w, int64_t nb)
{
    if (w.nbins_cap >= nb) return cudaSuccess;
    if (w.hist) cudaFree(w.hist);
    w.hist = nullptr;
    w.nbins_cap = 0;
    const cudaError_t e = cudaMalloc(&w.hist, (size_t)nb * 4);
    if (e == cudaSuccess) w.nbins_cap = nb;
    return e;
}
} // namespace

cudaError_t alloc_state(StateDev &s, int64_t cap) { return alloc_alt(s, cap); }

cudaError_t sort_preload()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, key_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, scan_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, scatter_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, unpermute_kernel);
    return e;
}
void free_state_arrays(StateDev &s) { free_alt(s); }

cudaError_t sort_reserve(SortWork &w, const StateDev &st, const GridHost &g)
{
    int64_t nb = 0;
    key_geom(g, &nb);
    cudaError_t e = ensure_alt(w, st.cap);
    if (e != cudaSuccess) return e;
    return ensure_hist(w, nb);
}

cudaError_t sort_by_cell(SortWork &w, StateDev &st, const GridHost &g, int n_ens, cudaStream_t s)
{
    (void)n_ens;
    const int64_t n = st.n;
    if (n < 2) return cudaSuccess;
    cudaGetLastError(); // report this sort's errors only
    int64_t nb = 0;
    const KeyGeom kg = key_geom(g, &nb);
    cudaError_t e;
    if ((e = ensure_alt(w, st.cap)) != cudaSuccess) return e;
    if ((e = ensure_hist(w, nb)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.hist, 0, (size_t)nb * 4, s)) != cudaSuccess) return e;
    const int grid = grid_for(n, 256);
    key_kernel<<<grid, 256, 0, s>>>(st.x, st.y, st.z, n, kg, w.key, w.rank, w.hist);
    scan_kernel<<<1, 1024, 0, s>>>(w.hist, (int)nb);
    scatter_kernel<<<grid, 256, 0, s>>>(make_scatter(st, w.alt), n, w.key, w.rank, w.hist);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // swap: the sorted copy becomes the state
    StateDev old = st;
    StateDev nw = w.alt;
    nw.n = old.n;
    nw.cap = old.cap;
    old.n = 0;
    w.alt = old;
    st = nw;
    return cudaSuccess;
}

} // namespace gcp
