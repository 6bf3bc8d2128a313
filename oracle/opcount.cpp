// opcount.cpp -- the floating-point operation count of one particle-step of the oracle
// (test infrastructure, like the rest of oracle/): gc_oracle.c compiled with an
// op-counting scalar in place of double, one particle advanced through the grid field of
// the perturbed Parker workload, and the operations counted per step.
//
// Counting convention: +, -, *, / one flop each (the oracle is compiled with
// floating-point contraction off, so a product and a sum are two flops, as a fused
// multiply-add is two); sqrt, atan2, exp, log, sin, cos, pow and floor one flop each; sign
// changes, absolute values, comparisons and conversions none.
//
// Usage: opcount <grid file of float32 nodes> n_r n_th n_ph r_min_m r_max_m n_steps
// prints: flop_per_step evaluations_per_step
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

namespace opc {
uint64_t n_flop = 0;
}

struct CD {
    double v;
    CD() : v(0.0) {}
    template <typename A, typename = typename std::enable_if<std::is_arithmetic<A>::value>::type>
    CD(A a) : v((double)a) {}
    explicit operator double() const { return v; }
    template <typename I, typename = typename std::enable_if<std::is_integral<I>::value>::type>
    explicit operator I() const { return (I)v; }
    CD &operator+=(const CD &o) { ++opc::n_flop; v += o.v; return *this; }
    CD &operator-=(const CD &o) { ++opc::n_flop; v -= o.v; return *this; }
    CD &operator*=(const CD &o) { ++opc::n_flop; v *= o.v; return *this; }
    CD &operator/=(const CD &o) { ++opc::n_flop; v /= o.v; return *this; }
    CD operator-() const { return CD(-v); }
};
inline CD operator+(const CD &a, const CD &b) { ++opc::n_flop; return CD(a.v + b.v); }
inline CD operator-(const CD &a, const CD &b) { ++opc::n_flop; return CD(a.v - b.v); }
inline CD operator*(const CD &a, const CD &b) { ++opc::n_flop; return CD(a.v * b.v); }
inline CD operator/(const CD &a, const CD &b) { ++opc::n_flop; return CD(a.v / b.v); }
inline bool operator<(const CD &a, const CD &b) { return a.v < b.v; }
inline bool operator>(const CD &a, const CD &b) { return a.v > b.v; }
inline bool operator<=(const CD &a, const CD &b) { return a.v <= b.v; }
inline bool operator>=(const CD &a, const CD &b) { return a.v >= b.v; }
inline bool operator==(const CD &a, const CD &b) { return a.v == b.v; }
inline bool operator!=(const CD &a, const CD &b) { return a.v != b.v; }
inline CD sqrt(const CD &a) { ++opc::n_flop; return CD(std::sqrt(a.v)); }
inline CD atan2(const CD &a, const CD &b) { ++opc::n_flop; return CD(std::atan2(a.v, b.v)); }
inline CD exp(const CD &a) { ++opc::n_flop; return CD(std::exp(a.v)); }
inline CD log(const CD &a) { ++opc::n_flop; return CD(std::log(a.v)); }
inline CD sin(const CD &a) { ++opc::n_flop; return CD(std::sin(a.v)); }
inline CD cos(const CD &a) { ++opc::n_flop; return CD(std::cos(a.v)); }
inline CD pow(const CD &a, const CD &b) { ++opc::n_flop; return CD(std::pow(a.v, b.v)); }
inline CD floor(const CD &a) { ++opc::n_flop; return CD(std::floor(a.v)); }
inline CD fabs(const CD &a) { return CD(std::fabs(a.v)); }
inline CD nearbyint(const CD &a) { return CD(std::nearbyint(a.v)); }
inline bool isfinite(const CD &a) { return std::isfinite(a.v); }
inline CD frexp(const CD &a, int *e) { return CD(std::frexp(a.v, e)); }
inline CD ldexp(const CD &a, int e) { return CD(std::ldexp(a.v, e)); }

#define double CD
#include "gc_oracle.c"
#undef double

int main(int argc, char **argv)
{
    if (argc < 8) {
        std::fprintf(stderr, "usage: %s nodes.f32 n_r n_th n_ph r_min_m r_max_m n_steps [n_particles]\n", argv[0]);
        return 2;
    }
    const int n_r = std::atoi(argv[2]), n_th = std::atoi(argv[3]), n_ph = std::atoi(argv[4]);
    const double r_min = std::atof(argv[5]), r_max = std::atof(argv[6]);
    const long n_steps = std::atol(argv[7]);
    const long n = argc > 8 ? std::atol(argv[8]) : 64;
    const size_t nval = (size_t)n_r * n_th * n_ph * 8;
    float *nodes = (float *)std::malloc(nval * sizeof(float));
    FILE *fp = std::fopen(argv[1], "rb");
    if (!fp || std::fread(nodes, sizeof(float), nval, fp) != nval) {
        std::fprintf(stderr, "cannot read %zu float32 node values from %s\n", nval, argv[1]);
        return 2;
    }
    std::fclose(fp);

    const double AU = 1.495978707e11, KEV = 1.602176634e-16, PI = 3.14159265358979323846;
    orc_field f;
    std::memset((void *)&f, 0, sizeof f);
    f.kind = 0;
    f.ideal = 1;
    f.dtype = 1;
    f.n_r = n_r;
    f.n_th = n_th;
    f.n_ph = n_ph;
    f.nodes = nodes;
    f.r_min = r_min;
    f.r_max = r_max;
    orc_params p;
    std::memset((void *)&p, 0, sizeof p);
    p.q = -1.602176634e-19;
    p.m = 9.1093837015e-31;
    orc_ensemble e;
    std::memset((void *)&e, 0, sizeof e);
    e.r0 = 0.28 * AU;
    e.lat = 24.0 * PI / 180.0;
    e.lon = 0.0;
    e.E0 = 81.0 * KEV;
    e.lambda = 0.5 * AU;
    e.r_in = 0.28 * AU;
    e.r_out = 2.4 * AU;

    CD *d[11];
    for (auto &a : d) a = new CD[n];
    CD *F0 = new CD[4 * n], *F1 = new CD[4 * n];
    uint32_t *u[5];
    for (auto &a : u) a = new uint32_t[n]();
    orc_state s;
    s.n = n;
    s.x = d[0]; s.y = d[1]; s.z = d[2]; s.u = d[3]; s.mub = d[4]; s.vpar = d[5]; s.s_rem = d[6];
    s.h_prev = d[7]; s.t_birth = d[8]; s.u_inj = d[9]; s.mub_inj = d[10];
    s.F0 = F0; s.F1 = F1;
    s.id = u[0]; s.ens = u[1]; s.event = u[2]; s.ncoll = u[3]; s.flags = u[4];
    const int64_t counts[1] = {n};
    if (orc_inject(&f, &p, &e, 1, counts, &s, 0, 0.0, 0.5, 1) != 0) return 1;
    uint64_t stats[2] = {0, 0};
    opc::n_flop = 0;
    if (orc_advance(&f, &p, &e, 1, &s, 0.0, 0, 0.5, n_steps, 0.0, nullptr, stats, 1) != 0) return 1;
    std::printf("%.3f %llu %llu\n", (double)opc::n_flop / ((double)n * (double)n_steps),
                (unsigned long long)stats[0], (unsigned long long)stats[1]);
    return 0;
}
