/*
 * gc_oracle.c -- plain FP64 CPU oracle of the guiding-centre (GC) electron
 * transport method of Houeibib, Pantellini & Griton, "Dynamics of energetic
 * electrons scattered in the solar wind" (arXiv:2403.06706).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library. The CUDA library of the
 * package never links or calls it, and the two share no source: no headers,
 * no helpers, no constants generator. It is written to be read against the
 * paper, not to be fast: every formula is spelled out in FP64 in the paper's
 * order, with no blocking, fusion or reordering.
 *
 * What it computes, by section of the paper:
 *   - field evaluation: trilinear interpolation of a spherical (r, theta, phi)
 *     grid of node values (Sect. 2.2, the sentence after Eq. 3), an
 *     analytic field (uniform + Parker spiral + dipole) used by the pins, or
 *     a neural field (a SIREN, Sitzmann et al. 2020, evaluated in FP64 with
 *     its exact Jacobian by forward-mode tangents);
 *   - the relativistic GC right-hand side F(X), X = {R, gamma v_par}: Eqs. 1-3;
 *   - the third-order predictor-corrector: Eqs. 5-6, with the backward-Euler
 *     start-up after injection and after every collision (Sect. 2.2);
 *   - hard-sphere pitch-angle scattering with a constant field-aligned mean
 *     free path: Eq. 9 (collision probability), Eq. 10 (isotropic law) and
 *     Eq. 12 (flux-weighted law), Sect. 2.3;
 *   - rebirth of particles that leave the shell, snapshot tallies (Sect. 3);
 *   - Philox-4x32-10 (Salmon et al., SC'11) as the counter-based generator.
 *
 * Readings where the paper is silent or ambiguous (each is also listed in
 * the design notes of the repository):
 *   - Eq. 1, the E_par term: the printed (v_par/gamma) E_par v_E is in units
 *     where q/m = c = 1; in SI it is (q v_par E_par / (gamma m c^2)) v_E.
 *   - "ideal" fields: E_par is set to zero after interpolation (ideal Ohm's
 *     law gives E.B = 0; separate interpolation of E and B would not).
 *   - B = |B_interp| and grad|B| = J_B^T b (gradient of the interpolated
 *     vector's norm), derivatives are those of the trilinear interpolant.
 *   - Eq. 9 uses the path length |v_par|: Delta s = dt (|v_par^n| +
 *     |v_par^{n+1}|) / 2 per step. The default collision trigger is an
 *     exponential free path (drawn, decremented by Delta s, at most one
 *     collision per step); the per-step Bernoulli draw of Eq. 9 is a flag.
 *     Both give the same law of the collision count.
 *   - Eq. 10 draws a in (0, 1], so mu' = 1 - 2a in [-1, 1).
 *   - after a collision, F^{n-1} is evaluated at X^{n-1} = X^n - dt F^n (the
 *     literal start-up rule); the same start-up follows injection and rebirth.
 *   - collisions in the inertial frame (Sect. 3): |p| and gamma conserved,
 *     mu_B recomputed with B at the collision point.
 *   - rebirth takes precedence over a collision in the same step.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_C 299792458.0 /* speed of light, m/s */
#define ORC_PI 3.14159265358979323846

/* flag bits returned per particle */
#define ORC_FLAG_OUT_OF_GRID 1u
#define ORC_FLAG_AXIS 2u
#define ORC_FLAG_NONFINITE 4u

typedef struct {
    int32_t kind;     /* 0 = grid, 1 = analytic, 2 = neural (SIREN) */
    int32_t ideal;    /* 1: E_par := 0 in the RHS; 0: E_par = E.b; 2: E_par = -b.grad(Phi) */
    int32_t dtype;    /* grid node type: 0 = float64, 1 = float32 */
    int32_t n_r, n_th, n_ph;
    int32_t parker_E; /* analytic: add E = -u x B_parker */
    int32_t pad0;
    const void *nodes; /* grid: [n_ph][n_th][n_r][8] = Bx By Bz Ex Ey Ez |B| Phi */
    double r_min, r_max; /* grid radial range, m */
    double B_unif[3];    /* T */
    double E_unif[3];    /* V/m */
    double parker_B0;    /* B_r at parker_rref, T (0 = no Parker term) */
    double parker_rref;  /* m */
    double parker_omega; /* rad/s */
    double parker_u;     /* m/s */
    double dipole_m[3];  /* T m^3, B = 3 (m.R) R / r^5 - m / r^3 */
    /* kind 2: SIREN 3 -> 256 x 4 -> 8 on x = R / siren_rscale; parameters (float64) in
     * the order W1 [256][3], b1, W2 [256][256] ([out][in]), b2, W3, b3, W4, b4, W5 [8][256],
     * b5; outputs y_B = B (r/AU)^2 / siren_Bs, y_E = E (r/AU) / siren_Es */
    const double *siren;
    double siren_omega0, siren_rscale, siren_Bs, siren_Es;
    int32_t siren_bf16; /* 1: the values carried between layers are rounded to bfloat16 */
    int32_t pad1;
    /* kind 0 with nodes1 set: a second snapshot; the field is linear in time between the
     * snapshots at t_snap0 < t_snap1 (held constant outside) */
    const void *nodes1;
    double t_snap0, t_snap1;
} orc_field;

typedef struct {
    double q, m;            /* particle charge (C) and rest mass (kg) */
    uint32_t seed;          /* Philox key word 1 */
    int32_t collision_form; /* 0: exponential free path, 1: per-step Bernoulli (Eq. 9) */
    int32_t drift_mask;     /* 0: full Eqs. 1-2; 1: dR/dt = v_par b only */
    int32_t no_scatter;     /* 1: never collide */
    int32_t no_rebirth;     /* 1: never reborn */
    int32_t pad0;
    double wind_u;          /* > 0: collisions in the frame of a radial wind of this speed
                               (m/s), Sect. 3.2; 0: in the fixed frame */
} orc_params;

typedef struct {
    double r0, lat, lon;        /* injection site: m, rad, rad */
    double E0;                  /* mono-energetic kinetic energy, J */
    double E_lo, E_hi, E_index; /* power-law spectrum dN/dE ~ E^-index on [E_lo, E_hi], J */
    double lambda;              /* field-aligned mean free path, m */
    double r_in, r_out;         /* shell, m */
    int32_t energy_law;         /* 0: mono, 1: power law */
    int32_t mu_law;             /* 0: mu0 uniform on (0,1], 1: mu0 = 1 */
    int32_t scatter_law;        /* 0: Eq. 10, 1: Eq. 12 */
    int32_t pad0;
} orc_ensemble;

typedef struct {
    int64_t n;
    double *x, *y, *z;   /* guiding-centre position R, m */
    double *u;           /* gamma v_par, m/s */
    double *mub;         /* magnetic moment mu_B, J/T */
    double *F0;          /* F^n, [4][n] */
    double *F1;          /* F^{n-1}, [4][n] */
    double *vpar;        /* v_par at X^n, m/s */
    double *s_rem;       /* remaining free path, m */
    double *h_prev;      /* step size that separates X^{n-1} from X^n, s */
    double *t_birth;     /* time of (re)birth, s */
    double *u_inj, *mub_inj; /* injection momentum state, reused at rebirth */
    uint32_t *id, *ens, *event, *ncoll, *flags;
} orc_state;

typedef struct {
    int32_t cadence, n_mu, n_E, n_r, n_age, n_ens;
    double t_start;          /* only particles born at t >= t_start are counted */
    double E_lo, E_hi;       /* log energy bins, J */
    double r_lo, r_hi;       /* linear r bins, m */
    double age_max;          /* linear age bins on [0, age_max), s */
    double rwin_lo, rwin_hi; /* radial window of the age-energy and young-PAD tallies, m */
    double age_young;        /* young-PAD age limit, s */
    uint32_t *h_mer;  /* [n_ens][n_mu][n_E][n_r] */
    uint32_t *h_age;  /* [n_ens][n_age][n_E] */
    uint32_t *h_pad;  /* [n_ens][n_mu]: age < age_young, >= 1 collision, r in window */
    uint64_t *m_cnt;  /* [n_ens][n_r] */
    uint64_t *m_sin2; /* [n_ens][n_r], sum of sin^2(alpha) in units of 2^-32 */
    uint64_t *n_seen; /* [2]: samples taken, samples outside the mu-E-r ranges */
} orc_tally;

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11, Sect. 4.2): ten rounds
 * of two 32x32->64 multiplications with the round keys bumped by the Weyl
 * constants between rounds.                                                  */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, x0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, x2, &hi1, &lo1);
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One draw of a particle's stream: key = (particle id, seed), counter =
 * (event index, 0, 0, 0); the event index is consumed.                      */
static void draw(const orc_params *p, uint32_t id, uint32_t *event, uint32_t w[4])
{
    uint32_t ctr[4] = {*event, 0u, 0u, 0u};
    uint32_t key[2] = {id, p->seed};
    orc_philox4x32_10(ctr, key, w);
    *event += 1u;
}

/* 53-bit uniform in (0, 1] from two 32-bit words. */
double orc_u53(uint32_t w_hi, uint32_t w_lo)
{
    uint64_t a = ((uint64_t)(w_hi >> 5) << 26) | (uint64_t)(w_lo >> 6);
    return ((double)a + 1.0) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* Field evaluation: values and Cartesian Jacobians J[i][j] = dF_i/dx_j.     */

typedef struct {
    double B[3], E[3];
    double JB[3][3], JE[3][3];
    double gPhi[3]; /* gradient of the potential channel (grid kind; 0 otherwise) */
    double dBdt[3], dEdt[3]; /* time derivatives (two snapshots; 0 otherwise) */
    uint32_t flags;
} orc_fields;

static double node_value(const orc_field *f, int64_t idx)
{
    if (f->dtype == 0)
        return ((const double *)f->nodes)[idx];
    return (double)((const float *)f->nodes)[idx];
}

/* Trilinear interpolation in (r, theta, phi) index space, Sect. 2.2. The grid
 * is node-centred: r_i = r_min + i dr (i < n_r), theta_j = j pi/(n_th-1)
 * (poles included), phi_k = 2 pi k / n_ph (periodic). Node vectors hold
 * Cartesian components, so the gradient needs only the chain rule
 * d/dx = rhat d/dr + thetahat (1/r) d/dtheta + phihat (1/(r sin theta)) d/dphi. */
static void grid_eval(const orc_field *f, const double R[3], orc_fields *o)
{
    const double x = R[0], y = R[1], z = R[2];
    double rho = sqrt(x * x + y * y);
    const double r = sqrt(x * x + y * y + z * z);
    o->flags = 0;
    if (rho < 1e-300) {
        o->flags |= ORC_FLAG_AXIS;
        rho = 1e-300;
    }
    const double theta = atan2(rho, z);
    double phi = atan2(y, x);
    if (phi < 0.0)
        phi += 2.0 * ORC_PI;

    const double dr = (f->r_max - f->r_min) / (double)(f->n_r - 1);
    const double dth = ORC_PI / (double)(f->n_th - 1);
    const double dph = 2.0 * ORC_PI / (double)f->n_ph;

    double xr = (r - f->r_min) / dr;
    double xt = theta / dth;
    double xp = phi / dph;
    if (!isfinite(xr) || !isfinite(xt) || !isfinite(xp)) {
        o->flags |= ORC_FLAG_NONFINITE;
        xr = 0.0; xt = 0.0; xp = 0.0;
    }
    /* positions more than one radial cell outside the grid are flagged; the
     * interpolant is extended as a constant beyond the edge nodes */
    if (xr < -1.0 || xr > (double)f->n_r)
        o->flags |= ORC_FLAG_OUT_OF_GRID;

    int64_t i = (int64_t)floor(xr);
    double fr = xr - (double)i;
    if (i < 0) {
        i = 0; fr = 0.0;
    } else if (i > f->n_r - 2) {
        i = f->n_r - 2; fr = 1.0;
    }
    int64_t j = (int64_t)floor(xt);
    double ft = xt - (double)j;
    if (j < 0) {
        j = 0; ft = 0.0;
    } else if (j > f->n_th - 2) {
        j = f->n_th - 2; ft = 1.0;
    }
    int64_t k = (int64_t)floor(xp);
    double fp = xp - (double)k;
    k = ((k % f->n_ph) + f->n_ph) % f->n_ph;

    double val[8] = {0}, d_r[8] = {0}, d_t[8] = {0}, d_p[8] = {0};
    for (int a = 0; a < 2; ++a) {
        for (int b = 0; b < 2; ++b) {
            for (int c = 0; c < 2; ++c) {
                const int64_t ii = i + a, jj = j + b, kk = (k + c) % f->n_ph;
                const double wr = a ? fr : 1.0 - fr, sr = a ? 1.0 : -1.0;
                const double wt = b ? ft : 1.0 - ft, st = b ? 1.0 : -1.0;
                const double wp = c ? fp : 1.0 - fp, sp = c ? 1.0 : -1.0;
                const int64_t base = ((kk * f->n_th + jj) * f->n_r + ii) * 8;
                for (int ch = 0; ch < 8; ++ch) {
                    const double v = node_value(f, base + ch);
                    val[ch] += wr * wt * wp * v;
                    d_r[ch] += sr * wt * wp * v;
                    d_t[ch] += wr * st * wp * v;
                    d_p[ch] += wr * wt * sp * v;
                }
            }
        }
    }
    const double rhat[3] = {x / r, y / r, z / r};
    const double that[3] = {z * x / (r * rho), z * y / (r * rho), -rho / r};
    const double phat[3] = {-y / rho, x / rho, 0.0};
    for (int ch = 0; ch < 6; ++ch) {
        const double gr = d_r[ch] / dr;
        const double gt = d_t[ch] / (dth * r);
        const double gp = d_p[ch] / (dph * rho);
        for (int jx = 0; jx < 3; ++jx) {
            const double g = gr * rhat[jx] + gt * that[jx] + gp * phat[jx];
            if (ch < 3)
                o->JB[ch][jx] = g;
            else
                o->JE[ch - 3][jx] = g;
        }
        if (ch < 3)
            o->B[ch] = val[ch];
        else
            o->E[ch - 3] = val[ch];
    }
    /* channel 7, the potential Phi of the two-fluid Ohm's law: its Cartesian gradient */
    for (int jx = 0; jx < 3; ++jx)
        o->gPhi[jx] = d_r[7] / dr * rhat[jx] + d_t[7] / (dth * r) * that[jx] + d_p[7] / (dph * rho) * phat[jx];
}

/* Analytic field used by the pins: uniform B and E, a unipolar Parker spiral
 * B = B0 rref^2 [R/r^3 - (Omega/u) zhat x R / r^2] with E = -u rhat x B
 * = B0 rref^2 Omega (zhat/r - z R/r^3), and a point dipole.                 */
static void analytic_eval(const orc_field *f, const double R[3], orc_fields *o)
{
    const double x = R[0], y = R[1], z = R[2];
    const double r2 = x * x + y * y + z * z;
    const double r = sqrt(r2);
    o->flags = 0;
    for (int i = 0; i < 3; ++i) {
        o->B[i] = f->B_unif[i];
        o->E[i] = f->E_unif[i];
        for (int j = 0; j < 3; ++j) {
            o->JB[i][j] = 0.0;
            o->JE[i][j] = 0.0;
        }
    }
    if (f->parker_B0 != 0.0) {
        const double C = f->parker_B0 * f->parker_rref * f->parker_rref;
        const double w = f->parker_omega / f->parker_u;
        const double zxR[3] = {-y, x, 0.0};
        const double Z[3][3] = {{0, -1, 0}, {1, 0, 0}, {0, 0, 0}}; /* d(zhat x R)/dR */
        const double r3 = r2 * r, r4 = r2 * r2, r5 = r4 * r;
        for (int i = 0; i < 3; ++i) {
            o->B[i] += C * (R[i] / r3 - w * zxR[i] / r2);
            for (int j = 0; j < 3; ++j) {
                const double dij = (i == j) ? 1.0 : 0.0;
                o->JB[i][j] += C * (dij / r3 - 3.0 * R[i] * R[j] / r5
                                    - w * (Z[i][j] / r2 - 2.0 * zxR[i] * R[j] / r4));
            }
        }
        if (f->parker_E) {
            const double CE = C * f->parker_omega;
            for (int i = 0; i < 3; ++i) {
                const double diz = (i == 2) ? 1.0 : 0.0;
                o->E[i] += CE * (diz / r - z * R[i] / r3);
                for (int j = 0; j < 3; ++j) {
                    const double dij = (i == j) ? 1.0 : 0.0;
                    const double djz = (j == 2) ? 1.0 : 0.0;
                    o->JE[i][j] += CE * (-diz * R[j] / r3 - djz * R[i] / r3
                                         - z * dij / r3 + 3.0 * z * R[i] * R[j] / r5);
                }
            }
        }
    }
    const double *m = f->dipole_m;
    if (m[0] != 0.0 || m[1] != 0.0 || m[2] != 0.0) {
        const double mR = m[0] * x + m[1] * y + m[2] * z;
        const double r3 = r2 * r, r5 = r3 * r2, r7 = r5 * r2;
        for (int i = 0; i < 3; ++i) {
            o->B[i] += 3.0 * mR * R[i] / r5 - m[i] / r3;
            for (int j = 0; j < 3; ++j) {
                const double dij = (i == j) ? 1.0 : 0.0;
                o->JB[i][j] += 3.0 * (m[j] * R[i] + mR * dij) / r5
                               - 15.0 * mR * R[i] * R[j] / r7 + 3.0 * m[i] * R[j] / r5;
            }
        }
    }
}

/* Neural field: the SIREN's forward pass with three forward-mode tangents t_j = dh/dx_j
 * per layer, then the unscaling B = Bs y_B (AU/r)^2, E = Es y_E (AU/r) with the product
 * rule for the Jacobians. bfloat16 rounding (8 significant bits, ties to even) of h and t
 * after each layer when siren_bf16 is set; the weights are used as given. */
#define ORC_AU 1.495978707e11
#define ORC_H 256

static double round_bf16(double a)
{
    int e;
    const double m = frexp(a, &e);
    return ldexp(nearbyint(m * 256.0), e - 8);
}

static void siren_eval(const orc_field *f, const double R[3], orc_fields *o)
{
    const double *P = f->siren;
    const double w0 = f->siren_omega0;
    const int rb = f->siren_bf16;
    double x[3], h[ORC_H], t[3][ORC_H], hn[ORC_H], tn[3][ORC_H];
    for (int j = 0; j < 3; ++j)
        x[j] = R[j] / f->siren_rscale;
    const double *W1 = P, *b1 = P + 768;
    for (int q = 0; q < ORC_H; ++q) {
        const double z = w0 * (W1[3 * q] * x[0] + W1[3 * q + 1] * x[1] + W1[3 * q + 2] * x[2] + b1[q]);
        h[q] = sin(z);
        for (int j = 0; j < 3; ++j)
            t[j][q] = w0 * cos(z) * W1[3 * q + j];
    }
    if (rb)
        for (int q = 0; q < ORC_H; ++q) {
            h[q] = round_bf16(h[q]);
            for (int j = 0; j < 3; ++j)
                t[j][q] = round_bf16(t[j][q]);
        }
    for (int k = 2; k <= 4; ++k) {
        const double *W = P + 1024 + (int64_t)(k - 2) * 65792, *b = W + 65536;
        for (int q = 0; q < ORC_H; ++q) {
            double z = b[q], a[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < ORC_H; ++i) {
                z += W[q * ORC_H + i] * h[i];
                for (int j = 0; j < 3; ++j)
                    a[j] += W[q * ORC_H + i] * t[j][i];
            }
            hn[q] = sin(z);
            for (int j = 0; j < 3; ++j)
                tn[j][q] = cos(z) * a[j];
        }
        for (int q = 0; q < ORC_H; ++q) {
            h[q] = rb ? round_bf16(hn[q]) : hn[q];
            for (int j = 0; j < 3; ++j)
                t[j][q] = rb ? round_bf16(tn[j][q]) : tn[j][q];
        }
    }
    const double *W5 = P + 198400, *b5 = P + 200448;
    double y[8], J[8][3];
    for (int c = 0; c < 8; ++c) {
        y[c] = b5[c];
        J[c][0] = J[c][1] = J[c][2] = 0.0;
        for (int i = 0; i < ORC_H; ++i) {
            y[c] += W5[c * ORC_H + i] * h[i];
            for (int j = 0; j < 3; ++j)
                J[c][j] += W5[c * ORC_H + i] * t[j][i];
        }
    }
    const double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    const double a = ORC_AU / sqrt(r2);
    for (int c = 0; c < 3; ++c) {
        o->B[c] = f->siren_Bs * y[c] * a * a;
        o->E[c] = f->siren_Es * y[3 + c] * a;
        for (int d = 0; d < 3; ++d) {
            o->JB[c][d] = f->siren_Bs * a * a * (J[c][d] / f->siren_rscale - 2.0 * y[c] * R[d] / r2);
            o->JE[c][d] = f->siren_Es * a * (J[3 + c][d] / f->siren_rscale - y[3 + c] * R[d] / r2);
        }
        /* y_Phi = Phi / (Es AU) */
        o->gPhi[c] = f->siren_Es * ORC_AU * J[7][c] / f->siren_rscale;
    }
    o->flags = 0;
}

/* Two snapshots: every quantity linear in time between them, d/dt the secant slope. */
static void grid_eval_t(const orc_field *f, const double R[3], double t, orc_fields *o)
{
    grid_eval(f, R, o);
    if (!f->nodes1)
        return;
    orc_field f1 = *f;
    f1.nodes = f->nodes1;
    orc_fields o1;
    o1.gPhi[0] = o1.gPhi[1] = o1.gPhi[2] = 0.0;
    grid_eval(&f1, R, &o1);
    const double span = f->t_snap1 - f->t_snap0;
    double w = (t - f->t_snap0) / span;
    int inside = 1;
    if (w < 0.0) {
        w = 0.0;
        inside = 0;
    } else if (w > 1.0) {
        w = 1.0;
        inside = 0;
    }
    for (int i = 0; i < 3; ++i) {
        o->dBdt[i] = inside ? (o1.B[i] - o->B[i]) / span : 0.0;
        o->dEdt[i] = inside ? (o1.E[i] - o->E[i]) / span : 0.0;
        o->B[i] = (1.0 - w) * o->B[i] + w * o1.B[i];
        o->E[i] = (1.0 - w) * o->E[i] + w * o1.E[i];
        o->gPhi[i] = (1.0 - w) * o->gPhi[i] + w * o1.gPhi[i];
        for (int j = 0; j < 3; ++j) {
            o->JB[i][j] = (1.0 - w) * o->JB[i][j] + w * o1.JB[i][j];
            o->JE[i][j] = (1.0 - w) * o->JE[i][j] + w * o1.JE[i][j];
        }
    }
    o->flags |= o1.flags;
}

static void field_eval(const orc_field *f, const double R[3], double t, orc_fields *o)
{
    o->gPhi[0] = o->gPhi[1] = o->gPhi[2] = 0.0;
    for (int i = 0; i < 3; ++i)
        o->dBdt[i] = o->dEdt[i] = 0.0;
    if (f->kind == 0)
        grid_eval_t(f, R, t, o);
    else if (f->kind == 2)
        siren_eval(f, R, o);
    else
        analytic_eval(f, R, o);
}

/* ------------------------------------------------------------------------ */
/* GC right-hand side, Eqs. 1-3. X = {R, u = gamma v_par}; mu_B constant.    */

typedef struct {
    double gamma, vpar, Bmag, Epar;
    double b[3]; /* unit vector along B */
} orc_aux;

static void cross(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void rhs_from_fields(const orc_field *f, const orc_params *p, const orc_fields *fl,
                            const double X[4], double mub, double F[4], orc_aux *aux)
{
    const double q = p->q, m = p->m, c2 = ORC_C * ORC_C;
    const double Bm = sqrt(dot(fl->B, fl->B));
    double b[3], gB[3], Jb[3][3], kap[3], vE[3], JvE[3][3];
    for (int i = 0; i < 3; ++i)
        b[i] = fl->B[i] / Bm;
    /* grad|B|_j = sum_i b_i dB_i/dx_j */
    for (int j = 0; j < 3; ++j)
        gB[j] = b[0] * fl->JB[0][j] + b[1] * fl->JB[1][j] + b[2] * fl->JB[2][j];
    /* db_i/dx_j = (dB_i/dx_j - b_i d|B|/dx_j) / |B| */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Jb[i][j] = (fl->JB[i][j] - b[i] * gB[j]) / Bm;
    /* curvature (b.grad) b */
    for (int i = 0; i < 3; ++i)
        kap[i] = Jb[i][0] * b[0] + Jb[i][1] * b[1] + Jb[i][2] * b[2];
    /* ideal 1: E_par = 0; 0: the interpolated E.b; 2: two-fluid Ohm's law (Sect. 2.2),
     * E = -u x B - grad(p)/(e n) with p = p(n), i.e. -grad(Phi): E_par = -b.grad(Phi) */
    const double Epar = f->ideal == 1 ? 0.0 : (f->ideal == 2 ? -dot(fl->gPhi, b) : dot(fl->E, b));
    /* v_E = E x b / B = E x B / B^2 */
    double ExB[3];
    cross(fl->E, fl->B, ExB);
    for (int i = 0; i < 3; ++i)
        vE[i] = ExB[i] / (Bm * Bm);
    /* dv_E/dx_j = (dE/dx_j x B + E x dB/dx_j) / B^2 - 2 v_E (d|B|/dx_j) / |B| */
    for (int j = 0; j < 3; ++j) {
        const double dE[3] = {fl->JE[0][j], fl->JE[1][j], fl->JE[2][j]};
        const double dB[3] = {fl->JB[0][j], fl->JB[1][j], fl->JB[2][j]};
        double t1[3], t2[3];
        cross(dE, fl->B, t1);
        cross(fl->E, dB, t2);
        for (int i = 0; i < 3; ++i)
            JvE[i][j] = (t1[i] + t2[i]) / (Bm * Bm) - 2.0 * vE[i] * gB[j] / Bm;
    }
    double vE_grad_b[3], b_grad_vE[3], vE_grad_vE[3];
    for (int i = 0; i < 3; ++i) {
        vE_grad_b[i] = Jb[i][0] * vE[0] + Jb[i][1] * vE[1] + Jb[i][2] * vE[2];
        b_grad_vE[i] = JvE[i][0] * b[0] + JvE[i][1] * b[1] + JvE[i][2] * b[2];
        vE_grad_vE[i] = JvE[i][0] * vE[0] + JvE[i][1] * vE[1] + JvE[i][2] * vE[2];
    }
    const double u = X[3];
    /* gamma^2 = 1 + (gamma v)^2 / c^2, (gamma v)^2 = u^2 + gamma^2 v_perp^2 = u^2 + 2 mu_B B / m */
    const double gamma = sqrt(1.0 + (u * u + 2.0 * mub * Bm / m) / c2);
    const double vpar = u / gamma;

    /* time-dependent fields (the terms of the GCA equations that vanish for the paper's
     * steady wind): db/dt = (dB/dt - b (b.dB/dt)) / B,
     * dv_E/dt = (dE/dt x B + E x dB/dt) / B^2 - 2 v_E (b.dB/dt) / B */
    double db_dt[3], dvE_dt[3];
    {
        const double bdB = dot(b, fl->dBdt);
        double t1[3], t2[3];
        cross(fl->dEdt, fl->B, t1);
        cross(fl->E, fl->dBdt, t2);
        for (int i = 0; i < 3; ++i) {
            db_dt[i] = (fl->dBdt[i] - b[i] * bdB) / Bm;
            dvE_dt[i] = (t1[i] + t2[i]) / (Bm * Bm) - 2.0 * vE[i] * bdB / Bm;
        }
    }

    /* Eq. 1, with v_par db/dt + dv_E/dt in the bracket for time-dependent fields */
    double br[3];
    for (int i = 0; i < 3; ++i)
        br[i] = mub / (gamma * gamma * m) * gB[i]
                + (q * vpar * Epar / (gamma * m * c2)) * vE[i]
                + vpar * vpar * kap[i]
                + vpar * (vE_grad_b[i] + b_grad_vE[i])
                + vE_grad_vE[i]
                + vpar * db_dt[i] + dvE_dt[i];
    double bxbr[3];
    cross(b, br, bxbr);
    const double pre = gamma * m / (q * Bm);
    if (p->drift_mask == 1) {
        for (int i = 0; i < 3; ++i)
            F[i] = vpar * b[i];
    } else {
        for (int i = 0; i < 3; ++i)
            F[i] = vpar * b[i] + vE[i] + pre * bxbr[i];
    }
    /* Eq. 2 */
    double w[3];
    for (int i = 0; i < 3; ++i)
        w[i] = vpar * kap[i] + vE_grad_b[i] + db_dt[i];
    if (p->drift_mask == 1)
        F[3] = (q / m) * Epar - mub / (gamma * m) * dot(b, gB);
    else
        F[3] = (q / m) * Epar - mub / (gamma * m) * dot(b, gB) + gamma * dot(vE, w);
    if (aux) {
        aux->gamma = gamma;
        aux->vpar = vpar;
        aux->Bmag = Bm;
        aux->Epar = Epar;
        for (int i = 0; i < 3; ++i)
            aux->b[i] = b[i];
    }
}

static uint32_t rhs(const orc_field *f, const orc_params *p, const double X[4], double t, double mub,
                    double F[4], orc_aux *aux)
{
    orc_fields fl;
    field_eval(f, X, t, &fl);
    rhs_from_fields(f, p, &fl, X, mub, F, aux);
    return fl.flags;
}

/* ------------------------------------------------------------------------ */
/* Predictor (Eq. 5) and corrector (Eq. 6), tau = dt^n / dt^{n-1}.            */

void orc_predictor(const double X[4], const double F0[4], const double F1[4], double dt,
                   double tau, double Xs[4])
{
    for (int i = 0; i < 4; ++i)
        Xs[i] = X[i] + dt * ((1.0 + tau / 2.0) * F0[i] - (tau / 2.0) * F1[i]);
}

void orc_corrector(const double X[4], const double F0[4], const double F1[4],
                   const double Fs[4], double dt, double tau, double X1[4])
{
    for (int i = 0; i < 4; ++i)
        X1[i] = X[i] + dt / (6.0 * (1.0 + tau))
                           * (3.0 * (F0[i] + Fs[i]) + 4.0 * tau * (F0[i] + Fs[i] / 2.0)
                              + tau * tau * (F0[i] - F1[i]));
}

/* ------------------------------------------------------------------------ */
/* Particle helpers.                                                          */

static void load(const orc_state *s, int64_t i, double X[4], double F0[4], double F1[4])
{
    X[0] = s->x[i]; X[1] = s->y[i]; X[2] = s->z[i]; X[3] = s->u[i];
    for (int c = 0; c < 4; ++c) {
        F0[c] = s->F0[c * s->n + i];
        F1[c] = s->F1[c * s->n + i];
    }
}

static void store(orc_state *s, int64_t i, const double X[4], const double F0[4], const double F1[4])
{
    s->x[i] = X[0]; s->y[i] = X[1]; s->z[i] = X[2]; s->u[i] = X[3];
    for (int c = 0; c < 4; ++c) {
        s->F0[c * s->n + i] = F0[c];
        s->F1[c * s->n + i] = F1[c];
    }
}

/* Start-up of the two-level history (Sect. 2.2): F^n = F(X^n, t),
 * X^{n-1} = X^n - dt F^n, F^{n-1} = F(X^{n-1}, t - dt).                     */
static uint32_t restart(const orc_field *f, const orc_params *p, const double X[4], double t, double mub,
                        double dt, double F0[4], double F1[4], double *vpar)
{
    orc_aux aux;
    uint32_t fl = rhs(f, p, X, t, mub, F0, &aux);
    *vpar = aux.vpar;
    double Xm[4];
    for (int c = 0; c < 4; ++c)
        Xm[c] = X[c] - dt * F0[c];
    fl |= rhs(f, p, Xm, t - dt, mub, F1, NULL);
    return fl;
}

static double lambda_of(const orc_ensemble *e, double lambda_override)
{
    return lambda_override > 0.0 ? lambda_override : e->lambda;
}

/* Injection (Sect. 3): all particles of an ensemble start at the same site
 * R0 = r0 (cos lat cos lon, cos lat sin lon, sin lat), with mu0 and, for a
 * spectrum, the energy drawn from the particle's Philox stream (events 0, 1).
 * Particle ids are contiguous from id0 in ensemble order.                    */
int orc_inject(const orc_field *f, const orc_params *p, const orc_ensemble *ens, int n_ens,
               const int64_t *counts, orc_state *s, uint32_t id0, double t0, double dt,
               int n_threads)
{
    const double c2 = ORC_C * ORC_C;
    int64_t first[256];
    int64_t total = 0;
    if (n_ens > 256)
        return -1;
    for (int e = 0; e < n_ens; ++e) {
        first[e] = total;
        total += counts[e];
    }
    if (total > s->n)
        return -2;
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < total; ++i) {
        int e = 0;
        while (e + 1 < n_ens && i >= first[e + 1])
            ++e;
        const orc_ensemble *E = &ens[e];
        uint32_t id = id0 + (uint32_t)i;
        uint32_t event = 0, w0[4], w1[4];
        draw(p, id, &event, w0);
        draw(p, id, &event, w1);
        double mu0 = (E->mu_law == 1) ? 1.0 : orc_u53(w0[0], w0[1]);
        double Ek = E->E0;
        if (E->energy_law == 1) {
            const double a = 1.0 - E->E_index;
            const double uu = orc_u53(w1[0], w1[1]);
            Ek = pow(pow(E->E_lo, a) + uu * (pow(E->E_hi, a) - pow(E->E_lo, a)), 1.0 / a);
        }
        const double mc2 = p->m * c2;
        const double gam = 1.0 + Ek / mc2;
        const double pm = ORC_C * sqrt(gam * gam - 1.0); /* |p| / m */
        double X[4];
        X[0] = E->r0 * cos(E->lat) * cos(E->lon);
        X[1] = E->r0 * cos(E->lat) * sin(E->lon);
        X[2] = E->r0 * sin(E->lat);
        orc_fields fl;
        field_eval(f, X, t0, &fl);
        const double Bm = sqrt(dot(fl.B, fl.B));
        X[3] = mu0 * pm;
        const double mub = (1.0 - mu0 * mu0) * pm * pm * p->m / (2.0 * Bm);
        double F0[4], F1[4], vpar;
        uint32_t flg = fl.flags | restart(f, p, X, t0, mub, dt, F0, F1, &vpar);
        store(s, i, X, F0, F1);
        s->mub[i] = mub;
        s->vpar[i] = vpar;
        s->s_rem[i] = -lambda_of(E, 0.0) * log(orc_u53(w0[2], w0[3]));
        s->h_prev[i] = dt;
        s->t_birth[i] = t0;
        s->u_inj[i] = X[3];
        s->mub_inj[i] = mub;
        s->id[i] = id;
        s->ens[i] = (uint32_t)e;
        s->event[i] = event;
        s->ncoll[i] = 0;
        s->flags[i] = flg;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Tally of one snapshot sample (Sect. 3: snapshots every K steps, counted
 * for particles injected after t_start).                                     */

static void tally_sample(const orc_tally *T, const orc_params *p, uint32_t e, const double X[4],
                         double mub, double Bm, double age, uint32_t ncoll)
{
    const double c2 = ORC_C * ORC_C;
    const double r = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    const double gv2 = X[3] * X[3] + 2.0 * mub * Bm / p->m; /* (gamma v)^2 */
    const double gamma = sqrt(1.0 + gv2 / c2);
    const double mu = X[3] / sqrt(gv2);
    const double Ek = (gamma - 1.0) * p->m * c2;
    const double sin2 = 1.0 - mu * mu;

    int im = (int)floor((mu + 1.0) / 2.0 * T->n_mu);
    if (im >= T->n_mu) im = T->n_mu - 1;
    if (im < 0) im = 0;
    const double xe = log(Ek / T->E_lo) / log(T->E_hi / T->E_lo) * T->n_E;
    const int iE = (xe >= 0.0 && xe < T->n_E) ? (int)floor(xe) : -1;
    const double xr = (r - T->r_lo) / (T->r_hi - T->r_lo) * T->n_r;
    const int ir = (xr >= 0.0 && xr < T->n_r) ? (int)floor(xr) : -1;

#ifdef _OPENMP
#pragma omp atomic
#endif
    T->n_seen[0] += 1;
    if (iE < 0 || ir < 0) {
#ifdef _OPENMP
#pragma omp atomic
#endif
        T->n_seen[1] += 1;
    } else {
        const int64_t h = (((int64_t)e * T->n_mu + im) * T->n_E + iE) * T->n_r + ir;
#ifdef _OPENMP
#pragma omp atomic
#endif
        T->h_mer[h] += 1;
    }
    if (ir >= 0) {
        const uint64_t s2 = (uint64_t)floor(sin2 * 4294967296.0 + 0.5);
#ifdef _OPENMP
#pragma omp atomic
#endif
        T->m_cnt[(int64_t)e * T->n_r + ir] += 1;
#ifdef _OPENMP
#pragma omp atomic
#endif
        T->m_sin2[(int64_t)e * T->n_r + ir] += s2;
    }
    if (r >= T->rwin_lo && r < T->rwin_hi) {
        const double xa = age / T->age_max * T->n_age;
        if (xa >= 0.0 && xa < T->n_age && iE >= 0) {
            const int64_t h = ((int64_t)e * T->n_age + (int)floor(xa)) * T->n_E + iE;
#ifdef _OPENMP
#pragma omp atomic
#endif
            T->h_age[h] += 1;
        }
        if (age < T->age_young && ncoll >= 1) {
#ifdef _OPENMP
#pragma omp atomic
#endif
            T->h_pad[(int64_t)e * T->n_mu + im] += 1;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Advance every particle by n_steps steps of size dt (Sect. 2.2-3).         */

int orc_advance(const orc_field *f, const orc_params *p, const orc_ensemble *ens, int n_ens,
                orc_state *s, double t0, int64_t step0, double dt, int64_t n_steps,
                double lambda_override, const orc_tally *T, uint64_t *stats, int n_threads)
{
    const double c2 = ORC_C * ORC_C;
    uint64_t n_coll = 0, n_reb = 0;
    (void)n_ens;
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : n_coll, n_reb)
#endif
    for (int64_t i = 0; i < s->n; ++i) {
        const orc_ensemble *E = &ens[s->ens[i]];
        const double lambda = lambda_of(E, lambda_override);
        double X[4], F0[4], F1[4];
        load(s, i, X, F0, F1);
        double mub = s->mub[i];
        double vpar0 = s->vpar[i];
        double s_rem = s->s_rem[i];
        double h_prev = s->h_prev[i];
        double t_birth = s->t_birth[i];
        uint32_t event = s->event[i], ncoll = s->ncoll[i], flags = s->flags[i];
        const uint32_t id = s->id[i];

        for (int64_t k = 0; k < n_steps; ++k) {
            const double t_new = t0 + (double)(k + 1) * dt;
            const double tau = dt / h_prev;
            double Xs[4], Fs[4], X1[4], Fn1[4];
            orc_aux aux1;
            orc_predictor(X, F0, F1, dt, tau, Xs);
            /* both evaluations of the step are at the step's end time t^{n+1} */
            flags |= rhs(f, p, Xs, t_new, mub, Fs, NULL);
            orc_corrector(X, F0, F1, Fs, dt, tau, X1);
            flags |= rhs(f, p, X1, t_new, mub, Fn1, &aux1);

            const double ds = dt * (fabs(vpar0) + fabs(aux1.vpar)) / 2.0;
            const double r1 = sqrt(X1[0] * X1[0] + X1[1] * X1[1] + X1[2] * X1[2]);
            int collide = 0;
            if (!p->no_scatter) {
                if (p->collision_form == 0) {
                    s_rem -= ds;
                    collide = (s_rem <= 0.0);
                } else {
                    uint32_t w[4];
                    draw(p, id, &event, w);
                    const double a = orc_u53(w[0], w[1]);
                    collide = (a < 1.0 - exp(-ds / lambda));
                }
            }
            const int reborn = !p->no_rebirth && (r1 < E->r_in || r1 > E->r_out);
            for (int c = 0; c < 4; ++c)
                X[c] = X1[c];

            if (reborn) {
                /* Sect. 3: re-initialised on the same field line with the same
                 * initial velocity */
                X[0] = E->r0 * cos(E->lat) * cos(E->lon);
                X[1] = E->r0 * cos(E->lat) * sin(E->lon);
                X[2] = E->r0 * sin(E->lat);
                X[3] = s->u_inj[i];
                mub = s->mub_inj[i];
                uint32_t w[4];
                draw(p, id, &event, w);
                s_rem = -lambda * log(orc_u53(w[2], w[3]));
                ncoll = 0;
                t_birth = t_new;
                flags |= restart(f, p, X, t_new, mub, dt, F0, F1, &vpar0);
                h_prev = dt;
                n_reb += 1;
            } else if (collide) {
                uint32_t w[4];
                draw(p, id, &event, w);
                const double a = orc_u53(w[0], w[1]);
                double mu_new;
                if (E->scatter_law == 0)
                    mu_new = 1.0 - 2.0 * a; /* Eq. 10 */
                else
                    mu_new = ((w[0] & 1u) ? -1.0 : 1.0) * sqrt(a); /* Eq. 12 */
                const double Bm = aux1.Bmag;
                if (p->wind_u > 0.0) {
                    /* Sect. 3.2: elastic in the frame of the scattering centres, which
                     * move with the wind u = wind_u R/r. The guiding centre already
                     * drifts with the perpendicular part of u (the E x B drift), so
                     * the frame change is a boost along b by V = u.b; p_perp is
                     * unchanged by it. Per unit mass: u~ = g_V (u - V gamma),
                     * gamma~ = g_V (gamma - V u / c^2), and back with -V. */
                    const double V = p->wind_u * dot(X, aux1.b) / r1;
                    const double gV = 1.0 / sqrt(1.0 - V * V / c2);
                    const double pp2 = 2.0 * mub * Bm / p->m; /* (p_perp/m)^2 */
                    const double gam = sqrt(1.0 + (X[3] * X[3] + pp2) / c2);
                    const double ut = gV * (X[3] - V * gam);
                    const double pt2 = ut * ut + pp2; /* (|p~|/m)^2, kept by the collision */
                    const double gt = sqrt(1.0 + pt2 / c2);
                    const double ut_new = mu_new * sqrt(pt2);
                    X[3] = gV * (ut_new + V * gt);
                    mub = (1.0 - mu_new * mu_new) * pt2 * p->m / (2.0 * Bm);
                } else {
                    /* inertial-frame elastic collision: |p| fixed, B at R^{n+1} */
                    const double pm2 = X[3] * X[3] + 2.0 * mub * Bm / p->m; /* (|p|/m)^2 */
                    const double pm = sqrt(pm2);
                    X[3] = mu_new * pm;
                    mub = (1.0 - mu_new * mu_new) * pm2 * p->m / (2.0 * Bm);
                }
                if (p->collision_form == 0)
                    s_rem = -lambda * log(orc_u53(w[2], w[3]));
                ncoll += 1;
                n_coll += 1;
                flags |= restart(f, p, X, t_new, mub, dt, F0, F1, &vpar0);
                h_prev = dt;
            } else {
                for (int c = 0; c < 4; ++c) {
                    F1[c] = F0[c];
                    F0[c] = Fn1[c];
                }
                vpar0 = aux1.vpar;
                h_prev = dt;
            }
            for (int c = 0; c < 4; ++c)
                if (!isfinite(X[c]) || !isfinite(F0[c]))
                    flags |= ORC_FLAG_NONFINITE;

            if (T && T->cadence > 0 && ((step0 + k + 1) % T->cadence) == 0
                && t_birth >= T->t_start) {
                orc_fields fl;
                field_eval(f, X, t_new, &fl);
                const double Bm = sqrt(dot(fl.B, fl.B));
                tally_sample(T, p, s->ens[i], X, mub, Bm, t_new - t_birth, ncoll);
            }
        }
        (void)c2;
        store(s, i, X, F0, F1);
        s->mub[i] = mub;
        s->vpar[i] = vpar0;
        s->s_rem[i] = s_rem;
        s->h_prev[i] = h_prev;
        s->t_birth[i] = t_birth;
        s->event[i] = event;
        s->ncoll[i] = ncoll;
        s->flags[i] = flags;
    }
    if (stats) {
        stats[0] += n_coll;
        stats[1] += n_reb;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Single-point entry points for the pins.                                    */

uint32_t orc_field_eval(const orc_field *f, const double R[3], double t, double out[33])
{
    orc_fields fl;
    field_eval(f, R, t, &fl);
    for (int i = 0; i < 3; ++i) {
        out[24 + i] = fl.gPhi[i];
        out[27 + i] = fl.dBdt[i];
        out[30 + i] = fl.dEdt[i];
        out[i] = fl.B[i];
        out[3 + i] = fl.E[i];
        for (int j = 0; j < 3; ++j) {
            out[6 + 3 * i + j] = fl.JB[i][j];
            out[15 + 3 * i + j] = fl.JE[i][j];
        }
    }
    return fl.flags;
}

uint32_t orc_rhs(const orc_field *f, const orc_params *p, const double X[4], double t, double mub,
                 double F[4], double aux_out[4])
{
    orc_aux aux;
    uint32_t fl = rhs(f, p, X, t, mub, F, &aux);
    if (aux_out) {
        aux_out[0] = aux.gamma;
        aux_out[1] = aux.vpar;
        aux_out[2] = aux.Bmag;
        aux_out[3] = aux.Epar;
    }
    return fl;
}

int orc_abi_version(void) { return 1; }
