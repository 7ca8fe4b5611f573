/*
 * cosmica_oracle.c -- plain, slow FP64 CPU oracle for the COSMICA hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * it is loaded by tests/, by __graft_entry__.smoke() and by bench.py's
 * cpu_baseline / reference leg, and by nothing else.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * What it computes (COSMICA, arXiv 2502.06319):
 *   - the Parker transport equation in momentum form (Eq. 5) written as the
 *     backward Kolmogorov problem (Eq. 2) and its Ito SDE system (Eq. 3),
 *     dy = A ds + B dW with C = B B^T, integrated with Euler-Maruyama (Sec. III);
 *   - the momentum drift A_P = (2/3)(V/r) P with L = 0 (Eq. 6, Sec. VI "Version 6"),
 *     integrated as d lnP = 2V/(3r) ds;
 *   - Philox4x32-10 normals (Sec. IV.A; Salmon et al., SC'11), made
 *     counter-based: counter = (step, pid_lo, pid_hi, tag), key = seed;
 *   - one independent quasi-particle per loop iteration (Sec. IV.A).
 *
 * The paper defers the SDE coefficients to another publication, so the
 * heliospheric model below is a stated reading (Parker spiral field,
 * latitude-dependent wind, field-aligned diffusion tensor, gradient-curvature
 * and current-sheet drift, termination-shock diffusion drop).  Every formula
 * is written out in FP64, in the order the step defines, with no fusion:
 * build with -O2 -ffp-contract=off.
 *
 * Elementary functions (exp, log, sin, cos, tanh, atan) are this file's own
 * Cody-Waite + series implementations, pinned against libm to a few ulp: the
 * wavy current sheet makes paths chaotic at the 1-ulp level, so the FP64 GPU
 * path evaluates the same algorithms to stay bit-identical.
 *
 * Parity status: Philox is pinned by statistics on the CPU and bit-for-bit
 * against cuRAND's Philox4_32_10 in a GPU test; the isotropic model is pinned
 * by closed forms (mean exit time, exit-point harmonic measure) and by an
 * independent 1-D PDE solver; the full-model coefficients are pinned by
 * Cartesian finite differences (Ito drift, curl, divergence), the closed-form
 * gradient-curvature drift and invariants; whole paths of the anisotropic
 * model with drifts, with no current sheet or a flat one (axisymmetric), are
 * pinned by an independent 2-D PDE solver; with the wavy (tilted) current
 * sheet, where no 2-D reduction exists, by an independent Monte Carlo solver
 * stepped in Cartesian coordinates (sde_cartesian.c: finite-difference
 * divergence of K and curl of the drift potential, its own noise factor and
 * random numbers), itself pinned to the 2-D PDE on the axisymmetric cases.
 * The adaptive step rule is pinned by scaling every limit of the rule: the
 * spectrum's deviation from the PDE falls as the square root of the step, and
 * the Richardson extrapolation to dt -> 0 meets the PDE.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- physical constants (SI unless stated) ---------------------------- */
#define ORC_PI        3.141592653589793
#define ORC_TWO_PI    6.283185307179586
#define ORC_AU_M      1.495978707e11      /* metres per astronomical unit  */
#define ORC_AU_KM     1.495978707e8       /* kilometres per AU             */
#define ORC_DAY_S     86400.0             /* seconds per day               */
#define ORC_C_MS      299792458.0         /* speed of light                */
#define ORC_DEG       0.017453292519943295

/* Exit status codes (same meaning as the library's, declared separately). */
#define ORC_RUNNING    0
#define ORC_EXIT       1
#define ORC_STEP_LIMIT 2
#define ORC_NONFINITE  3

#define ORC_MAX_SHELLS 16

/* Model parameters.  Every field is a double so that the Python side can
 * build it from a flat list; flags are 0.0 / 1.0. */
typedef struct {
    double K0;            /* AU^2/day: K_par = K0 * beta * P[GV] * g(r)         */
    double kperp_r_frac;  /* K_perp,r / K_par                                    */
    double kperp_th_frac; /* K_perp,theta / K_par                                */
    double B1AU_nT;       /* |B| at r = 1 AU in the ecliptic                     */
    double V_slow_kms;    /* wind speed at low latitude                          */
    double V_fast_kms;    /* wind speed at high latitude                         */
    double lat_fast_deg;  /* latitude of the slow/fast transition               */
    double tilt_deg;      /* current-sheet tilt angle alpha                      */
    double polarity;      /* sign of A (+1: outward field in the north)         */
    double drift_on;      /* 1: gradient-curvature (+ sheet) drift              */
    double hcs_on;        /* 1: wavy current sheet, 0: unipolar field (h = +1)  */
    double R_out;         /* AU, absorbing outer boundary                        */
    double R_ts;          /* AU, termination shock radius (0: none)              */
    double ts_K_factor;   /* diffusion factor beyond the shock                  */
    double r_in;          /* AU, reflecting inner boundary                       */
    double dt_max;        /* day                                                 */
    double dt_fixed;      /* day, > 0 selects a fixed step                       */
    double max_steps;     /* step limit                                          */
    double isotropic;     /* 1: K = K0 beta P * identity, V = V_const uniform    */
    double V_const_kms;   /* wind of the isotropic model                         */
    double eps_adv;       /* adaptive dt: advective / diffusive ratio           */
    double eps_diff;      /* adaptive dt: diffusive step / length scale         */
    double dt_min;        /* day, floor of the adaptive step                    */
    double dlat_deg;      /* width of the wind transition                        */
    double dts_AU;        /* width of the termination-shock transition           */
    double dcs_min_deg;   /* floor of the current-sheet half-width              */
    double rot_period_day;/* solar sidereal rotation period                      */
    double r0;            /* AU, start radius                                    */
    double th0;           /* rad, start colatitude                               */
    double ph0;           /* rad, start longitude                                */
    double formulation;   /* 0: momentum form (Eq. 5-6, L = 0); 1: energy form
                             (Eq. 1: T-SDE with the loss weight of Eq. 4)         */
    double n_shells;      /* radial shells of the inner heliosphere (Sec. II.B);
                             0: one region with K0 and tilt_deg above             */
    double shell_blend_AU;/* half-width of the blend at each interior shell edge */
    double squashed;      /* 1: termination shock and outer boundary are spheroids
                             squashed toward the nose (Sec. II.B); 0: spheres     */
    double nose_th;       /* rad, colatitude of the nose direction              */
    double nose_ph;       /* rad, longitude of the nose direction               */
    double ts_tail;       /* tail distance / nose distance (R_ts) of the shock   */
    double ts_flank;      /* flank semi-axis / nose distance of the shock        */
    double hp_tail;       /* the same for the outer boundary (R_out at the nose) */
    double hp_flank;
    double shell_K0[ORC_MAX_SHELLS];       /* K0 of shell k, innermost first      */
    double shell_tilt_deg[ORC_MAX_SHELLS]; /* sheet tilt of shell k               */
} orc_params;

typedef struct {
    double A;             /* mass number               */
    double Z;             /* charge number (signed)    */
    double m0;            /* rest mass per nucleon, GeV */
} orc_species;


/* ======================================================================= */
/* Deterministic FP64 elementary functions.                                 */
/* The wavy current sheet makes paths sensitive to single-ulp differences, */
/* so the oracle and the FP64 GPU path evaluate every transcendental with  */
/* the same classical algorithm in plain IEEE +,-,*,/ (no fused operations):*/
/* Cody-Waite argument reduction (Cody & Waite, "Software Manual for the   */
/* Elementary Functions", 1980) followed by truncated Taylor series.        */
/* Accuracy (pinned against libm in the tests): a few ulp; tanh to 4e-16   */
/* absolute.  sqrt is IEEE correctly rounded on both sides and stays libm. */
/* ======================================================================= */
static double dm_from_bits(uint64_t b) { double x; memcpy(&x, &b, 8); return x; }
static uint64_t dm_bits(double x) { uint64_t b; memcpy(&b, &x, 8); return b; }

/* ln 2 split so that k * DM_LN2_HI is exact for |k| < 2^21 */
#define DM_LN2_HI   0.6931471803691238
#define DM_LN2_LO   1.9082149292705877e-10
#define DM_LOG2E    1.4426950408889634
/* pi/2 split in three 33-bit pieces */
#define DM_PIO2_1   1.5707963267341256
#define DM_PIO2_2   6.077100506303966e-11
#define DM_PIO2_3   2.0222662487959506e-21
#define DM_2_OVER_PI 0.6366197723675814
#define DM_PI_2     1.5707963267948966
#define DM_PI_4     0.7853981633974483
#define DM_PI_8     0.39269908169872414
#define DM_TAN_PI_8 0.41421356237309503
#define DM_SQRT2    1.4142135623730951

double orc_exp(double x)
{
    if (!(x < 709.0)) return (x != x) ? x : 1.0 / 0.0;
    if (x < -708.0) return 0.0;
    double k = floor(x * DM_LOG2E + 0.5);
    double r = (x - k * DM_LN2_HI) - k * DM_LN2_LO;        /* |r| <= ln2 / 2 */
    double p = 1.0 / 6227020800.0;                          /* 1/13! */
    p = p * r + 1.0 / 479001600.0;
    p = p * r + 1.0 / 39916800.0;
    p = p * r + 1.0 / 3628800.0;
    p = p * r + 1.0 / 362880.0;
    p = p * r + 1.0 / 40320.0;
    p = p * r + 1.0 / 5040.0;
    p = p * r + 1.0 / 720.0;
    p = p * r + 1.0 / 120.0;
    p = p * r + 1.0 / 24.0;
    p = p * r + 1.0 / 6.0;
    p = p * r + 0.5;
    p = p * r + 1.0;
    p = p * r + 1.0;
    int ki = (int)k;
    return p * dm_from_bits((uint64_t)(ki + 1023) << 52);
}

double orc_log(double x)
{
    if (!(x > 0.0)) return (x == 0.0) ? -1.0 / 0.0 : 0.0 / 0.0;
    if (x == 1.0 / 0.0) return x;
    uint64_t b = dm_bits(x);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    double m = dm_from_bits((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull);  /* [1, 2) */
    if (m > DM_SQRT2) { m = m * 0.5; e = e + 1; }
    double s = (m - 1.0) / (m + 1.0);                       /* |s| <= 0.1716 */
    double s2 = s * s;
    /* log m = 2 atanh s = 2 s (1 + s^2/3 + s^4/5 + ... + s^22/23) */
    double q = 1.0 / 23.0;
    q = q * s2 + 1.0 / 21.0;
    q = q * s2 + 1.0 / 19.0;
    q = q * s2 + 1.0 / 17.0;
    q = q * s2 + 1.0 / 15.0;
    q = q * s2 + 1.0 / 13.0;
    q = q * s2 + 1.0 / 11.0;
    q = q * s2 + 1.0 / 9.0;
    q = q * s2 + 1.0 / 7.0;
    q = q * s2 + 1.0 / 5.0;
    q = q * s2 + 1.0 / 3.0;
    q = q * s2 + 1.0;
    double lm = 2.0 * s * q;
    double de = (double)e;
    return de * DM_LN2_HI + (de * DM_LN2_LO + lm);
}

void orc_sincos(double x, double *sn, double *cs)
{
    double k = floor(x * DM_2_OVER_PI + 0.5);
    double r = ((x - k * DM_PIO2_1) - k * DM_PIO2_2) - k * DM_PIO2_3;   /* |r| <= pi/4 */
    double r2 = r * r;
    double ps = -1.0 / 121645100408832000.0;                /* -1/19! */
    ps = ps * r2 + 1.0 / 355687428096000.0;
    ps = ps * r2 - 1.0 / 1307674368000.0;
    ps = ps * r2 + 1.0 / 6227020800.0;
    ps = ps * r2 - 1.0 / 39916800.0;
    ps = ps * r2 + 1.0 / 362880.0;
    ps = ps * r2 - 1.0 / 5040.0;
    ps = ps * r2 + 1.0 / 120.0;
    ps = ps * r2 - 1.0 / 6.0;
    ps = ps * r2 + 1.0;
    double sr = r * ps;
    double pc = 1.0 / 2432902008176640000.0;                /* 1/20! */
    pc = pc * r2 - 1.0 / 6402373705728000.0;
    pc = pc * r2 + 1.0 / 20922789888000.0;
    pc = pc * r2 - 1.0 / 87178291200.0;
    pc = pc * r2 + 1.0 / 479001600.0;
    pc = pc * r2 - 1.0 / 3628800.0;
    pc = pc * r2 + 1.0 / 40320.0;
    pc = pc * r2 - 1.0 / 720.0;
    pc = pc * r2 + 1.0 / 24.0;
    pc = pc * r2 - 0.5;
    pc = pc * r2 + 1.0;
    double cr = pc;
    int q = (int)((long long)k & 3);
    if (q == 0)      { *sn = sr;  *cs = cr;  }
    else if (q == 1) { *sn = cr;  *cs = -sr; }
    else if (q == 2) { *sn = -sr; *cs = -cr; }
    else             { *sn = -cr; *cs = sr;  }
}

double orc_tanh(double x)
{
    double a = fabs(x);
    double t;
    if (a > 20.0) t = 1.0;
    else {
        double e = orc_exp(2.0 * a);
        t = 1.0 - 2.0 / (e + 1.0);
    }
    return (x < 0.0) ? -t : t;
}

double orc_atan(double x)
{
    double a = fabs(x);
    int inv = 0;
    if (a > 1.0) { a = 1.0 / a; inv = 1; }
    double base = 0.0, y = a;
    if (a > 0.66817863791929891) {              /* tan(3 pi / 16) */
        y = (a - 1.0) / (a + 1.0);
        base = DM_PI_4;
    } else if (a > 0.19891236737965800) {       /* tan(pi / 16) */
        y = (a - DM_TAN_PI_8) / (1.0 + a * DM_TAN_PI_8);
        base = DM_PI_8;
    }
    double y2 = y * y;                          /* |y| <= 0.2 */
    double q = -1.0 / 23.0;
    q = q * y2 + 1.0 / 21.0;
    q = q * y2 - 1.0 / 19.0;
    q = q * y2 + 1.0 / 17.0;
    q = q * y2 - 1.0 / 15.0;
    q = q * y2 + 1.0 / 13.0;
    q = q * y2 - 1.0 / 11.0;
    q = q * y2 + 1.0 / 9.0;
    q = q * y2 - 1.0 / 7.0;
    q = q * y2 + 1.0 / 5.0;
    q = q * y2 - 1.0 / 3.0;
    q = q * y2 + 1.0;
    double res = base + y * q;
    if (inv) res = DM_PI_2 - res;
    return (x < 0.0) ? -res : res;
}

/* Element-wise evaluation for the tests: 0 exp, 1 log, 2 sin, 3 cos, 4 tanh, 5 atan. */
void orc_fn(int which, uint64_t n, const double *x, double *y)
{
    for (uint64_t i = 0; i < n; ++i) {
        double s, c;
        switch (which) {
        case 0: y[i] = orc_exp(x[i]); break;
        case 1: y[i] = orc_log(x[i]); break;
        case 2: orc_sincos(x[i], &s, &c); y[i] = s; break;
        case 3: orc_sincos(x[i], &s, &c); y[i] = c; break;
        case 4: y[i] = orc_tanh(x[i]); break;
        default: y[i] = orc_atan(x[i]); break;
        }
    }
}

/* ======================================================================= */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).                       */
/* Round: two 32x32->64 products of the even words with the multipliers    */
/* 0xD2511F53 and 0xCD9E8D57; the high halves are xored with the odd words */
/* and the key, the low halves pass through; the key is bumped by the Weyl */
/* constants 0x9E3779B9, 0xBB67AE85 between rounds.                         */
/* ======================================================================= */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_philox_many(uint64_t n, const uint32_t *ctr, const uint32_t key[2], uint32_t *out)
{
    for (uint64_t i = 0; i < n; ++i) orc_philox(ctr + 4 * i, key, out + 4 * i);
}

/* Three standard normals for step k of particle pid (Sec. III: dW = sqrt(ds) N(0,1)).
 * Box-Muller on the four Philox words mapped to (0,1) as (x + 1/2) 2^-32. */
void orc_normals(uint64_t seed, uint64_t pid, uint32_t step, uint32_t tag, double z[3])
{
    uint32_t ctr[4] = { step, (uint32_t)pid, (uint32_t)(pid >> 32), tag };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t w[4];
    orc_philox(ctr, key, w);
    const double two_m32 = 2.3283064365386963e-10; /* 2^-32 */
    double u0 = ((double)w[0] + 0.5) * two_m32;
    double u1 = ((double)w[1] + 0.5) * two_m32;
    double u2 = ((double)w[2] + 0.5) * two_m32;
    double u3 = ((double)w[3] + 0.5) * two_m32;
    double rho0 = sqrt(-2.0 * orc_log(u0));
    double rho2 = sqrt(-2.0 * orc_log(u2));
    double a1 = ORC_TWO_PI * u1;
    double a3 = ORC_TWO_PI * u3;
    double s1, c1, s3, c3;
    orc_sincos(a1, &s1, &c1);
    orc_sincos(a3, &s3, &c3);
    z[0] = rho0 * c1;
    z[1] = rho0 * s1;
    z[2] = rho2 * c3;
}

void orc_normals_many(uint64_t seed, uint64_t pid0, uint64_t n, uint32_t step, double *z)
{
    for (uint64_t i = 0; i < n; ++i) orc_normals(seed, pid0 + i, step, 0u, z + 3 * i);
}

/* ======================================================================= */
/* Heliospheric model (a stated reading; the paper defers the formulas).   */
/* ======================================================================= */

/* Every quantity one step needs, named after the physics. */
typedef struct {
    double P, beta;               /* rigidity [GV], speed / c            */
    double V, dV_dth;             /* radial wind [AU/day] and dV/dtheta   */
    double Gam, dGam_dr, dGam_dth;/* Parker winding Gamma = Omega r sin(th) / V */
    double Bmag, Br, Bph;         /* field [nT]: |B|, signed components   */
    double h, dh_dr, dh_dth, dh_dph, delta_cs; /* sheet polarity and width */
    double g, dg_dr;              /* termination-shock diffusion factor   */
    double dg_dth, dg_dph;        /* its angular derivatives (squashed shock) */
    double Kpar;                  /* AU^2/day                              */
    double K[3][3];               /* physical components, order r,th,ph   */
    double dKdr[3][3], dKdth[3][3], dKdph[3][3];
    double Adiv[3];               /* (1/sqrt g) d_j (sqrt g K^ij), coordinate form */
    double L[3][3];               /* lower Cholesky factor of 2K          */
    double W[3];                  /* kappa_A h e_B, physical components   */
    double vd[3];                 /* drift velocity, physical components  */
    double dlnP;                  /* d lnP / ds                            */
    double Ar_tot;                /* total radial drift of the SDE         */
    double dt;                    /* step length [day]                     */
} orc_coef;

static double sgn(double x) { return (x > 0.0) - (x < 0.0); }

/* Latitude-dependent wind: V(th) = Vs + (Vf - Vs) (1 + tanh((|lat| - lat_f)/dlat)) / 2. */
static void wind(const orc_params *p, double th, double *V, double *dV)
{
    if (p->isotropic != 0.0) {
        *V = p->V_const_kms * ORC_DAY_S / ORC_AU_KM;
        *dV = 0.0;
        return;
    }
    double Vs = p->V_slow_kms * ORC_DAY_S / ORC_AU_KM;
    double Vf = p->V_fast_kms * ORC_DAY_S / ORC_AU_KM;
    double lat = 0.5 * ORC_PI - th;
    double lat_f = p->lat_fast_deg * ORC_DEG;
    double dlat = p->dlat_deg * ORC_DEG;
    double t = orc_tanh((fabs(lat) - lat_f) / dlat);
    *V = Vs + (Vf - Vs) * 0.5 * (1.0 + t);
    /* d|lat|/dth = -sgn(lat) */
    *dV = (Vf - Vs) * 0.5 * (1.0 - t * t) / dlat * (-sgn(lat));
}

/* Field magnitude scale B0 [nT] such that |B|(1 AU, equator) = B1AU. */
static double field_B0(const orc_params *p)
{
    double V_eq, dV;
    wind(p, 0.5 * ORC_PI, &V_eq, &dV);
    double Omega = ORC_TWO_PI / p->rot_period_day;
    double G0 = Omega / V_eq;     /* r = 1 AU, sin(th) = 1 */
    return p->B1AU_nT / sqrt(1.0 + G0 * G0);
}

/* Radial shells of the inner heliosphere (Sec. II.B: the region inside the
 * termination shock is split into expanding shells, one per Carrington
 * rotation of the wind that fills it, each with its own parameters).
 * Reading: n equal shells between the Sun and the termination shock (the
 * outer boundary when there is none); shell k holds v[k]; the outermost
 * shell continues beyond the shock.  Across each interior edge R_e = e dR the
 * value passes from v[e-1] to v[e] along the cubic smoothstep
 * S(x) = x^2 (3 - 2x), x = (r - R_e + w) / (2w), over [R_e - w, R_e + w]:
 * continuous with its first derivative, which is all the drift terms use. */
static void shell_value(const orc_params *p, const double *v, double r, double *val, double *dval)
{
    int n = (int)p->n_shells;
    double R_edge = (p->R_ts > 0.0) ? p->R_ts : p->R_out;
    double dR = R_edge / n;
    double w = p->shell_blend_AU;
    int k = (int)floor(r / dR);
    if (k > n - 1) k = n - 1;
    if (k < 0) k = 0;
    int lo = -1;   /* inner shell of the edge whose blend window holds r */
    if (k >= 1 && r < k * dR + w) lo = k - 1;
    else if (k + 1 <= n - 1 && r > (k + 1) * dR - w) lo = k;
    if (lo < 0) {
        *val = v[k];
        *dval = 0.0;
        return;
    }
    double x = (r - ((lo + 1) * dR - w)) / (2.0 * w);
    double S = x * x * (3.0 - 2.0 * x);
    double dS = 6.0 * x * (1.0 - x) / (2.0 * w);
    *val = v[lo] + (v[lo + 1] - v[lo]) * S;
    *dval = (v[lo + 1] - v[lo]) * dS;
}

/* Nose-squashed heliosphere (Sec. II.B: the inner heliosphere and the
 * heliosheath are both squashed in the nose direction, the Sun's direction of
 * motion through the interstellar medium).  Reading: each surface is a spheroid
 * about the nose axis n, with the Sun on its axis, nose distance R, tail
 * distance R t and flank semi-axis R f: semi-axis a = R (1 + t)/2 along n,
 * b = R f across, centre at distance c = R (t - 1)/2 behind the Sun.  With
 * mu = cos(angle between the position and n), a point at radius r is outside
 * when (r mu + c)^2 / a^2 + r^2 (1 - mu^2) / b^2 >= 1. */
static double nose_mu(const orc_params *p, double th, double ph, double *dmu_dth, double *dmu_dph)
{
    double st, ct, sn, cn, sd, cd;
    orc_sincos(th, &st, &ct);
    orc_sincos(p->nose_th, &sn, &cn);
    orc_sincos(ph - p->nose_ph, &sd, &cd);
    if (dmu_dth) *dmu_dth = ct * sn * cd - st * cn;
    if (dmu_dph) *dmu_dph = -st * sn * sd;
    return st * sn * cd + ct * cn;
}

/* Distance R(mu) from the Sun to the spheroid (nose distance R, ratios t, f)
 * along the direction mu, and dR/dmu: the positive root of
 * A R^2 + 2 B R + C = 0, A = mu^2/a^2 + (1 - mu^2)/b^2, B = mu c / a^2,
 * C = c^2/a^2 - 1 < 0, written as R = -C / (B + sqrt(B^2 - A C)). */
static double spheroid_radius(double R, double t, double f, double mu, double *dR_dmu)
{
    double a = R * (1.0 + t) / 2.0, b = R * f, c = R * (t - 1.0) / 2.0;
    double A = mu * mu / (a * a) + (1.0 - mu * mu) / (b * b);
    double B = mu * c / (a * a);
    double C = c * c / (a * a) - 1.0;
    double Rm = -C / (B + sqrt(B * B - A * C));
    if (dR_dmu) {
        double dF_dmu = Rm * Rm * mu * (1.0 / (a * a) - 1.0 / (b * b)) + Rm * c / (a * a);
        *dR_dmu = -dF_dmu / (A * Rm + B);
    }
    return Rm;
}

/* Evaluate every coefficient of Eq. 3 at (r, th, ph, lnP). */
static void eval_coef(const orc_params *p, const orc_species *sp,
                      double r, double th, double ph, double lnP, orc_coef *c)
{
    memset(c, 0, sizeof(*c));
    double sin_th, cos_th;
    orc_sincos(th, &sin_th, &cos_th);
    double cot_th = cos_th / sin_th;

    /* rigidity and speed: P = (A/|Z|) p_n, beta = p_n / sqrt(p_n^2 + m0^2) */
    c->P = orc_exp(lnP);
    double aoz = sp->A / fabs(sp->Z);
    double pn = c->P / aoz;
    c->beta = pn / sqrt(pn * pn + sp->m0 * sp->m0);

    /* wind */
    wind(p, th, &c->V, &c->dV_dth);

    /* termination shock: g = 1 - (1 - f)(1 + tanh((r - Rts)/d))/2, with Rts the shock's
     * distance along the direction of the point when the heliosphere is squashed */
    c->dg_dth = 0.0;
    c->dg_dph = 0.0;
    if (p->R_ts > 0.0 && p->squashed != 0.0) {
        double dmu_dth, dmu_dph, dR_dmu;
        double mu = nose_mu(p, th, ph, &dmu_dth, &dmu_dph);
        double Rts = spheroid_radius(p->R_ts, p->ts_tail, p->ts_flank, mu, &dR_dmu);
        double t = orc_tanh((r - Rts) / p->dts_AU);
        double sech2 = 1.0 - t * t;
        c->g = 1.0 - (1.0 - p->ts_K_factor) * 0.5 * (1.0 + t);
        c->dg_dr = -(1.0 - p->ts_K_factor) * 0.5 * sech2 / p->dts_AU;
        c->dg_dth = (1.0 - p->ts_K_factor) * 0.5 * sech2 / p->dts_AU * dR_dmu * dmu_dth;
        c->dg_dph = (1.0 - p->ts_K_factor) * 0.5 * sech2 / p->dts_AU * dR_dmu * dmu_dph;
    } else if (p->R_ts > 0.0) {
        double t = orc_tanh((r - p->R_ts) / p->dts_AU);
        c->g = 1.0 - (1.0 - p->ts_K_factor) * 0.5 * (1.0 + t);
        c->dg_dr = -(1.0 - p->ts_K_factor) * 0.5 * (1.0 - t * t) / p->dts_AU;
    } else {
        c->g = 1.0;
        c->dg_dr = 0.0;
    }

    /* the shell holding r sets K0 and the sheet tilt */
    double K0 = p->K0, dK0_dr = 0.0, tilt = p->tilt_deg, dtilt_dr = 0.0;
    if (p->n_shells > 0.0) {
        shell_value(p, p->shell_K0, r, &K0, &dK0_dr);
        shell_value(p, p->shell_tilt_deg, r, &tilt, &dtilt_dr);
    }

    /* parallel diffusion K_par = K0(r) beta P g(r) */
    double Kbase = K0 * c->beta * c->P;
    c->Kpar = Kbase * c->g;
    double dKpar_dr = Kbase * c->dg_dr;
    if (p->n_shells > 0.0) dKpar_dr = dKpar_dr + dK0_dr * c->beta * c->P * c->g;
    double dKpar_dth = Kbase * c->dg_dth;
    double dKpar_dph = Kbase * c->dg_dph;

    if (p->isotropic != 0.0) {
        /* K = K_par * identity */
        for (int i = 0; i < 3; ++i) {
            c->K[i][i] = c->Kpar;
            c->dKdr[i][i] = dKpar_dr;
            c->dKdth[i][i] = dKpar_dth;
            c->dKdph[i][i] = dKpar_dph;
        }
        c->Gam = 0.0;
    } else {
        /* Parker spiral: Gamma = Omega r sin(th) / V(th), tan(psi) = Gamma */
        double Omega = ORC_TWO_PI / p->rot_period_day;
        c->Gam = Omega * r * sin_th / c->V;
        c->dGam_dr = c->Gam / r;
        c->dGam_dth = c->Gam * (cot_th - c->dV_dth / c->V);
        double G = c->Gam, G2 = G * G, one_G2 = 1.0 + G2;
        double c2 = 1.0 / one_G2;          /* cos^2 psi        */
        double s2 = G2 / one_G2;           /* sin^2 psi        */
        double sc = G / one_G2;            /* sin psi cos psi  */
        double dc2_dr = -2.0 * G * c->dGam_dr / (one_G2 * one_G2);
        double dc2_dth = -2.0 * G * c->dGam_dth / (one_G2 * one_G2);
        double ds2_dr = -dc2_dr, ds2_dth = -dc2_dth;
        double dsc_dr = c->dGam_dr * (1.0 - G2) / (one_G2 * one_G2);
        double dsc_dth = c->dGam_dth * (1.0 - G2) / (one_G2 * one_G2);
        double er = p->kperp_r_frac, et = p->kperp_th_frac;
        double Kpr = er * c->Kpar, Kpt = et * c->Kpar;
        double dKpr_dr = er * dKpar_dr, dKpt_dr = et * dKpar_dr;
        double dKpr_dth = er * dKpar_dth, dKpt_dth = et * dKpar_dth;

        /* K = K_par b b^T + K_perp,r n n^T + K_perp,th e_th e_th^T,
         * b = (cos psi, 0, -sin psi), n = (sin psi, 0, cos psi). */
        c->K[0][0] = c->Kpar * c2 + Kpr * s2;
        c->K[2][2] = c->Kpar * s2 + Kpr * c2;
        c->K[0][2] = (Kpr - c->Kpar) * sc;
        c->K[1][1] = Kpt;
        c->K[0][1] = 0.0;
        c->K[1][2] = 0.0;

        c->dKdr[0][0] = dKpar_dr * c2 + c->Kpar * dc2_dr + dKpr_dr * s2 + Kpr * ds2_dr;
        c->dKdr[2][2] = dKpar_dr * s2 + c->Kpar * ds2_dr + dKpr_dr * c2 + Kpr * dc2_dr;
        c->dKdr[0][2] = (dKpr_dr - dKpar_dr) * sc + (Kpr - c->Kpar) * dsc_dr;
        c->dKdr[1][1] = dKpt_dr;
        c->dKdth[0][0] = dKpar_dth * c2 + c->Kpar * dc2_dth + dKpr_dth * s2 + Kpr * ds2_dth;
        c->dKdth[2][2] = dKpar_dth * s2 + c->Kpar * ds2_dth + dKpr_dth * c2 + Kpr * dc2_dth;
        c->dKdth[0][2] = (dKpr_dth - dKpar_dth) * sc + (Kpr - c->Kpar) * dsc_dth;
        c->dKdth[1][1] = dKpt_dth;
        /* only g depends on ph (squashed shock); the spiral does not */
        double dKpr_dph = er * dKpar_dph, dKpt_dph = et * dKpar_dph;
        c->dKdph[0][0] = dKpar_dph * c2 + dKpr_dph * s2;
        c->dKdph[2][2] = dKpar_dph * s2 + dKpr_dph * c2;
        c->dKdph[0][2] = (dKpr_dph - dKpar_dph) * sc;
        c->dKdph[1][1] = dKpt_dph;
    }
    /* symmetric completion */
    c->K[1][0] = c->K[0][1];  c->K[2][0] = c->K[0][2];  c->K[2][1] = c->K[1][2];
    c->dKdr[1][0] = c->dKdr[0][1]; c->dKdr[2][0] = c->dKdr[0][2]; c->dKdr[2][1] = c->dKdr[1][2];
    c->dKdth[1][0] = c->dKdth[0][1]; c->dKdth[2][0] = c->dKdth[0][2]; c->dKdth[2][1] = c->dKdth[1][2];
    c->dKdph[1][0] = c->dKdph[0][1]; c->dKdph[2][0] = c->dKdph[0][2]; c->dKdph[2][1] = c->dKdph[1][2];

    /* Ito drift of the diffusion term in (r, th, ph): A^i = (1/sqrt g) d_j (sqrt g K^ij),
     * sqrt g = r^2 sin(th), K^ij = K_(ij) / (h_i h_j), h = (1, r, r sin th).
     * d_ph K = 0 except through a squashed shock, whose terms d_ph K^(i ph) are added. */
    {
        const double (*K)[3] = (const double (*)[3])c->K;
        const double (*Kr)[3] = (const double (*)[3])c->dKdr;
        const double (*Kt)[3] = (const double (*)[3])c->dKdth;
        c->Adiv[0] = Kr[0][0] + 2.0 * K[0][0] / r + Kt[0][1] / r + K[0][1] * cot_th / r;
        c->Adiv[1] = (Kt[1][1] + K[1][1] * cot_th) / (r * r) + Kr[0][1] / r + K[0][1] / (r * r);
        c->Adiv[2] = (Kr[0][2] + K[0][2] / r) / (r * sin_th) + Kt[1][2] / (r * r * sin_th);
        if (p->squashed != 0.0) {
            const double (*Kp)[3] = (const double (*)[3])c->dKdph;
            c->Adiv[0] = c->Adiv[0] + Kp[0][2] / (r * sin_th);
            c->Adiv[1] = c->Adiv[1] + Kp[1][2] / (r * r * sin_th);
            c->Adiv[2] = c->Adiv[2] + Kp[2][2] / (r * r * sin_th * sin_th);
        }
    }

    /* C = B B^T = 2K: lower Cholesky factor (Eq. 3) */
    {
        double a00 = 2.0 * c->K[0][0], a10 = 2.0 * c->K[1][0], a11 = 2.0 * c->K[1][1];
        double a20 = 2.0 * c->K[2][0], a21 = 2.0 * c->K[2][1], a22 = 2.0 * c->K[2][2];
        double l00 = sqrt(a00);
        double l10 = a10 / l00;
        double l11 = sqrt(a11 - l10 * l10);
        double l20 = a20 / l00;
        double l21 = (a21 - l20 * l10) / l11;
        double l22 = sqrt(a22 - l20 * l20 - l21 * l21);
        c->L[0][0] = l00;
        c->L[1][0] = l10; c->L[1][1] = l11;
        c->L[2][0] = l20; c->L[2][1] = l21; c->L[2][2] = l22;
    }

    /* field B = A h B0 (1 AU / r)^2 (e_r - Gamma e_ph)  [nT] */
    double B0 = (p->isotropic != 0.0) ? 0.0 : field_B0(p);
    c->Bmag = B0 / (r * r) * sqrt(1.0 + c->Gam * c->Gam);

    /* current-sheet polarity h = tanh((th_cs - th)/delta),
     * th_cs = pi/2 + atan(tan(alpha) sin(ph + Omega r / V(th))) */
    c->h = 1.0;
    c->delta_cs = 0.0;
    if (p->isotropic == 0.0 && p->hcs_on != 0.0) {
        double Omega = ORC_TWO_PI / p->rot_period_day;
        double sa, ca;
        orc_sincos(tilt * ORC_DEG, &sa, &ca);
        double ta = sa / ca;
        double dta_dr = (1.0 + ta * ta) * dtilt_dr * ORC_DEG;   /* shells: tilt varies with r */
        double phs = ph + Omega * r / c->V;
        double dphs_dr = Omega / c->V;
        double dphs_dth = -Omega * r * c->dV_dth / (c->V * c->V);
        double sp_, cp_;
        orc_sincos(phs, &sp_, &cp_);
        double th_cs = 0.5 * ORC_PI + orc_atan(ta * sp_);
        double dthcs = ta * cp_ / (1.0 + ta * ta * sp_ * sp_);   /* d th_cs / d phs */
        double dthcs_dta = sp_ / (1.0 + ta * ta * sp_ * sp_);    /* d th_cs / d tan(alpha) */
        /* half-width: max(2 r_L / r, delta_min), r_L = P/(c |B|) */
        double D = c->P * 1e9 / (ORC_C_MS * B0 * 1e-9 * ORC_AU_M);
        double G = c->Gam, one_G2 = 1.0 + G * G;
        double w_rl = 2.0 * D * r / sqrt(one_G2);
        double dmin = p->dcs_min_deg * ORC_DEG;
        double dd_dr = 0.0, dd_dth = 0.0;
        double delta;
        if (w_rl > dmin) {
            delta = w_rl;
            dd_dr = 2.0 * D / (one_G2 * sqrt(one_G2));
            dd_dth = -2.0 * D * r * G * c->dGam_dth / (one_G2 * sqrt(one_G2));
        } else {
            delta = dmin;
        }
        double u = (th_cs - th) / delta;
        double h = orc_tanh(u);
        double du_dr = (dthcs * dphs_dr - u * dd_dr) / delta;
        if (p->n_shells > 0.0) du_dr = du_dr + dthcs_dta * dta_dr / delta;
        double du_dth = (dthcs * dphs_dth - 1.0 - u * dd_dth) / delta;
        double du_dph = dthcs / delta;
        c->h = h;
        c->dh_dr = (1.0 - h * h) * du_dr;
        c->dh_dth = (1.0 - h * h) * du_dth;
        c->dh_dph = (1.0 - h * h) * du_dph;
        c->delta_cs = delta;
    }
    c->Br = p->polarity * c->h * B0 / (r * r);
    c->Bph = -p->polarity * c->h * B0 / (r * r) * c->Gam;

    /* drift v_d = sgn(q) sgn(A) curl(kappa_A h e_B), kappa_A = beta P / (3 |B|).
     * W_r = C_A h F, W_ph = -C_A h G with F = r^2/(1+Gamma^2), G = r^2 Gamma/(1+Gamma^2),
     * C_A = beta P / (3 B0) converted to AU^2/day. */
    if (p->isotropic == 0.0 && p->drift_on != 0.0) {
        double CA = c->beta * c->P * 1e9 * ORC_DAY_S / (3.0 * B0 * 1e-9 * ORC_AU_M * ORC_AU_M);
        double G = c->Gam, G2 = G * G, one_G2 = 1.0 + G2;
        double F = r * r / one_G2;
        double Gf = r * r * G / one_G2;
        double dF_dth = -2.0 * r * r * G * c->dGam_dth / (one_G2 * one_G2);
        double dGf_dr = r * G * (3.0 + G2) / (one_G2 * one_G2);
        double dGf_dth = r * r * c->dGam_dth * (1.0 - G2) / (one_G2 * one_G2);
        double h = c->h;
        double Wr = CA * h * F;
        double Wph = -CA * h * Gf;
        double dWph_dth = -CA * (c->dh_dth * Gf + h * dGf_dth);
        double dWph_dr = -CA * (c->dh_dr * Gf + h * dGf_dr);
        double dWr_dph = CA * c->dh_dph * F;
        double dWr_dth = CA * (c->dh_dth * F + h * dF_dth);
        double curl_r = (cot_th * Wph + dWph_dth) / r;
        double curl_th = (dWr_dph / sin_th - Wph - r * dWph_dr) / r;
        double curl_ph = -dWr_dth / r;
        double s = sgn(sp->Z) * p->polarity;
        c->W[0] = Wr; c->W[1] = 0.0; c->W[2] = Wph;
        c->vd[0] = s * curl_r;
        c->vd[1] = s * curl_th;
        c->vd[2] = s * curl_ph;
    }

    /* momentum term, Eq. 6: d lnP / ds = (1/3) div V = 2 V / (3 r) */
    c->dlnP = 2.0 * c->V / (3.0 * r);

    /* step length */
    c->Ar_tot = c->Adiv[0] - c->V - c->vd[0];
    if (p->dt_fixed > 0.0) {
        c->dt = p->dt_fixed;
    } else {
        double dt = p->dt_max;
        double Krr = c->K[0][0];
        /* advective displacement small against the diffusive one (Kruells 1994) */
        double num = p->eps_adv * 2.0 * Krr;
        double den = c->Ar_tot * c->Ar_tot;
        if (num < dt * den) dt = num / den;
        /* radial diffusive step small against r */
        double t2 = p->eps_diff * r * r / Krr;
        if (t2 < dt) dt = t2;
        /* latitudinal diffusive step small against the sheet width */
        if (c->delta_cs > 0.0 && p->drift_on != 0.0) {
            double rd = r * c->delta_cs;
            double t3 = p->eps_diff * rd * rd / c->K[1][1];
            if (t3 < dt) dt = t3;
        }
        if (dt < p->dt_min) dt = p->dt_min;
        c->dt = dt;
    }
}

/* Flattened view of eval_coef for the tests. */
enum {
    OE_P, OE_BETA, OE_V, OE_DV, OE_GAM, OE_DGAM_DR, OE_DGAM_DTH,
    OE_BMAG, OE_BR, OE_BPH, OE_H, OE_DH_DR, OE_DH_DTH, OE_DH_DPH, OE_DELTA,
    OE_G, OE_DG, OE_KPAR,
    OE_KRR, OE_KRT, OE_KRP, OE_KTT, OE_KTP, OE_KPP,
    OE_DKRR_DR, OE_DKRP_DR, OE_DKTT_DTH, OE_DKRR_DTH, OE_DKRP_DTH,
    OE_AR, OE_ATH, OE_APH,
    OE_L00, OE_L10, OE_L11, OE_L20, OE_L21, OE_L22,
    OE_WR, OE_WPH, OE_VDR, OE_VDTH, OE_VDPH,
    OE_DLNP, OE_ARTOT, OE_DT,
    OE_DG_DTH, OE_DG_DPH,
    OE_N
};

int orc_eval_n(void) { return OE_N; }

void orc_eval(const orc_params *p, const orc_species *sp,
              double r, double th, double ph, double lnP, double *out)
{
    orc_coef c;
    eval_coef(p, sp, r, th, ph, lnP, &c);
    out[OE_P] = c.P; out[OE_BETA] = c.beta; out[OE_V] = c.V; out[OE_DV] = c.dV_dth;
    out[OE_GAM] = c.Gam; out[OE_DGAM_DR] = c.dGam_dr; out[OE_DGAM_DTH] = c.dGam_dth;
    out[OE_BMAG] = c.Bmag; out[OE_BR] = c.Br; out[OE_BPH] = c.Bph;
    out[OE_H] = c.h; out[OE_DH_DR] = c.dh_dr; out[OE_DH_DTH] = c.dh_dth; out[OE_DH_DPH] = c.dh_dph;
    out[OE_DELTA] = c.delta_cs; out[OE_G] = c.g; out[OE_DG] = c.dg_dr; out[OE_KPAR] = c.Kpar;
    out[OE_KRR] = c.K[0][0]; out[OE_KRT] = c.K[0][1]; out[OE_KRP] = c.K[0][2];
    out[OE_KTT] = c.K[1][1]; out[OE_KTP] = c.K[1][2]; out[OE_KPP] = c.K[2][2];
    out[OE_DKRR_DR] = c.dKdr[0][0]; out[OE_DKRP_DR] = c.dKdr[0][2];
    out[OE_DKTT_DTH] = c.dKdth[1][1]; out[OE_DKRR_DTH] = c.dKdth[0][0]; out[OE_DKRP_DTH] = c.dKdth[0][2];
    out[OE_AR] = c.Adiv[0]; out[OE_ATH] = c.Adiv[1]; out[OE_APH] = c.Adiv[2];
    out[OE_L00] = c.L[0][0]; out[OE_L10] = c.L[1][0]; out[OE_L11] = c.L[1][1];
    out[OE_L20] = c.L[2][0]; out[OE_L21] = c.L[2][1]; out[OE_L22] = c.L[2][2];
    out[OE_WR] = c.W[0]; out[OE_WPH] = c.W[2];
    out[OE_VDR] = c.vd[0]; out[OE_VDTH] = c.vd[1]; out[OE_VDPH] = c.vd[2];
    out[OE_DLNP] = c.dlnP; out[OE_ARTOT] = c.Ar_tot; out[OE_DT] = c.dt;
    out[OE_DG_DTH] = c.dg_dth; out[OE_DG_DPH] = c.dg_dph;
}

/* ======================================================================= */
/* Euler-Maruyama step (Eq. 3) and the per-particle loop (Sec. IV.A).       */
/* Order per step: normals -> coefficients at the old state -> dt ->        */
/* update -> reflect -> s += dt, k += 1 -> exit test.                       */
/* ======================================================================= */
typedef struct {
    double r, th, ph, lnP, s;
    double T, Lam;        /* energy form: kinetic energy per nucleon, loss integral */
    double r_old;         /* radius at the start of the step */
    uint32_t k;
    int status;
} orc_state;

/* Outer boundary: r >= R_out, or outside the squashed outer spheroid. */
static int outside(const orc_params *p, double r, double th, double ph)
{
    if (p->squashed == 0.0) return r >= p->R_out;
    double mu = nose_mu(p, th, ph, 0, 0);
    double a = p->R_out * (1.0 + p->hp_tail) / 2.0, b = p->R_out * p->hp_flank;
    double c = p->R_out * (p->hp_tail - 1.0) / 2.0;
    double xa = r * mu + c;
    return xa * xa / (a * a) + r * r * (1.0 - mu * mu) / (b * b) >= 1.0;
}

static void em_step(const orc_params *p, const orc_species *sp, uint64_t seed, uint64_t pid,
                    orc_state *x, double *dt_out)
{
    double z[3];
    x->r_old = x->r;
    orc_normals(seed, pid, x->k, 0u, z);
    orc_coef c;
    eval_coef(p, sp, x->r, x->th, x->ph, x->lnP, &c);
    double dt = c.dt;
    double sdt = sqrt(dt);
    double sin_th, cos_th;
    orc_sincos(x->th, &sin_th, &cos_th);
    double Lz_r = c.L[0][0] * z[0];
    double Lz_th = c.L[1][0] * z[0] + c.L[1][1] * z[1];
    double Lz_ph = c.L[2][0] * z[0] + c.L[2][1] * z[1] + c.L[2][2] * z[2];
    double dr = (c.Adiv[0] - c.V - c.vd[0]) * dt + Lz_r * sdt;
    double dth = (c.Adiv[1] - c.vd[1] / x->r) * dt + Lz_th * sdt / x->r;
    double dph = (c.Adiv[2] - c.vd[2] / (x->r * sin_th)) * dt + Lz_ph * sdt / (x->r * sin_th);
    double dlnP = c.dlnP * dt;
    x->r = x->r + dr;
    x->th = x->th + dth;
    x->ph = x->ph + dph;
    if (p->formulation != 0.0) {
        /* Eq. 1 backward: A_T = (1/3) div V alpha T = (2/3)(V/r) alpha T,
         * alpha = (T + 2 m0)/(T + m0); loss L = div V - (1/3) div V d(alpha T)/dT
         * = (2V/(3r)) (1 + beta^2), accumulated for the weight exp(-sum L ds) of Eq. 4 */
        double alpha = (x->T + 2.0 * sp->m0) / (x->T + sp->m0);
        double A_T = 2.0 * c.V / (3.0 * x->r_old) * alpha * x->T;
        double Lloss = 2.0 * c.V / (3.0 * x->r_old) * (1.0 + c.beta * c.beta);
        x->T = x->T + A_T * dt;
        x->Lam = x->Lam + Lloss * dt;
        x->lnP = orc_log(sp->A / fabs(sp->Z) * sqrt(x->T * (x->T + 2.0 * sp->m0)));
    } else {
        x->lnP = x->lnP + dlnP;
    }
    /* reflecting inner boundary */
    if (x->r < p->r_in) x->r = 2.0 * p->r_in - x->r;
    /* fold th into [0, pi]; crossing a pole shifts ph by pi */
    {
        double t = x->th - ORC_TWO_PI * floor(x->th / ORC_TWO_PI);
        if (t > ORC_PI) {
            x->th = ORC_TWO_PI - t;
            x->ph = x->ph + ORC_PI;
        } else {
            x->th = t;
        }
    }
    x->ph = x->ph - ORC_TWO_PI * floor(x->ph / ORC_TWO_PI);
    x->s = x->s + dt;
    x->k = x->k + 1u;
    if (!(isfinite(x->r) && isfinite(x->th) && isfinite(x->ph) && isfinite(x->lnP) && isfinite(x->s))) {
        x->status = ORC_NONFINITE;
    } else if (outside(p, x->r, x->th, x->ph)) {
        x->status = ORC_EXIT;
    } else if ((double)x->k >= p->max_steps) {
        x->status = ORC_STEP_LIMIT;
    }
    if (dt_out) *dt_out = dt;
}

/* Rigidity from kinetic energy per nucleon: P = (A/|Z|) sqrt(T (T + 2 m0)). */
static double rigidity(const orc_species *sp, double T)
{
    return sp->A / fabs(sp->Z) * sqrt(T * (T + 2.0 * sp->m0));
}

static void init_state(const orc_species *sp, double T_in, double r0, double th0, double ph0, orc_state *x)
{
    x->r = r0; x->th = th0; x->ph = ph0;
    x->lnP = orc_log(rigidity(sp, T_in));
    x->T = T_in; x->Lam = 0.0;
    x->s = 0.0; x->k = 0u; x->status = ORC_RUNNING;
}

/* Propagate n quasi-particles; particle i uses parameter set prm_idx[i],
 * species sp_idx[i], initial energy T_in[i], identity pid[i], key seed[i] and
 * starts at start[3i .. 3i+2] = (r0, th0, ph0) (a point of the detector's
 * orbit, Sec. IV.A), or at the parameter set's (r0, th0, ph0) when start is
 * NULL.  Each particle is independent, so any thread count gives the same
 * result. */
void orc_run_particles(const orc_params *prm, const orc_species *spc, uint64_t n,
                       const uint32_t *prm_idx, const uint32_t *sp_idx, const double *T_in,
                       const uint64_t *pid, const uint64_t *seed, const double *start,
                       double *r, double *th, double *ph, double *lnP, double *s,
                       uint32_t *steps, uint8_t *status, double *lw, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        const orc_params *p = prm + prm_idx[i];
        const orc_species *sp = spc + sp_idx[i];
        orc_state x;
        if (start)
            init_state(sp, T_in[i], start[3 * i], start[3 * i + 1], start[3 * i + 2], &x);
        else
            init_state(sp, T_in[i], p->r0, p->th0, p->ph0, &x);
        while (x.status == ORC_RUNNING) em_step(p, sp, seed[i], pid[i], &x, 0);
        r[i] = x.r; th[i] = x.th; ph[i] = x.ph; lnP[i] = x.lnP; s[i] = x.s;
        steps[i] = x.k; status[i] = (uint8_t)x.status;
        lw[i] = -x.Lam;
    }
}

/* First nsteps states of one particle (r, th, ph, lnP, s, dt per row). */
int orc_trace(const orc_params *p, const orc_species *sp, double T_in, uint64_t pid, uint64_t seed,
              uint32_t nsteps, double *out)
{
    orc_state x;
    init_state(sp, T_in, p->r0, p->th0, p->ph0, &x);
    uint32_t i = 0;
    for (; i < nsteps && x.status == ORC_RUNNING; ++i) {
        double dt;
        em_step(p, sp, seed, pid, &x, &dt);
        out[6 * i + 0] = x.r; out[6 * i + 1] = x.th; out[6 * i + 2] = x.ph;
        out[6 * i + 3] = x.lnP; out[6 * i + 4] = x.s; out[6 * i + 5] = dt;
    }
    return (int)i;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
