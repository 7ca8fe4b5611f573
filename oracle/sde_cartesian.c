/*
 * sde_cartesian.c -- an independent Monte Carlo solution of the backward
 * transport SDE in Cartesian coordinates (test infrastructure only: used by
 * tests/ to pin the oracle, never by the library).
 *
 * The oracle (cosmica_oracle.c) steps (r, theta, phi, ln P) with the spherical
 * form of the Ito drift (1/sqrt g) d_j (sqrt g K^ij), the analytic curl of the
 * drift potential and the Cholesky factor of 2K.  This program steps the
 * position x in Cartesian coordinates instead, with none of those pieces:
 *   dx     = (div K - V - v_d) ds + sigma dW,   sigma sigma^T = 2K        (Eq. 2-3)
 *   d lnP  = (2 V / (3 r)) ds                                             (Eq. 6)
 * where
 *   div K  (the Cartesian divergence of the tensor, sum_j d_j K_ij) and
 *   v_d    = sgn(q) sgn(A) curl(kappa_A h e_B)                             (Eq. 1)
 * are taken by central finite differences of the tensor and of the drift
 * potential as Cartesian fields, and sigma = sqrt(2 K_par) b (x) e1 +
 * sqrt(2 K_perp,r) n (x) e2 + sqrt(2 K_perp,th) e_th (x) e3 is built from the
 * field-aligned frame.  Only the model's definitions are common to both
 * programs (written here again from the reading: wind profile, Parker spiral,
 * |B| normalised at 1 AU on the equator, K_par = K0 beta P g(r), the wavy
 * current sheet h, kappa_A in AU^2/day), so a wrong coordinate scaling, a
 * dropped or mis-signed term of the spherical drift or curl, or a wrong
 * longitude equation in the oracle changes the oracle's spectrum and not this
 * one -- also when the model depends on the longitude (a tilted sheet), where
 * no 2-D reduction exists.
 *
 * Step rule: the reading of the oracle, dt = min(dt_max, eps_adv 2 K_rr / A_r^2,
 * eps_diff r^2 / K_rr, eps_diff (r delta)^2 / K_thth) >= dt_min, with K_rr and
 * K_thth the tensor's radial and polar components and A_r the radial drift of
 * r (r_hat . (div K - V - v_d) + (tr K - K_rr) / r, Ito's formula for r = |x|);
 * the caller may scale every limit.  Boundaries: exit when |x| >= R_out after a
 * step, radial reflection at r_in (x <- x (2 r_in - |x|) / |x|).
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) per particle, seeded
 * by splitmix64 of (seed, pid); normals by Box-Muller.  Particles run in
 * parallel (OpenMP); each particle's result depends only on its (seed, pid).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    double K0, kperp_r, kperp_th, B1AU_nT, V_slow_kms, V_fast_kms, lat_fast_deg, dlat_deg;
    double tilt_deg, polarity, drift_on, hcs_on;
    double R_out, R_ts, ts_K_factor, dts_AU, r_in;
    double dt_max, dt_min, eps_adv, eps_diff, dcs_min_deg, rot_period_day;
    double r0, th0, ph0;
    double A, Z, m0;
    double max_steps;
} cart_model;

#define PI 3.14159265358979323846
static const double AU_KM = 1.495978707e8, AU_M = 1.495978707e11, DAY_S = 86400.0, C_MS = 299792458.0;

/* ------------------------------------------------------------ the model -- */
typedef struct {
    double Om;          /* rotation rate [rad/day]                */
    double Vs, Vf;      /* [AU/day]                               */
    double lat_f, dlat; /* [rad]                                  */
    double B0;          /* [nT] so that |B|(1 AU, equator) = B1AU */
    double tan_tilt, dcs_min;
    double sgn_qA;
    double aoz_m0;      /* (A/|Z|) m0: rest mass per charge [GV]  */
} derived;

static double wind(const derived *d, double th)
{
    const double lat = 0.5 * PI - th;
    return d->Vs + (d->Vf - d->Vs) * 0.5 * (1.0 + tanh((fabs(lat) - d->lat_f) / d->dlat));
}

static void derive(const cart_model *m, derived *d)
{
    d->Om = 2.0 * PI / m->rot_period_day;
    d->Vs = m->V_slow_kms * DAY_S / AU_KM;
    d->Vf = m->V_fast_kms * DAY_S / AU_KM;
    d->lat_f = m->lat_fast_deg * PI / 180.0;
    d->dlat = m->dlat_deg * PI / 180.0;
    const double G0 = d->Om * 1.0 / wind(d, 0.5 * PI);
    d->B0 = m->B1AU_nT / sqrt(1.0 + G0 * G0);
    d->tan_tilt = tan(m->tilt_deg * PI / 180.0);
    d->dcs_min = m->dcs_min_deg * PI / 180.0;
    d->sgn_qA = (m->Z > 0 ? 1.0 : -1.0) * (m->polarity > 0 ? 1.0 : -1.0);
    d->aoz_m0 = m->A / fabs(m->Z) * m->m0;
}

/* spherical coordinates and the unit vectors of x */
typedef struct {
    double r, th, ph, st, ct, sp, cp;
    double er[3], et[3], ep[3];
} sph;

static void to_sph(const double x[3], sph *s)
{
    const double rho = hypot(x[0], x[1]);
    s->r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    s->th = atan2(rho, x[2]);
    s->ph = atan2(x[1], x[0]);
    s->st = rho / s->r;
    s->ct = x[2] / s->r;
    s->cp = rho > 0.0 ? x[0] / rho : 1.0;
    s->sp = rho > 0.0 ? x[1] / rho : 0.0;
    s->er[0] = s->st * s->cp; s->er[1] = s->st * s->sp; s->er[2] = s->ct;
    s->et[0] = s->ct * s->cp; s->et[1] = s->ct * s->sp; s->et[2] = -s->st;
    s->ep[0] = -s->sp;        s->ep[1] = s->cp;         s->ep[2] = 0.0;
}

static double shock(const cart_model *m, double r)
{
    if (!(m->R_ts > 0.0)) return 1.0;
    return 1.0 - (1.0 - m->ts_K_factor) * 0.5 * (1.0 + tanh((r - m->R_ts) / m->dts_AU));
}

/* field-aligned frame at x: b (along A > 0, h = +1 field), n, and Gamma */
static void frame(const cart_model *m, const derived *d, const sph *s, double b[3], double n[3], double *Gam,
                  double *V)
{
    *V = wind(d, s->th);
    *Gam = d->Om * s->r * s->st / *V;
    const double q = 1.0 / sqrt(1.0 + *Gam * *Gam);
    for (int i = 0; i < 3; ++i) {
        b[i] = q * (s->er[i] - *Gam * s->ep[i]);
        n[i] = q * (*Gam * s->er[i] + s->ep[i]);
    }
}

/* K (Cartesian, 3x3) at x for rigidity P [GV] */
static void Ktensor(const cart_model *m, const derived *d, const double x[3], double P, double K[3][3])
{
    sph s;
    to_sph(x, &s);
    double b[3], n[3], Gam, V;
    frame(m, d, &s, b, n, &Gam, &V);
    const double beta = P / sqrt(P * P + d->aoz_m0 * d->aoz_m0);
    const double Kp = m->K0 * beta * P * shock(m, s.r);
    const double Kr = m->kperp_r * Kp, Kt = m->kperp_th * Kp;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) K[i][j] = Kp * b[i] * b[j] + Kr * n[i] * n[j] + Kt * s.et[i] * s.et[j];
}

/* |B| [nT] and the current-sheet polarity h (with its half-width delta) */
static double polarity(const cart_model *m, const derived *d, const sph *s, double P, double Bmag, double *delta)
{
    *delta = 0.0;
    if (!(m->hcs_on > 0.5)) return 1.0;
    const double V = wind(d, s->th);
    const double th_cs = 0.5 * PI + atan(d->tan_tilt * sin(s->ph + d->Om * s->r / V));
    const double rL = P * 1e9 / (C_MS * Bmag * 1e-9) / AU_M;   /* Larmor radius [AU] */
    double w = 2.0 * rL / s->r;
    if (w < d->dcs_min) w = d->dcs_min;
    *delta = w;
    return tanh((th_cs - s->th) / w);
}

/* drift potential kappa_A h e_B (Cartesian) [AU^2/day] */
static void potential(const cart_model *m, const derived *d, const double x[3], double P, double W[3])
{
    sph s;
    to_sph(x, &s);
    double b[3], n[3], Gam, V, delta;
    frame(m, d, &s, b, n, &Gam, &V);
    const double Bmag = d->B0 / (s.r * s.r) * sqrt(1.0 + Gam * Gam);
    const double h = polarity(m, d, &s, P, Bmag, &delta);
    const double beta = P / sqrt(P * P + d->aoz_m0 * d->aoz_m0);
    /* kappa_A = beta P / (3 |B|): P [V] / B [T] in m^2/s, then AU^2/day */
    const double kA = beta * P * 1e9 / (3.0 * Bmag * 1e-9) * DAY_S / (AU_M * AU_M);
    for (int i = 0; i < 3; ++i) W[i] = kA * h * b[i];
}

/* drift of the SDE, b = div K - V - v_d, with the pieces the step rule needs */
static void sde_drift(const cart_model *m, const derived *d, const double x[3], double P, double bvec[3],
                      double K[3][3], double *Krr, double *Ktt, double *Ar, double *V_out, double *delta)
{
    sph s;
    to_sph(x, &s);
    Ktensor(m, d, x, P, K);
    const double hs = 1e-6 * s.r;
    double divK[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < 3; ++j) {
        double xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
        xp[j] += hs;
        xm[j] -= hs;
        double Kp[3][3], Km[3][3];
        Ktensor(m, d, xp, P, Kp);
        Ktensor(m, d, xm, P, Km);
        for (int i = 0; i < 3; ++i) divK[i] += (Kp[i][j] - Km[i][j]) / (2.0 * hs);
    }
    double vd[3] = {0.0, 0.0, 0.0};
    if (m->drift_on > 0.5) {
        double dW[3][3];   /* dW[j][i] = d_j W_i */
        for (int j = 0; j < 3; ++j) {
            double xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
            xp[j] += hs;
            xm[j] -= hs;
            double Wp[3], Wm[3];
            potential(m, d, xp, P, Wp);
            potential(m, d, xm, P, Wm);
            for (int i = 0; i < 3; ++i) dW[j][i] = (Wp[i] - Wm[i]) / (2.0 * hs);
        }
        vd[0] = d->sgn_qA * (dW[1][2] - dW[2][1]);
        vd[1] = d->sgn_qA * (dW[2][0] - dW[0][2]);
        vd[2] = d->sgn_qA * (dW[0][1] - dW[1][0]);
    }
    const double V = wind(d, s.th);
    for (int i = 0; i < 3; ++i) bvec[i] = divK[i] - V * s.er[i] - vd[i];
    double kr = 0.0, kt = 0.0, tr = 0.0, br = 0.0;
    for (int i = 0; i < 3; ++i) {
        tr += K[i][i];
        br += s.er[i] * bvec[i];
        for (int j = 0; j < 3; ++j) {
            kr += s.er[i] * K[i][j] * s.er[j];
            kt += s.et[i] * K[i][j] * s.et[j];
        }
    }
    *Krr = kr;
    *Ktt = kt;
    *Ar = br + (tr - kr) / s.r;
    *V_out = V;
    *delta = 0.0;
    if (m->hcs_on > 0.5 && m->drift_on > 0.5) {
        double bb[3], nn[3], Gam, VV;
        frame(m, d, &s, bb, nn, &Gam, &VV);
        const double Bmag = d->B0 / (s.r * s.r) * sqrt(1.0 + Gam * Gam);
        polarity(m, d, &s, P, Bmag, delta);
    }
}

/* ------------------------------------------------------------------ RNG -- */
static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xoshiro;

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xo_next(xoshiro *g)
{
    const uint64_t result = rotl(g->s[1] * 5, 7) * 9;
    const uint64_t t = g->s[1] << 17;
    g->s[2] ^= g->s[0];
    g->s[3] ^= g->s[1];
    g->s[1] ^= g->s[2];
    g->s[0] ^= g->s[3];
    g->s[2] ^= t;
    g->s[3] = rotl(g->s[3], 45);
    return result;
}

static double uniform(xoshiro *g) { return ((double)(xo_next(g) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

static void normals3(xoshiro *g, double z[3])
{
    const double u0 = uniform(g), u1 = uniform(g), u2 = uniform(g), u3 = uniform(g);
    const double a = sqrt(-2.0 * log(u0)), c = sqrt(-2.0 * log(u2));
    z[0] = a * cos(2.0 * PI * u1);
    z[1] = a * sin(2.0 * PI * u1);
    z[2] = c * cos(2.0 * PI * u3);
}

/* --------------------------------------------------------------- paths -- */
/* status: 1 exit, 2 step limit, 3 non-finite */
static void one_path(const cart_model *m, const derived *d, double T, uint64_t seed, uint64_t pid, double *lnP_out,
                     double *s_out, uint32_t *steps_out, uint8_t *status_out, double *r_out)
{
    uint64_t sm = seed * 0x2545F4914F6CDD1Dull ^ (pid + 0x632BE59BD9B4E019ull);
    xoshiro g;
    for (int i = 0; i < 4; ++i) g.s[i] = splitmix64(&sm);
    const double aoz = m->A / fabs(m->Z);
    double lnP = log(aoz * sqrt(T * (T + 2.0 * m->m0)));
    double x[3] = {m->r0 * sin(m->th0) * cos(m->ph0), m->r0 * sin(m->th0) * sin(m->ph0), m->r0 * cos(m->th0)};
    double s = 0.0;
    uint32_t k = 0;
    uint8_t status = 0;
    const uint32_t kmax = (uint32_t)m->max_steps;
    while (!status) {
        const double P = exp(lnP);
        double bvec[3], K[3][3], Krr, Ktt, Ar, V, delta;
        sde_drift(m, d, x, P, bvec, K, &Krr, &Ktt, &Ar, &V, &delta);
        sph sp;
        to_sph(x, &sp);
        double dt = m->dt_max;
        const double t1 = m->eps_adv * 2.0 * Krr / (Ar * Ar);
        const double t2 = m->eps_diff * sp.r * sp.r / Krr;
        if (t1 < dt) dt = t1;
        if (t2 < dt) dt = t2;
        if (delta > 0.0) {
            const double t3 = m->eps_diff * (sp.r * delta) * (sp.r * delta) / Ktt;
            if (t3 < dt) dt = t3;
        }
        if (dt < m->dt_min) dt = m->dt_min;
        /* noise sigma z from the field-aligned frame: sigma sigma^T = 2K */
        double b[3], n[3], Gam, VV;
        frame(m, d, &sp, b, n, &Gam, &VV);
        const double beta = P / sqrt(P * P + d->aoz_m0 * d->aoz_m0);
        const double Kp = m->K0 * beta * P * shock(m, sp.r);
        double z[3];
        normals3(&g, z);
        const double a1 = sqrt(2.0 * Kp * dt) * z[0];
        const double a2 = sqrt(2.0 * m->kperp_r * Kp * dt) * z[1];
        const double a3 = sqrt(2.0 * m->kperp_th * Kp * dt) * z[2];
        for (int i = 0; i < 3; ++i) x[i] += bvec[i] * dt + a1 * b[i] + a2 * n[i] + a3 * sp.et[i];
        lnP += 2.0 * V / (3.0 * sp.r) * dt;
        double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        if (r < m->r_in) {
            const double f = (2.0 * m->r_in - r) / r;
            for (int i = 0; i < 3; ++i) x[i] *= f;
            r = 2.0 * m->r_in - r;
        }
        s += dt;
        ++k;
        if (!isfinite(r + lnP + s)) status = 3;
        else if (r >= m->R_out) status = 1;
        else if (k >= kmax) status = 2;
        if (status) *r_out = r;
    }
    *lnP_out = lnP;
    *s_out = s;
    *steps_out = k;
    *status_out = status;
}

/* n paths of the energies T[i] with identities pid[i] */
void cart_run(const cart_model *m, uint64_t n, const double *T, const uint64_t *pid, uint64_t seed, double *lnP,
              double *s, uint32_t *steps, uint8_t *status, double *r, int threads)
{
    derived d;
    derive(m, &d);
#pragma omp parallel for schedule(dynamic, 16) num_threads(threads > 0 ? threads : omp_get_max_threads())
    for (int64_t i = 0; i < (int64_t)n; ++i)
        one_path(m, &d, T[i], seed, pid[i], lnP + i, s + i, steps + i, status + i, r + i);
}
