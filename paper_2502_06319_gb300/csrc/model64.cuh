// model64.cuh -- the FP64 step: coefficients of Eq. 3 and one Euler-Maruyama
// step, evaluated in double in the order the definitions give them.
//
// This is the "plain FP64 GPU path".  It is written to evaluate every
// expression in the same association order as its written definition and
// uses the deterministic elementary functions of detmath64.cuh, so that,
// compiled with -fmad=false, it reproduces an FP64 reference integration of
// the same definitions bit for bit -- necessary because paths through the
// wavy current sheet amplify single roundings.
//
// Model (the paper defers the coefficients to another publication; this is
// the reading documented in cosmica.h):
//   V(th)   = Vs + (Vf - Vs) (1 + tanh((|lat| - lat_f)/dlat)) / 2
//   Gamma   = Omega r sin(th) / V(th)           (Parker spiral, tan psi = Gamma)
//   K       = K_par b b^T + K_perp,r n n^T + K_perp,th e_th e_th^T,
//             b = (cos psi, 0, -sin psi), n = (sin psi, 0, cos psi),
//             K_par = K0 beta P g(r)
//   A^i     = (1/sqrt g) d_j (sqrt g K^ij) in (r, th, ph), sqrt g = r^2 sin th
//   L L^T   = 2K (lower Cholesky)               (Eq. 3: C = B B^T)
//   v_d     = sgn(qA) curl(kappa_A h e_B), kappa_A = beta P / (3 |B|)
//   d lnP   = 2V/(3r) ds                         (Eq. 6)
#pragma once
#include "common.cuh"
#include "detmath64.cuh"
#include "philox.cuh"

namespace cosmica {
namespace m64 {

struct Coef {
    double V, dV_dth, Gam, dGam_dth;
    double K00, K11, K22, K02;
    double Ar, Ath, Aph;
    double l00, l10, l11, l20, l21, l22;
    double h, delta_cs;
    double vd0, vd1, vd2;
    double dlnP, Ar_tot, dt;
    // extra quantities for the debug evaluator
    double P, beta, Bmag, dKrr_dr, dKrp_dr, Kpar;
};

__device__ __forceinline__ double sgn(double x) { return (double)((x > 0.0) - (x < 0.0)); }

__device__ __forceinline__ void wind(const DevParams &p, double th, double *V, double *dV)
{
    if (p.isotropic != 0.0) {
        *V = p.V_const_kms * kDay_s / kAU_km;
        *dV = 0.0;
        return;
    }
    const double Vs = p.Vs_kms * kDay_s / kAU_km;
    const double Vf = p.Vf_kms * kDay_s / kAU_km;
    const double lat = 0.5 * kPi - th;
    const double lat_f = p.lat_fast_deg * kDeg;
    const double dlat = p.dlat_deg * kDeg;
    const double t = dm::tanh((fabs(lat) - lat_f) / dlat);
    *V = Vs + (Vf - Vs) * 0.5 * (1.0 + t);
    *dV = (Vf - Vs) * 0.5 * (1.0 - t * t) / dlat * (-sgn(lat));
}

// |B| scale at 1 AU; evaluated once per parameter set by k_derive.
__device__ __forceinline__ double field_B0(const DevParams &p)
{
    double V_eq, dV;
    wind(p, 0.5 * kPi, &V_eq, &dV);
    const double Omega = kTwoPi / p.rot_period;
    const double G0 = Omega / V_eq;
    return p.B1AU / sqrt(1.0 + G0 * G0);
}

// Radial shells of the inner heliosphere (Sec. II.B): n equal shells out to the
// termination shock (the outer boundary without one), shell k holding v[k], the
// outermost continuing beyond; across interior edge R_e = e dR the value passes
// from v[e-1] to v[e] along S(x) = x^2 (3 - 2x), x = (r - R_e + w)/(2w), over
// [R_e - w, R_e + w].  Same operations, in the same order, as the definition.
__device__ __forceinline__ void shell_value(const DevParams &p, const double *v, double r, double *val,
                                            double *dval)
{
    const int n = (int)p.n_shells;
    const double R_edge = (p.R_ts > 0.0) ? p.R_ts : p.R_out;
    const double dR = R_edge / n;
    const double w = p.shell_w;
    int k = (int)floor(r / dR);
    if (k > n - 1) k = n - 1;
    if (k < 0) k = 0;
    int lo = -1;
    if (k >= 1 && r < k * dR + w) lo = k - 1;
    else if (k + 1 <= n - 1 && r > (k + 1) * dR - w) lo = k;
    if (lo < 0) {
        *val = v[k];
        *dval = 0.0;
        return;
    }
    const double x = (r - ((lo + 1) * dR - w)) / (2.0 * w);
    const double S = x * x * (3.0 - 2.0 * x);
    const double dS = 6.0 * x * (1.0 - x) / (2.0 * w);
    *val = v[lo] + (v[lo + 1] - v[lo]) * S;
    *dval = (v[lo + 1] - v[lo]) * dS;
}

// Nose-squashed heliosphere (Sec. II.B): surfaces are spheroids about the nose
// axis with the Sun on the axis (nose distance R, tail R t, flank semi-axis R f).
// mu = cosine of the angle between the point's direction and the nose.
__device__ __forceinline__ double nose_mu(const DevParams &p, double th, double ph, double *dmu_dth,
                                          double *dmu_dph)
{
    double st, ct, sn, cn, sd, cd;
    dm::sincos(th, &st, &ct);
    dm::sincos(p.nose_th, &sn, &cn);
    dm::sincos(ph - p.nose_ph, &sd, &cd);
    if (dmu_dth) *dmu_dth = ct * sn * cd - st * cn;
    if (dmu_dph) *dmu_dph = -st * sn * sd;
    return st * sn * cd + ct * cn;
}

// Distance from the Sun to the spheroid along mu and dR/dmu (positive root of
// A R^2 + 2 B R + C = 0, in the cancellation-free form R = -C / (B + sqrt(B^2 - A C))).
__device__ __forceinline__ double spheroid_radius(double R, double t, double f, double mu, double *dR_dmu)
{
    const double a = R * (1.0 + t) / 2.0, b = R * f, c = R * (t - 1.0) / 2.0;
    const double A = mu * mu / (a * a) + (1.0 - mu * mu) / (b * b);
    const double B = mu * c / (a * a);
    const double C = c * c / (a * a) - 1.0;
    const double Rm = -C / (B + sqrt(B * B - A * C));
    if (dR_dmu) {
        const double dF_dmu = Rm * Rm * mu * (1.0 / (a * a) - 1.0 / (b * b)) + Rm * c / (a * a);
        *dR_dmu = -dF_dmu / (A * Rm + B);
    }
    return Rm;
}

// Outer boundary: r >= R_out, or outside the squashed outer spheroid.
__device__ __forceinline__ bool outside(const DevParams &p, double r, double th, double ph)
{
    if (p.squashed == 0.0) return r >= p.R_out;
    const double mu = nose_mu(p, th, ph, nullptr, nullptr);
    const double a = p.R_out * (1.0 + p.hp_tail) / 2.0, b = p.R_out * p.hp_flank;
    const double c = p.R_out * (p.hp_tail - 1.0) / 2.0;
    const double xa = r * mu + c;
    return xa * xa / (a * a) + r * r * (1.0 - mu * mu) / (b * b) >= 1.0;
}

__device__ __forceinline__ void eval(const DevParams &p, const DevSpecies &sp, double r, double th,
                                     double ph, double lnP, Coef &c)
{
    double sin_th, cos_th;
    dm::sincos(th, &sin_th, &cos_th);
    const double cot_th = cos_th / sin_th;

    const double P = dm::exp(lnP);
    const double aoz = sp.A / fabs(sp.Z);
    const double pn = P / aoz;
    const double beta = pn / sqrt(pn * pn + sp.m0 * sp.m0);
    c.P = P;
    c.beta = beta;

    wind(p, th, &c.V, &c.dV_dth);

    double g, dg_dr, dg_dth = 0.0, dg_dph = 0.0;
    if (p.R_ts > 0.0 && p.squashed != 0.0) {
        double dmu_dth, dmu_dph, dR_dmu;
        const double mu = nose_mu(p, th, ph, &dmu_dth, &dmu_dph);
        const double Rts = spheroid_radius(p.R_ts, p.ts_tail, p.ts_flank, mu, &dR_dmu);
        const double t = dm::tanh((r - Rts) / p.dts);
        const double sech2 = 1.0 - t * t;
        g = 1.0 - (1.0 - p.ts_f) * 0.5 * (1.0 + t);
        dg_dr = -(1.0 - p.ts_f) * 0.5 * sech2 / p.dts;
        dg_dth = (1.0 - p.ts_f) * 0.5 * sech2 / p.dts * dR_dmu * dmu_dth;
        dg_dph = (1.0 - p.ts_f) * 0.5 * sech2 / p.dts * dR_dmu * dmu_dph;
    } else if (p.R_ts > 0.0) {
        const double t = dm::tanh((r - p.R_ts) / p.dts);
        g = 1.0 - (1.0 - p.ts_f) * 0.5 * (1.0 + t);
        dg_dr = -(1.0 - p.ts_f) * 0.5 * (1.0 - t * t) / p.dts;
    } else {
        g = 1.0;
        dg_dr = 0.0;
    }

    // the shell holding r sets K0 and the sheet tilt
    double K0 = p.K0, dK0_dr = 0.0, tilt = p.tilt_deg, dtilt_dr = 0.0;
    if (p.n_shells > 0.0) {
        shell_value(p, p.shell_K0, r, &K0, &dK0_dr);
        shell_value(p, p.shell_tilt_deg, r, &tilt, &dtilt_dr);
    }
    const double Kbase = K0 * beta * P;
    const double Kpar = Kbase * g;
    double dKpar_dr = Kbase * dg_dr;
    if (p.n_shells > 0.0) dKpar_dr = dKpar_dr + dK0_dr * beta * P * g;
    const double dKpar_dth = Kbase * dg_dth;
    const double dKpar_dph = Kbase * dg_dph;
    c.Kpar = Kpar;

    // tensor components and the derivatives the drift needs; K_rth = K_thph = 0
    double K00, K11, K22, K02 = 0.0, K01 = 0.0, K12 = 0.0;
    double Kr00, Kr02 = 0.0, Kr01 = 0.0;
    double Kt11, Kt01 = 0.0, Kt12 = 0.0;
    double Kp02 = 0.0, Kp12 = 0.0, Kp22;   // d/dph (a squashed shock makes K depend on ph)
    c.Gam = 0.0;
    c.dGam_dth = 0.0;
    if (p.isotropic != 0.0) {
        K00 = Kpar; K11 = Kpar; K22 = Kpar;
        Kr00 = dKpar_dr;
        Kt11 = dKpar_dth;
        Kp22 = dKpar_dph;
    } else {
        const double Omega = kTwoPi / p.rot_period;
        const double Gam = Omega * r * sin_th / c.V;
        const double dGam_dr = Gam / r;
        const double dGam_dth = Gam * (cot_th - c.dV_dth / c.V);
        c.Gam = Gam;
        c.dGam_dth = dGam_dth;
        const double G = Gam, G2 = G * G, one_G2 = 1.0 + G2;
        const double c2 = 1.0 / one_G2;
        const double s2 = G2 / one_G2;
        const double sc = G / one_G2;
        const double dc2_dr = -2.0 * G * dGam_dr / (one_G2 * one_G2);
        const double ds2_dr = -dc2_dr;
        const double dsc_dr = dGam_dr * (1.0 - G2) / (one_G2 * one_G2);
        const double er = p.er, et = p.et;
        const double Kpr = er * Kpar, Kpt = et * Kpar;
        const double dKpr_dr = er * dKpar_dr;
        const double dKpt_dth = et * dKpar_dth;
        K00 = Kpar * c2 + Kpr * s2;
        K22 = Kpar * s2 + Kpr * c2;
        K02 = (Kpr - Kpar) * sc;
        K11 = Kpt;
        Kr00 = dKpar_dr * c2 + Kpar * dc2_dr + dKpr_dr * s2 + Kpr * ds2_dr;
        Kr02 = (dKpr_dr - dKpar_dr) * sc + (Kpr - Kpar) * dsc_dr;
        Kt11 = dKpt_dth;
        const double dKpr_dph = er * dKpar_dph;
        Kp02 = (dKpr_dph - dKpar_dph) * sc;
        Kp22 = dKpar_dph * s2 + dKpr_dph * c2;
    }
    c.K00 = K00; c.K11 = K11; c.K22 = K22; c.K02 = K02;
    c.dKrr_dr = Kr00; c.dKrp_dr = Kr02;

    // Ito drift A^i = (1/sqrt g) d_j (sqrt g K^ij)
    c.Ar = Kr00 + 2.0 * K00 / r + Kt01 / r + K01 * cot_th / r;
    c.Ath = (Kt11 + K11 * cot_th) / (r * r) + Kr01 / r + K01 / (r * r);
    c.Aph = (Kr02 + K02 / r) / (r * sin_th) + Kt12 / (r * r * sin_th);
    if (p.squashed != 0.0) {
        c.Ar = c.Ar + Kp02 / (r * sin_th);
        c.Ath = c.Ath + Kp12 / (r * r * sin_th);
        c.Aph = c.Aph + Kp22 / (r * r * sin_th * sin_th);
    }

    // lower Cholesky factor of 2K
    {
        const double a00 = 2.0 * K00, a10 = 2.0 * K01, a11 = 2.0 * K11;
        const double a20 = 2.0 * K02, a21 = 2.0 * K12, a22 = 2.0 * K22;
        const double l00 = sqrt(a00);
        const double l10 = a10 / l00;
        const double l11 = sqrt(a11 - l10 * l10);
        const double l20 = a20 / l00;
        const double l21 = (a21 - l20 * l10) / l11;
        const double l22 = sqrt(a22 - l20 * l20 - l21 * l21);
        c.l00 = l00; c.l10 = l10; c.l11 = l11; c.l20 = l20; c.l21 = l21; c.l22 = l22;
    }

    const double B0 = (p.isotropic != 0.0) ? 0.0 : p.B0;
    c.Bmag = B0 / (r * r) * sqrt(1.0 + c.Gam * c.Gam);

    // current-sheet polarity and its gradient
    double h = 1.0, dh_dr = 0.0, dh_dth = 0.0, dh_dph = 0.0;
    c.delta_cs = 0.0;
    if (p.isotropic == 0.0 && p.hcs_on != 0.0) {
        const double Omega = kTwoPi / p.rot_period;
        double sa, ca;
        dm::sincos(tilt * kDeg, &sa, &ca);
        const double ta = sa / ca;
        const double dta_dr = (1.0 + ta * ta) * dtilt_dr * kDeg;
        const double phs = ph + Omega * r / c.V;
        const double dphs_dr = Omega / c.V;
        const double dphs_dth = -Omega * r * c.dV_dth / (c.V * c.V);
        double sp_, cp_;
        dm::sincos(phs, &sp_, &cp_);
        const double th_cs = 0.5 * kPi + dm::atan(ta * sp_);
        const double dthcs = ta * cp_ / (1.0 + ta * ta * sp_ * sp_);
        const double dthcs_dta = sp_ / (1.0 + ta * ta * sp_ * sp_);
        const double D = P * 1e9 / (kC_ms * B0 * 1e-9 * kAU_m);
        const double G = c.Gam, one_G2 = 1.0 + G * G;
        const double w_rl = 2.0 * D * r / sqrt(one_G2);
        const double dmin = p.dcs_min_deg * kDeg;
        double dd_dr = 0.0, dd_dth = 0.0, delta;
        if (w_rl > dmin) {
            delta = w_rl;
            dd_dr = 2.0 * D / (one_G2 * sqrt(one_G2));
            dd_dth = -2.0 * D * r * G * c.dGam_dth / (one_G2 * sqrt(one_G2));
        } else {
            delta = dmin;
        }
        const double u = (th_cs - th) / delta;
        h = dm::tanh(u);
        double du_dr = (dthcs * dphs_dr - u * dd_dr) / delta;
        if (p.n_shells > 0.0) du_dr = du_dr + dthcs_dta * dta_dr / delta;
        const double du_dth = (dthcs * dphs_dth - 1.0 - u * dd_dth) / delta;
        const double du_dph = dthcs / delta;
        dh_dr = (1.0 - h * h) * du_dr;
        dh_dth = (1.0 - h * h) * du_dth;
        dh_dph = (1.0 - h * h) * du_dph;
        c.delta_cs = delta;
    }
    c.h = h;

    // drift v_d = sgn(q A) curl(kappa_A h e_B)
    c.vd0 = 0.0; c.vd1 = 0.0; c.vd2 = 0.0;
    if (p.isotropic == 0.0 && p.drift_on != 0.0) {
        const double CA = beta * P * 1e9 * kDay_s / (3.0 * B0 * 1e-9 * kAU_m * kAU_m);
        const double G = c.Gam, G2 = G * G, one_G2 = 1.0 + G2;
        const double F = r * r / one_G2;
        const double Gf = r * r * G / one_G2;
        const double dF_dth = -2.0 * r * r * G * c.dGam_dth / (one_G2 * one_G2);
        const double dGf_dr = r * G * (3.0 + G2) / (one_G2 * one_G2);
        const double dGf_dth = r * r * c.dGam_dth * (1.0 - G2) / (one_G2 * one_G2);
        const double Wph = -CA * h * Gf;
        const double dWph_dth = -CA * (dh_dth * Gf + h * dGf_dth);
        const double dWph_dr = -CA * (dh_dr * Gf + h * dGf_dr);
        const double dWr_dph = CA * dh_dph * F;
        const double dWr_dth = CA * (dh_dth * F + h * dF_dth);
        const double curl_r = (cot_th * Wph + dWph_dth) / r;
        const double curl_th = (dWr_dph / sin_th - Wph - r * dWph_dr) / r;
        const double curl_ph = -dWr_dth / r;
        const double s = sgn(sp.Z) * p.polarity;
        c.vd0 = s * curl_r;
        c.vd1 = s * curl_th;
        c.vd2 = s * curl_ph;
    }

    c.dlnP = 2.0 * c.V / (3.0 * r);

    c.Ar_tot = c.Ar - c.V - c.vd0;
    if (p.dt_fixed > 0.0) {
        c.dt = p.dt_fixed;
    } else {
        double dt = p.dt_max;
        const double Krr = K00;
        const double num = p.eps_adv * 2.0 * Krr;
        const double den = c.Ar_tot * c.Ar_tot;
        if (num < dt * den) dt = num / den;
        const double t2 = p.eps_diff * r * r / Krr;
        if (t2 < dt) dt = t2;
        if (c.delta_cs > 0.0 && p.drift_on != 0.0) {
            const double rd = r * c.delta_cs;
            const double t3 = p.eps_diff * rd * rd / K11;
            if (t3 < dt) dt = t3;
        }
        if (dt < p.dt_min) dt = p.dt_min;
        c.dt = dt;
    }
}

// Three N(0,1) for step k of particle pid: Box-Muller on the four Philox
// words mapped to (0,1) as (x + 1/2) 2^-32.
__device__ __forceinline__ void normals(uint64_t seed, uint64_t pid, uint32_t k, double z[3])
{
    const uint4 w = philox_step_block(seed, pid, k);
    const double two_m32 = 2.3283064365386963e-10;
    const double u0 = ((double)w.x + 0.5) * two_m32;
    const double u1 = ((double)w.y + 0.5) * two_m32;
    const double u2 = ((double)w.z + 0.5) * two_m32;
    const double u3 = ((double)w.w + 0.5) * two_m32;
    const double rho0 = sqrt(-2.0 * dm::log(u0));
    const double rho2 = sqrt(-2.0 * dm::log(u2));
    const double a1 = kTwoPi * u1;
    const double a3 = kTwoPi * u3;
    double s1, c1, s3, c3;
    dm::sincos(a1, &s1, &c1);
    dm::sincos(a3, &s3, &c3);
    z[0] = rho0 * c1;
    z[1] = rho0 * s1;
    z[2] = rho2 * c3;
}

struct State {
    double r, th, ph, lnP, s;
    double T, Lam, r_old;      // energy form: kinetic energy per nucleon, loss integral
    uint32_t k;
    int status;
};

// Order per step: normals -> coefficients at the old state -> dt -> update
// -> reflect -> s += dt, k += 1 -> exit test.
__device__ __forceinline__ void em_step(const DevParams &p, const DevSpecies &sp, uint64_t seed,
                                        uint64_t pid, State &x)
{
    double z[3];
    x.r_old = x.r;
    normals(seed, pid, x.k, z);
    Coef c;
    eval(p, sp, x.r, x.th, x.ph, x.lnP, c);
    const double dt = c.dt;
    const double sdt = sqrt(dt);
    double sin_th, cos_th;
    dm::sincos(x.th, &sin_th, &cos_th);
    const double Lz_r = c.l00 * z[0];
    const double Lz_th = c.l10 * z[0] + c.l11 * z[1];
    const double Lz_ph = c.l20 * z[0] + c.l21 * z[1] + c.l22 * z[2];
    const double dr = (c.Ar - c.V - c.vd0) * dt + Lz_r * sdt;
    const double dth = (c.Ath - c.vd1 / x.r) * dt + Lz_th * sdt / x.r;
    const double dph = (c.Aph - c.vd2 / (x.r * sin_th)) * dt + Lz_ph * sdt / (x.r * sin_th);
    const double dlnP = c.dlnP * dt;
    x.r = x.r + dr;
    x.th = x.th + dth;
    x.ph = x.ph + dph;
    if (p.formulation != 0.0) {
        // Eq. 1 backward: A_T = (2/3)(V/r) alpha T, loss L = (2V/(3r)) (1 + beta^2)
        const double alpha = (x.T + 2.0 * sp.m0) / (x.T + sp.m0);
        const double A_T = 2.0 * c.V / (3.0 * x.r_old) * alpha * x.T;
        const double Lloss = 2.0 * c.V / (3.0 * x.r_old) * (1.0 + c.beta * c.beta);
        x.T = x.T + A_T * dt;
        x.Lam = x.Lam + Lloss * dt;
        x.lnP = dm::log(sp.A / fabs(sp.Z) * sqrt(x.T * (x.T + 2.0 * sp.m0)));
    } else {
        x.lnP = x.lnP + dlnP;
    }
    if (x.r < p.r_in) x.r = 2.0 * p.r_in - x.r;
    {
        const double t = x.th - kTwoPi * floor(x.th / kTwoPi);
        if (t > kPi) {
            x.th = kTwoPi - t;
            x.ph = x.ph + kPi;
        } else {
            x.th = t;
        }
    }
    x.ph = x.ph - kTwoPi * floor(x.ph / kTwoPi);
    x.s = x.s + dt;
    x.k = x.k + 1u;
    if (!(isfinite(x.r) && isfinite(x.th) && isfinite(x.ph) && isfinite(x.lnP) && isfinite(x.s))) {
        x.status = COSMICA_PATH_NONFINITE;
    } else if (outside(p, x.r, x.th, x.ph)) {
        x.status = COSMICA_PATH_EXIT;
    } else if ((double)x.k >= p.max_steps) {
        x.status = COSMICA_PATH_STEP_LIMIT;
    }
}

__device__ __forceinline__ void init_state(const DevSpecies &sp, double T, double r0, double th0, double ph0,
                                           State &x)
{
    x.r = r0; x.th = th0; x.ph = ph0;
    const double P0 = sp.A / fabs(sp.Z) * sqrt(T * (T + 2.0 * sp.m0));
    x.lnP = dm::log(P0);
    x.T = T;
    x.Lam = 0.0;
    x.s = 0.0;
    x.k = 0u;
    x.status = COSMICA_PATH_RUNNING;
}

}  // namespace m64
}  // namespace cosmica
