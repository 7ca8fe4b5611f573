// model32.cuh -- the mixed-precision step.
//
// Coefficients, the tensor square root and the normals are evaluated in FP32
// with the SFU (MUFU) approximations of exp2/log2/sin/cos/rsqrt/rcp; the
// state r, theta, phi, lnP and s is accumulated either as float-float pairs
// (compensated FP32: TwoSum of each increment, error carried in a low word
// and renormalised) or in FP64.  The outer-boundary test is exact in both:
// a float-float value is compared lexicographically against the float-float
// split of R_out, which equals comparing the exact sum with R_out.
//
// Every fused multiply-add is written out (fmaf) and the translation units
// that include this file are built with -fmad=false, so the compiler never
// contracts differently in different inlining contexts: the step's rounding is
// the same in the batched kernel, the serving kernel and both phases of each,
// which keeps every path identical across launch shapes (the wavy current
// sheet amplifies single roundings).
//
// The model is the same reading as the FP64 step; the algebra is rearranged
// for FP32 (closed forms instead of cancelling differences):
//   (1 + tanh x)/2 = 1/(1 + e^-2x),   1 - tanh^2 x = 4 s (1 - s) with s = that logistic,
//   L_rr = sqrt(2 K_rr), L_phr = 2 K_rph / L_rr, L_phph = K_par sqrt(2 er / K_rr)
//   (det of the (r,ph) block is er K_par^2 because cos^2 + sin^2 = 1).
#pragma once
#include "common.cuh"
#include "philox.cuh"

namespace cosmica {
namespace m32 {

constexpr float kHalfPiF = 1.57079632679489662f;
constexpr float kPiF = 3.14159265358979324f;          // pi rounded to FP32 (above pi)
constexpr float kPiLoF = -8.74227766e-8f;             // pi - kPiF, rounded to FP32
constexpr float kTwoPiF = 6.28318530717958648f;
constexpr float kInvTwoPiF = 0.159154943091895336f;
constexpr float kSqrt2F = 1.41421356237309505f;

// 1/(1 + e^{-2x}) = (1 + tanh x) / 2, safe for any finite x
__device__ __forceinline__ float half_one_plus_tanh(float x)
{
    return __fdividef(1.0f, 1.0f + __expf(-2.0f * x));
}

struct Drift {
    float Ar_tot;      // radial drift of the SDE, A^r - V - v_d,r   [AU/day]
    float dth_drift;   // d theta / ds                                [1/day]
    float dph_drift;   // d phi / ds                                  [1/day]
    float l00, l11, l20, l22;
    float inv_r, inv_rs;
    float dlnP, dt;
    float beta;        // speed / c at the start of the step
};

// Radial shells (Sec. II.B): the shells a, b whose values blend at r and the
// smoothstep weight S(x) = x^2 (3 - 2x) with its radial derivative; a = b and
// S = 0 away from the edge windows, so v[a] + (v[b] - v[a]) S is the shell's value.
template <uint32_t ST>
__device__ __forceinline__ void shell_weights(const P32<ST> &q, float r, int &a, int &b, float &S, float &dS)
{
    const int n = (int)P32F(q, n_sh);
    const int k = min(max((int)(r * P32F(q, sh_inv_dr)), 0), n - 1);
    float x = 0.0f;
    a = k;
    b = k;
    const float lo_edge = (float)k * P32F(q, sh_dr);
    const float hi_edge = (float)(k + 1) * P32F(q, sh_dr);
    if (k >= 1 && r < lo_edge + P32F(q, sh_w)) {
        a = k - 1;
        x = (r - (lo_edge - P32F(q, sh_w))) * P32F(q, sh_inv_2w);
    } else if (k + 1 <= n - 1 && r > hi_edge - P32F(q, sh_w)) {
        b = k + 1;
        x = (r - (hi_edge - P32F(q, sh_w))) * P32F(q, sh_inv_2w);
    }
    S = x * x * fmaf(-2.0f, x, 3.0f);
    dS = 6.0f * x * (1.0f - x) * P32F(q, sh_inv_2w);
}

// Coefficients at (r, th, ph, lnP).  q: FP32 constants of the heliosphere (read through P32).
// M2 = (A/|Z| m0)^2, sq = sign of the charge.
// Nose-squashed spheroid (Sec. II.B) in FP32: distance R from the Sun along
// the direction mu and dR/dmu; ia2 = 1/a^2, ib2 = 1/b^2, c = centre offset,
// C = c^2/a^2 - 1 (the positive root of A R^2 + 2 B R + C = 0).
__device__ __forceinline__ float spheroid_radius(float ia2, float ib2, float c, float C, float mu, float &dR_dmu)
{
    const float mu2 = mu * mu;
    const float A = fmaf(mu2, ia2 - ib2, ib2);
    const float B = mu * c * ia2;
    const float Rm = __fdividef(-C, B + sqrtf(fmaf(B, B, -A * C)));
    dR_dmu = -__fdividef(Rm * fmaf(Rm * mu, ia2 - ib2, c * ia2), fmaf(A, Rm, B));
    return Rm;
}

// cos of the angle between the direction (th, ph) and the nose, with its derivatives
template <uint32_t ST>
__device__ __forceinline__ float nose_mu(const P32<ST> &q, float sn, float cs, float ph, float &dmu_dth,
                                         float &dmu_dph)
{
    float d = ph - P32F(q, nose_ph);                      // nose_ph in [0, 2 pi): d in (-2 pi, 2 pi)
    d = (d > kPiF) ? d - kTwoPiF : ((d < -kPiF) ? d + kTwoPiF : d);
    float sd, cd;
    __sincosf(d, &sd, &cd);
    dmu_dth = fmaf(cs * P32F(q, sin_nth), cd, -sn * P32F(q, cos_nth));
    dmu_dph = -sn * P32F(q, sin_nth) * sd;
    return fmaf(sn * P32F(q, sin_nth), cd, cs * P32F(q, cos_nth));
}

// Outside the squashed outer spheroid (FP32; the spherical boundary keeps its exact test).
template <uint32_t ST>
__device__ __forceinline__ bool outside_squashed(const P32<ST> &q, float r, float th, float ph)
{
    float sn, cs, dth, dph;
    __sincosf(th, &sn, &cs);
    const float mu = nose_mu(q, sn, cs, ph, dth, dph);
    const float xa = fmaf(r, mu, P32F(q, hp_c));
    const float rp2 = r * r * fmaf(-mu, mu, 1.0f);
    return fmaf(xa * xa, P32F(q, hp_ia2), rp2 * P32F(q, hp_ib2)) >= 1.0f;
}

// sin(theta) from the distance d to the nearer pole (d >= 0, exact to FP32).  The
// SFU sine has an absolute, not a relative, error bound, so near a pole it can
// return 0 (and 1/sin theta = inf): below d = 0.1 a Taylor polynomial is used,
// d (1 - d^2/6 (1 - d^2/20)), whose truncation error is below 2e-11 relative.
__device__ __forceinline__ float sin_from_pole_distance(float d)
{
    const float d2 = d * d;
    const float taylor = d * fmaf(-d2 * 0.16666667f, fmaf(-d2, 0.05f, 1.0f), 1.0f);
    return d < 0.1f ? taylor : __sinf(d);
}

// The same for a theta given in FP64 (the debug evaluator, FP64-accumulated states).
__device__ __forceinline__ float sin_theta_f64(double th)
{
    const double d = th < 0.5 * kPi ? th : kPi - th;
    return sin_from_pole_distance((float)d);
}

// EXT: the parameter sets of the launch may have radial shells or a squashed
// heliosphere (compile-time, so that launches of the basic model carry none of
// that code or its registers).  FULL: every set of the launch is the full model
// (drift and current sheet on, adaptive step); the uniform branches on those
// switches then vanish and the step is one long branch-free block, which the
// compiler schedules with more instruction-level parallelism (the latency of a
// lone path is what bounds the end of a launch).
// sin_th: sin(theta) accurate relative to itself near the poles (the caller derives
// it from the compensated state, see sin_from_pole_distance); cos theta is taken
// from the SFU, whose absolute error is harmless in cot theta.
template <bool EXT, bool FULL, uint32_t ST>
__device__ __forceinline__ void eval(const P32<ST> &q, float M2, float sq, float r, float th, float sin_th,
                                     float ph, float lnP, Drift &o, float *dbg = nullptr)
{
    const float P = __expf(lnP);
    const float beta = P * rsqrtf(fmaf(P, P, M2));
    o.beta = beta;
    const float sn = sin_th;
    const float cs = __cosf(th);
    const float inv_sn = __fdividef(1.0f, sn);
    const float cot = cs * inv_sn;
    const float inv_r = __fdividef(1.0f, r);

    // wind V(th) and dV/dth
    const float lat = kHalfPiF - th;
    const float sw = half_one_plus_tanh((fabsf(lat) - P32F(q, lat_f)) * P32F(q, inv_dlat));
    const float V = fmaf(P32F(q, dV), sw, P32F(q, Vs));
    const float sgn_lat = (lat > 0.0f) ? -1.0f : ((lat < 0.0f) ? 1.0f : 0.0f);   // d|lat|/dth
    const float dV = P32F(q, dV) * 2.0f * sw * (1.0f - sw) * P32F(q, inv_dlat) * sgn_lat;
    const float inv_V = __fdividef(1.0f, V);

    // Parker spiral
    const float Gam = P32F(q, Omega) * r * sn * inv_V;
    const float G2 = Gam * Gam;
    const float iq = __fdividef(1.0f, fmaf(Gam, Gam, 1.0f));
    const float dGam_dth = Gam * fmaf(-dV, inv_V, cot);

    // termination shock factor (uniform branch: no shock in the parameter set); a
    // squashed shock sits at its spheroid's distance along the point's direction.  The
    // full-model variant evaluates it without the branch: with ts_drop = 0 it gives g = 1
    // and dg = -0 exactly, which leave every later value as the branch would (measured:
    // +2.6 % steps/s on config 3, +2.4 % on config 2, which has no shock)
    float g = 1.0f, dg = 0.0f, dg_dth = 0.0f, dg_dph = 0.0f;
    const bool squashed = EXT && P32F(q, sq) != 0.0f;
    if (FULL || P32F(q, ts_drop) != 0.0f) {
        float Rts = P32F(q, R_ts), dR_dmu = 0.0f, dmu_dth = 0.0f, dmu_dph = 0.0f;
        if (squashed) {
            const float mu = nose_mu(q, sn, cs, ph, dmu_dth, dmu_dph);
            Rts = P32F(q, ts_R) * spheroid_radius(P32F(q, ts_ia2), P32F(q, ts_ib2), P32F(q, ts_c), P32F(q, ts_C), mu, dR_dmu);
            dR_dmu *= P32F(q, ts_R);
        }
        const float st = half_one_plus_tanh((r - Rts) * P32F(q, inv_dts));
        g = fmaf(-P32F(q, ts_drop), st, 1.0f);
        const float w = P32F(q, ts_drop) * 2.0f * st * (1.0f - st) * P32F(q, inv_dts);
        dg = -w;
        if (squashed) {
            dg_dth = w * dR_dmu * dmu_dth;
            dg_dph = w * dR_dmu * dmu_dph;
        }
    }

    // radial shells: K0 and the sheet tilt of the shell holding r (the single-region
    // tilt is read where the sheet needs it, so that it is not live before)
    const bool shells = EXT && P32F(q, n_sh) != 0.0f;
    float K0 = P32F(q, K0), dK0 = 0.0f, sh_ta = 0.0f, sh_ta2 = 0.0f, dta = 0.0f;
    if (shells) {
        int a, b;
        float S, dS;
        shell_weights(q, r, a, b, S, dS);
        const float Ka = P32A(q, sh_K0, a), dKab = P32A(q, sh_K0, b) - Ka;
        K0 = fmaf(dKab, S, Ka);
        dK0 = dKab * dS;
        const float al = P32A(q, sh_alpha, a), dal = P32A(q, sh_alpha, b) - al;
        float sa, ca;
        __sincosf(fmaf(dal, S, al), &sa, &ca);
        sh_ta = __fdividef(sa, ca);
        sh_ta2 = sh_ta * sh_ta;
        dta = fmaf(sh_ta, sh_ta, 1.0f) * dal * dS;
    }

    // diffusion tensor in (r, th, ph); K_rth = K_thph = 0
    const float Kb = K0 * beta * P;
    const float Kpar = Kb * g;
    float dKpar = Kb * dg;
    if (shells) dKpar = fmaf(dK0 * beta * P, g, dKpar);
    const float c2s = fmaf(P32F(q, er), G2 * iq, iq);            // cos^2 + er sin^2
    const float iq2 = iq * iq;
    const float dc2_dr = -2.0f * G2 * iq2 * inv_r;         // d cos^2 psi / dr
    const float sc = Gam * iq;
    const float dsc_dr = Gam * (1.0f - G2) * iq2 * inv_r;
    const float Krr = Kpar * c2s;
    const float erm1 = P32F(q, er) - 1.0f;
    const float Krp = erm1 * Kpar * sc;
    const float Ktt = P32F(q, et) * Kpar;
    const float dKrr = fmaf(dKpar, c2s, -Kpar * erm1 * dc2_dr);
    const float dKrp = erm1 * fmaf(dKpar, sc, Kpar * dsc_dr);

    // Ito drift (1/sqrt g) d_j (sqrt g K^ij)
    float Ar = fmaf(2.0f * Krr, inv_r, dKrr);
    float Ath = Ktt * cot * inv_r * inv_r;
    const float inv_rs = inv_r * inv_sn;
    float Aph = fmaf(Krp, inv_r, dKrp) * inv_rs;
    if (squashed) {
        // K depends on th and ph through the squashed shock: d_th K_thth / r^2,
        // d_ph K_rph / (r sin th) and d_ph K_phph / (r sin th)^2
        const float dKpar_th = Kb * dg_dth, dKpar_ph = Kb * dg_dph;
        Ath = fmaf(P32F(q, et) * dKpar_th, inv_r * inv_r, Ath);
        Ar = fmaf(erm1 * dKpar_ph * sc, inv_rs, Ar);
        Aph = fmaf(dKpar_ph * fmaf(P32F(q, er), iq, G2 * iq), inv_rs * inv_rs, Aph);
    }

    // Cholesky factor of 2K
    const float rK = rsqrtf(Krr);
    o.l00 = kSqrt2F * Krr * rK;
    o.l20 = kSqrt2F * Krp * rK;
    o.l22 = P32F(q, sqrt2er) * Kpar * rK;
    o.l11 = sqrtf(2.0f * Ktt);

    // drift v_d = sgn(qA) curl(kappa_A h e_B)
    float vd0 = 0.0f, vd1 = 0.0f, vd2 = 0.0f, delta = 0.0f, h = 1.0f;
    if (FULL || P32F(q, drift) != 0.0f) {
        const float r2 = r * r;
        const float F = r2 * iq;
        const float Gf = F * Gam;
        const float dF_dth = -2.0f * r2 * Gam * dGam_dth * iq2;
        const float dGf_dr = r * Gam * (3.0f + G2) * iq2;
        const float dGf_dth = r2 * dGam_dth * (1.0f - G2) * iq2;
        float hr = 0.0f, ht = 0.0f, hp = 0.0f;
        if (FULL || P32F(q, hcs) != 0.0f) {
            const float phs = fmaf(P32F(q, Omega) * r, inv_V, ph);
            const float dphs_dr = P32F(q, Omega) * inv_V;
            const float dphs_dth = -P32F(q, Omega) * r * dV * inv_V * inv_V;
            // nearest integer by the 1.5 2^23 shift (|phs| / 2 pi < 2^22): two FADDs
            const float turns = __fsub_rn(__fadd_rn(phs * kInvTwoPiF, 12582912.0f), 12582912.0f);
            const float red = fmaf(-kTwoPiF, turns, phs);
            float sp, cp;
            __sincosf(red, &sp, &cp);
            const float ta = shells ? sh_ta : P32F(q, ta);
            const float ta2 = shells ? sh_ta2 : P32F(q, ta2);
            const float th_cs = kHalfPiF + atanf(ta * sp);
            const float inv_den = __fdividef(1.0f, fmaf(ta2, sp * sp, 1.0f));
            const float dthcs = (ta * cp) * inv_den;
            const float sqiq = sqrtf(iq);
            const float w_rl = P32F(q, D2) * P * r * sqiq;
            // half-width max(2 r_L / r, floor) and its derivatives, by selects (no branch)
            const bool rl = w_rl > P32F(q, dcs_min);
            const float k3 = P32F(q, D2) * P * iq * sqiq;
            delta = rl ? w_rl : P32F(q, dcs_min);
            const float dd_dr = rl ? k3 : 0.0f;
            const float dd_dth = rl ? -k3 * r * Gam * dGam_dth : 0.0f;
            const float inv_d = __fdividef(1.0f, delta);
            const float u = (th_cs - th) * inv_d;
            const float sh = half_one_plus_tanh(u);
            h = fmaf(2.0f, sh, -1.0f);
            const float sech2 = 4.0f * sh * (1.0f - sh);
            float ur = fmaf(dthcs, dphs_dr, -u * dd_dr);
            if (shells) ur = fmaf(sp * inv_den, dta, ur);    // the tilt changes with r
            hr = sech2 * ur * inv_d;
            ht = sech2 * fmaf(-u, dd_dth, fmaf(dthcs, dphs_dth, -1.0f)) * inv_d;
            hp = sech2 * dthcs * inv_d;
        }
        const float s = sq * P32F(q, polarity) * P32F(q, CA0) * beta * P * inv_r;
        const float Wph = -h * Gf;                       // W_ph / C_A
        const float dWph_dth = -fmaf(ht, Gf, h * dGf_dth);
        const float dWph_dr = -fmaf(hr, Gf, h * dGf_dr);
        vd0 = s * fmaf(cot, Wph, dWph_dth);
        vd1 = s * fmaf(-r, dWph_dr, fmaf(hp * F, inv_sn, -Wph));
        vd2 = -s * fmaf(ht, F, h * dF_dth);
    }

    const float Ar_tot = Ar - V - vd0;
    o.Ar_tot = Ar_tot;
    o.dth_drift = fmaf(-vd1, inv_r, Ath);
    o.dph_drift = fmaf(-vd2, inv_rs, Aph);
    o.inv_r = inv_r;
    o.inv_rs = inv_rs;
    o.dlnP = 0.66666666666666667f * V * inv_r;

    // step length
    float dt;
    if (!FULL && P32F(q, dt_fixed) > 0.0f) {
        dt = P32F(q, dt_fixed);
    } else {
        const float t1 = __fdividef(P32F(q, eps_adv2) * Krr, Ar_tot * Ar_tot);
        const float t2 = __fdividef(P32F(q, eps_diff) * r * r, Krr);
        dt = fminf(P32F(q, dt_max), fminf(t1, t2));
        if (FULL || delta > 0.0f) {
            const float rd = r * delta;
            dt = fminf(dt, __fdividef(P32F(q, eps_diff) * rd * rd, Ktt));
        }
        dt = fmaxf(dt, P32F(q, dt_min));
    }
    o.dt = dt;
    if (dbg) {
        dbg[0] = V; dbg[1] = Gam; dbg[2] = Kpar; dbg[3] = Krr; dbg[4] = Ktt; dbg[5] = Kpar * fmaf(G2, iq, P32F(q, er) * iq);
        dbg[6] = Krp; dbg[7] = Ar; dbg[8] = Ath; dbg[9] = Aph; dbg[10] = o.l00; dbg[11] = o.l11;
        dbg[12] = o.l20; dbg[13] = o.l22; dbg[14] = h; dbg[15] = delta;
        dbg[16] = vd0; dbg[17] = vd1; dbg[18] = vd2; dbg[19] = o.dlnP; dbg[20] = dt;
    }
}

// A Philox word mapped to (0,1) as ((x >> 9) + 1/2) 2^-23, exactly: the top 23
// bits become the mantissa of a float in [1,2), then 1 - 2^-24 is subtracted.
__device__ __forceinline__ float uniform01(uint32_t x)
{
    return __fsub_rn(__uint_as_float(0x3F800000u | (x >> 9)), 0.99999994039535522f);
}

// Three N(0,1) in FP32: Box-Muller on the four Philox words.
__device__ __forceinline__ void normals(uint64_t seed, uint64_t pid, uint32_t k, float &z0, float &z1,
                                        float &z2)
{
    const uint4 w = philox_step_block(seed, pid, k);
    const float u0 = uniform01(w.x);
    const float u1 = uniform01(w.y);
    const float u2 = uniform01(w.z);
    const float u3 = uniform01(w.w);
    const float rho0 = sqrtf(-2.0f * __logf(u0));
    const float rho2 = sqrtf(-2.0f * __logf(u2));
    // angle 2 pi u - pi lies in (-pi, pi], where the SFU sin/cos are accurate;
    // cos(a - pi) = -cos a, sin(a - pi) = -sin a
    float s1, c1, s3, c3;
    __sincosf(fmaf(u1, kTwoPiF, -kPiF), &s1, &c1);
    __sincosf(fmaf(u3, kTwoPiF, -kPiF), &s3, &c3);
    z0 = -rho0 * c1;
    z1 = -rho0 * s1;
    z2 = -rho2 * c3;
}

// ---- compensated FP32 accumulation ---------------------------------------
struct FF {
    float hi, lo;
};

// (hi, lo) += d: TwoSum of hi + d, error carried into lo, then renormalised
// so that |lo| <= ulp(hi)/2.
// (the _rn intrinsics keep every rounding exactly as written)
__device__ __forceinline__ void ff_add(FF &a, float d)
{
    const float s = __fadd_rn(a.hi, d);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(d, bb));
    const float lo = __fadd_rn(a.lo, err);
    const float hi = __fadd_rn(s, lo);
    a.lo = __fsub_rn(lo, __fsub_rn(hi, s));
    a.hi = hi;
}

__device__ __forceinline__ void ff_add_ff(FF &a, float bh, float bl)
{
    ff_add(a, bh);
    ff_add(a, bl);
}

__device__ __forceinline__ FF ff_from_double(double x)
{
    FF r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}

__device__ __forceinline__ double ff_to_double(const FF &a) { return (double)a.hi + (double)a.lo; }

// exact test a >= b for normalised float-float values
__device__ __forceinline__ bool ff_ge(const FF &a, const FF &b)
{
    return (a.hi > b.hi) || (a.hi == b.hi && a.lo >= b.lo);
}

__device__ __forceinline__ bool ff_lt(const FF &a, const FF &b) { return !ff_ge(a, b); }

}  // namespace m32
}  // namespace cosmica
