// mixed_state.cuh -- per-lane state of the mixed-precision persistent kernels
// (batched propagation and serving quanta): the particle's identity and the
// accumulated (r, theta, phi, lnP, s), either as compensated float-float
// pairs or in FP64, with the boundary handling of the step.
#pragma once
#include "common.cuh"
#include "model32.cuh"

namespace cosmica {

struct Lane {
    const float *q;            // field 0 of the particle's FP32 parameter block (see P32)
    float M2, sq;
    uint64_t pid, seed, g;
    uint32_t item, k, max_steps;
};

template <int ACC>
struct Acc;

// compensated FP32 state
template <>
struct Acc<COSMICA_PREC_MIXED> {
    m32::FF r, th, ph, lnP, s;
    m32::FF Rout;
    float r_in2;   // 2 r_in
    __device__ void init(double r0, double th0, double ph0, double lnP0, double R_out, float r_in)
    {
        r = m32::ff_from_double(r0);
        th = m32::ff_from_double(th0);
        ph = m32::ff_from_double(ph0);
        lnP = m32::ff_from_double(lnP0);
        s.hi = 0.0f; s.lo = 0.0f;
        Rout = m32::ff_from_double(R_out);
        r_in2 = 2.0f * r_in;
    }
    __device__ float fr() const { return r.hi; }
    __device__ float fth() const { return th.hi; }
    __device__ float fph() const { return ph.hi; }
    __device__ float flnP() const { return lnP.hi; }
    // distance of theta (hi + lo, in [0, pi]) to the nearer pole, to FP32 accuracy:
    // near pi it is formed from the float-float splits of pi and theta (the high
    // parts subtract exactly), so it keeps its sign and relative accuracy even
    // where the FP32 theta rounds to pi or beyond
    __device__ float pole_distance() const
    {
        if (th.hi < m32::kHalfPiF) return th.hi;
        return __fadd_rn(__fsub_rn(m32::kPiF, th.hi), __fsub_rn(m32::kPiLoF, th.lo));
    }
    __device__ float sin_th() const { return m32::sin_from_pole_distance(pole_distance()); }
    __device__ void add(float dr, float dth, float dph, float dlnP, float dt)
    {
        m32::ff_add(r, dr);
        m32::ff_add(th, dth);
        m32::ff_add(ph, dph);
        m32::ff_add(lnP, dlnP);
        m32::ff_add(s, dt);
    }
    // reflect at r_in, fold theta at the poles, wrap phi; all rare branches
    __device__ void boundaries(float r_in)
    {
        const bool fold = th.hi < 0.0f || pole_distance() < 0.0f;   // theta < 0 or theta > pi
        // one rarely taken branch for the three boundaries
        if ((r.hi < r_in) | fold | (ph.hi < 0.0f) | (ph.hi >= m32::kTwoPiF)) {
            if (r.hi < r_in) {           // r <- 2 r_in - r
                r.hi = -r.hi; r.lo = -r.lo;
                m32::ff_add(r, r_in2);
            }
            if (fold) fold_theta();
            if (ph.hi < 0.0f || ph.hi >= m32::kTwoPiF) wrap_phi();
        }
    }
    __device__ void fold_theta()
    {
        // t = th mod 2 pi in [0, 2pi); if t > pi: th = 2pi - t, ph += pi
        const double t0 = m32::ff_to_double(th);
        double t = t0 - kTwoPi * floor(t0 / kTwoPi);
        if (t > kPi) {
            t = kTwoPi - t;
            const double p = m32::ff_to_double(ph) + kPi;
            ph = m32::ff_from_double(p);
        }
        th = m32::ff_from_double(t);
    }
    __device__ void wrap_phi()
    {
        const double p0 = m32::ff_to_double(ph);
        ph = m32::ff_from_double(p0 - kTwoPi * floor(p0 / kTwoPi));
    }
    __device__ bool exited() const { return m32::ff_ge(r, Rout); }
    __device__ bool finite() const { return isfinite(r.hi + th.hi + ph.hi + lnP.hi + s.hi); }
    __device__ void write(const ExitPtrs &out, uint64_t g) const
    {
        out.r[g] = m32::ff_to_double(r);
        out.th[g] = m32::ff_to_double(th);
        out.ph[g] = m32::ff_to_double(ph);
        out.lnP[g] = m32::ff_to_double(lnP);
        out.s[g] = m32::ff_to_double(s);
    }
};

// FP64 accumulation of FP32 increments
template <>
struct Acc<COSMICA_PREC_MIXED_F64ACC> {
    double r, th, ph, lnP, s, Rout, r_in;
    __device__ void init(double r0, double th0, double ph0, double lnP0, double R_out, float r_in_f)
    {
        r = r0; th = th0; ph = ph0; lnP = lnP0; s = 0.0; Rout = R_out; r_in = (double)r_in_f;
    }
    __device__ float fr() const { return (float)r; }
    __device__ float fth() const { return (float)th; }
    __device__ float fph() const { return (float)ph; }
    __device__ float flnP() const { return (float)lnP; }
    __device__ float sin_th() const { return m32::sin_theta_f64(th); }
    __device__ void add(float dr, float dth, float dph, float dlnP, float dt)
    {
        r += (double)dr; th += (double)dth; ph += (double)dph; lnP += (double)dlnP; s += (double)dt;
    }
    __device__ void boundaries(float)
    {
        if (r < r_in) r = 2.0 * r_in - r;
        if (th < 0.0 || th > kPi) {
            double t = th - kTwoPi * floor(th / kTwoPi);
            if (t > kPi) { t = kTwoPi - t; ph += kPi; }
            th = t;
        }
        if (ph < 0.0 || ph >= kTwoPi) ph = ph - kTwoPi * floor(ph / kTwoPi);
    }
    __device__ bool exited() const { return r >= Rout; }
    __device__ bool finite() const { return isfinite(r + th + ph + lnP + s); }
    __device__ void write(const ExitPtrs &out, uint64_t g) const
    {
        out.r[g] = r; out.th[g] = th; out.ph[g] = ph; out.lnP[g] = lnP; out.s[g] = s;
    }
};


// Energy form (Eq. 1): kinetic energy per nucleon T and the loss integral
// Lam = sum L ds of Eq. 4, accumulated with the same precision as the state.
// The momentum form carries nothing.
template <int ACC, bool EN>
struct EnergyAcc {
    __device__ void init(double, float, float) {}
};

template <>
struct EnergyAcc<COSMICA_PREC_MIXED, true> {
    m32::FF T, Lam;
    float m0, aoz;
    __device__ void init(double T0, float m0_, float aoz_)
    {
        T = m32::ff_from_double(T0);
        Lam.hi = 0.0f; Lam.lo = 0.0f;
        m0 = m0_; aoz = aoz_;
    }
    __device__ float fT() const { return T.hi; }
    __device__ void add(float dT, float dLam) { m32::ff_add(T, dT); m32::ff_add(Lam, dLam); }
    __device__ double T64() const { return m32::ff_to_double(T); }
    __device__ double lw() const { return -m32::ff_to_double(Lam); }
};

template <>
struct EnergyAcc<COSMICA_PREC_MIXED_F64ACC, true> {
    double T, Lam;
    float m0, aoz;
    __device__ void init(double T0, float m0_, float aoz_) { T = T0; Lam = 0.0; m0 = m0_; aoz = aoz_; }
    __device__ float fT() const { return (float)T; }
    __device__ void add(float dT, float dLam) { T += (double)dT; Lam += (double)dLam; }
    __device__ double T64() const { return T; }
    __device__ double lw() const { return -Lam; }
};

// a lane's complete state, moved through shared memory by block compaction
template <int ACC, bool EN>
struct Packed {
    Lane L;
    Acc<ACC> x;
    EnergyAcc<ACC, EN> en;
};

}  // namespace cosmica
