// k_spectrum.cu -- exit-rigidity histogram and modulated spectrum (Eq. 4).
// Built with -fmad=false so that the bin of every exit is decided by the
// same FP64 operations as its definition: b = floor((lnP / ln 10 - x_lo) / dx).
//
//   k_histogram  one thread per exit state; lanes of a warp that fall in the
//                same (item, bin) are merged with __match_any_sync and add
//                their count with one 64-bit atomic (integer, deterministic)
//   k_spectrum   one block per item: J = P0^2 (1/N) sum_b c_b w_b,
//                w_b = J_LIS(T_b) / P_b^2 at the bin's log-centre (J = f P^2 is
//                the intensity per unit kinetic energy and f is conserved along
//                a path), and sigma = std of the summand / sqrt(N); fixed-order
//                reductions
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace cosmica {

namespace {

__global__ void k_histogram(ExitPtrs ex, uint64_t n, uint32_t n_items, uint32_t nbins, double x_lo,
                            double dx, unsigned long long *__restrict__ hist)
{
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // exit states come from the caller: an entry whose item is out of range is not counted
    const bool valid = g < n && ex.item[g] < n_items;
    unsigned long long key = 0;
    if (valid) {
        const uint32_t stride = nbins + 3u;
        uint32_t slot;
        if (ex.status[g] != COSMICA_PATH_EXIT) {
            slot = nbins + 2u;
        } else {
            const double x = ex.lnP[g] / kLn10;
            const double b = floor((x - x_lo) / dx);
            if (b < 0.0) slot = 0u;
            else if (b >= (double)nbins) slot = nbins + 1u;
            else slot = 1u + (uint32_t)b;
        }
        key = (unsigned long long)ex.item[g] * stride + slot;
    }
    const unsigned active = __ballot_sync(0xffffffffu, valid);
    if (!valid) return;
    const unsigned peers = __match_any_sync(active, key);
    const unsigned lane = threadIdx.x & 31u;
    if (lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(hist + key, (unsigned long long)__popc(peers));
}

__device__ double lis_value(int kind, double T, const double *lnT, const double *lnJ, uint32_t m)
{
    if (kind == 0) return pow(T, -2.7) / (1.0 + pow(T, -3.7));
    const double x = log(T);
    if (x <= lnT[0]) return exp(lnJ[0]);
    if (x >= lnT[m - 1]) return exp(lnJ[m - 1]);
    uint32_t lo = 0, hi = m - 1;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (lnT[mid] <= x) lo = mid; else hi = mid;
    }
    const double t = (x - lnT[lo]) / (lnT[hi] - lnT[lo]);
    return exp(lnJ[lo] + t * (lnJ[hi] - lnJ[lo]));
}

template <int NT>
__device__ double block_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

constexpr int kSpecThreads = 256;

__global__ void __launch_bounds__(kSpecThreads) k_spectrum(const unsigned long long *__restrict__ hist,
                                                           uint32_t nbins, double x_lo, double dx,
                                                           const SpecItem *__restrict__ items, int lis_kind,
                                                           const double *lnT, const double *lnJ, uint32_t lis_n,
                                                           double *J, double *sigma)
{
    __shared__ double sh[kSpecThreads];
    const uint32_t e = blockIdx.x;
    const SpecItem it = items[e];
    const unsigned long long *h = hist + (size_t)e * (nbins + 3u) + 1u;
    const double zoa = fabs(it.Z) / it.A;
    // bin weight w_b = J_LIS(T_b) / P_b^2
    double cnt = 0.0, s1 = 0.0;
    for (uint32_t b = threadIdx.x; b < nbins; b += kSpecThreads) {
        const double c = (double)h[b];
        if (c == 0.0) continue;
        const double Pb = pow(10.0, x_lo + ((double)b + 0.5) * dx);
        const double pn = Pb * zoa;
        const double En = sqrt(pn * pn + it.m0 * it.m0);
        const double Tb = pn * pn / (En + it.m0);
        const double w = lis_value(lis_kind, Tb, lnT, lnJ, lis_n) / (Pb * Pb);
        cnt += c;
        s1 += c * w;
    }
    const double N = block_sum<kSpecThreads>(cnt, sh);
    const double S1 = block_sum<kSpecThreads>(s1, sh);
    const double mu = S1 / N;
    double s2 = 0.0;
    for (uint32_t b = threadIdx.x; b < nbins; b += kSpecThreads) {
        const double c = (double)h[b];
        if (c == 0.0) continue;
        const double Pb = pow(10.0, x_lo + ((double)b + 0.5) * dx);
        const double pn = Pb * zoa;
        const double En = sqrt(pn * pn + it.m0 * it.m0);
        const double Tb = pn * pn / (En + it.m0);
        const double w = lis_value(lis_kind, Tb, lnT, lnJ, lis_n) / (Pb * Pb);
        s2 += c * (w - mu) * (w - mu);
    }
    const double S2 = block_sum<kSpecThreads>(s2, sh);
    if (threadIdx.x == 0) {
        const double T0 = it.T;
        const double P0 = it.A / fabs(it.Z) * sqrt(T0 * (T0 + 2.0 * it.m0));
        const double pref = P0 * P0;
        if (N == 0.0) {
            J[e] = __longlong_as_double(0x7FF8000000000000ll);
            sigma[e] = __longlong_as_double(0x7FF8000000000000ll);
        } else {
            J[e] = pref * mu;
            sigma[e] = (N > 1.0) ? pref * sqrt(S2 / (N - 1.0) / N) : 0.0;
        }
    }
}

// Unbinned Eq. 4 over the contiguous exit states of one item per block:
//   momentum form: summand P0^2 J_LIS(T_ex) / P_ex^2
//   energy form:   summand beta0 J_LIS(T_ex) exp(lw) / beta_ex  (lw = -sum L ds)
__device__ double unbinned_summand(const SpecItem &it, int form, double lnP, double lw, int lis_kind,
                                   const double *lnT, const double *lnJ, uint32_t lis_n)
{
    const double zoa = fabs(it.Z) / it.A;
    const double P = exp(lnP);
    const double pn = P * zoa;
    const double En = sqrt(pn * pn + it.m0 * it.m0);
    const double T = pn * pn / (En + it.m0);
    const double J = lis_value(lis_kind, T, lnT, lnJ, lis_n);
    const double T0 = it.T;
    const double P0 = it.A / fabs(it.Z) * sqrt(T0 * (T0 + 2.0 * it.m0));
    if (form == 0) return P0 * P0 * J / (P * P);
    const double pn0 = P0 * zoa;
    const double b0 = pn0 / sqrt(pn0 * pn0 + it.m0 * it.m0);
    return b0 * J * exp(lw) / (pn / En);
}

__global__ void __launch_bounds__(kSpecThreads) k_spectrum_unbinned(ExitPtrs ex, const uint64_t *__restrict__ prefix,
                                                                    const SpecItem *__restrict__ items, int form,
                                                                    int lis_kind, const double *lnT, const double *lnJ,
                                                                    uint32_t lis_n, double *J, double *sigma)
{
    __shared__ double sh[kSpecThreads];
    const uint32_t e = blockIdx.x;
    const SpecItem it = items[e];
    const uint64_t lo = prefix[e], hi = prefix[e + 1];
    double cnt = 0.0, s1 = 0.0;
    for (uint64_t g = lo + threadIdx.x; g < hi; g += kSpecThreads) {
        if (ex.status[g] != COSMICA_PATH_EXIT) continue;
        s1 += unbinned_summand(it, form, ex.lnP[g], ex.lw ? ex.lw[g] : 0.0, lis_kind, lnT, lnJ, lis_n);
        cnt += 1.0;
    }
    const double N = block_sum<kSpecThreads>(cnt, sh);
    const double mu = block_sum<kSpecThreads>(s1, sh) / N;
    double s2 = 0.0;
    for (uint64_t g = lo + threadIdx.x; g < hi; g += kSpecThreads) {
        if (ex.status[g] != COSMICA_PATH_EXIT) continue;
        const double d = unbinned_summand(it, form, ex.lnP[g], ex.lw ? ex.lw[g] : 0.0, lis_kind, lnT, lnJ, lis_n) - mu;
        s2 += d * d;
    }
    const double S2 = block_sum<kSpecThreads>(s2, sh);
    if (threadIdx.x == 0) {
        if (N == 0.0) {
            J[e] = __longlong_as_double(0x7FF8000000000000ll);
            sigma[e] = __longlong_as_double(0x7FF8000000000000ll);
        } else {
            J[e] = mu;
            sigma[e] = (N > 1.0) ? sqrt(S2 / (N - 1.0) / N) : 0.0;
        }
    }
}

}  // namespace

cudaError_t launch_spectrum_unbinned(const ExitPtrs &ex, const uint64_t *prefix, uint32_t n_items,
                                     const SpecItem *items, int form, int lis_kind, const double *lis_lnT,
                                     const double *lis_lnJ, uint32_t lis_n, double *J, double *sigma, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    cudaGetLastError();
    k_spectrum_unbinned<<<n_items, kSpecThreads, 0, s>>>(ex, prefix, items, form, lis_kind, lis_lnT, lis_lnJ, lis_n,
                                                         J, sigma);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_histogram(const ExitPtrs &ex, uint64_t n, uint32_t n_items, uint32_t nbins, double x_lo,
                             double dx, unsigned long long *hist, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaGetLastError();
    k_histogram<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ex, n, n_items, nbins, x_lo, dx, hist);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_spectrum(const unsigned long long *hist, uint32_t n_items, uint32_t nbins, double x_lo,
                            double dx, const SpecItem *items, int lis_kind, const double *lis_lnT,
                            const double *lis_lnJ, uint32_t lis_n, double *J, double *sigma, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    cudaGetLastError();
    k_spectrum<<<n_items, kSpecThreads, 0, s>>>(hist, nbins, x_lo, dx, items, lis_kind, lis_lnT, lis_lnJ,
                                                lis_n, J, sigma);
    note_launch();
    return cudaGetLastError();
}

}  // namespace cosmica
