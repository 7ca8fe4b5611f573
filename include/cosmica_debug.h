/*
 * cosmica_debug.h -- probe entry points of libcosmica used by its tests.
 * They expose single pieces of the propagation path (the counter-based
 * Philox generator, the FP64 normals, the deterministic FP64 elementary
 * functions, the coefficient evaluators) so that each can be compared with
 * an independent implementation.  Same conventions as cosmica.h: device
 * pointers, stream-ordered, cosmica_status return, message via
 * cosmica_last_error().  Errors of every probe: INVALID for a NULL handle,
 * species or array (with n > 0) or an unknown function code, CUDA when the
 * launch fails; n = 0 launches nothing.
 */
#ifndef COSMICA_DEBUG_H
#define COSMICA_DEBUG_H

#include "cosmica.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Number of doubles cosmica_debug_eval writes per state:
 * V, Gamma, K_par, K_rr, K_thth, K_phph, K_rph, A^r, A^th, A^ph, L_rr, L_thth,
 * L_phr, L_phph, h, delta_cs, v_d,r, v_d,th, v_d,ph, dlnP/ds, dt. */
#define COSMICA_DEBUG_EVAL_N 21

/* Philox4x32-10 blocks (Salmon et al., SC'11): out[4i..4i+3] = Philox(ctr[4i..4i+3], (k0, k1)).
 * ctr, out: device uint32 [4 n]. */
cosmica_status cosmica_debug_philox(uint32_t n, const uint32_t *ctr, uint32_t k0, uint32_t k1,
                                    uint32_t *out, void *stream);

/* First block of cuRAND's device Philox4_32_10 after curand_init(seed, subseq[i], offset[i]).
 * subseq, offset: device uint64 [n]; out: device uint32 [4 n]. */
cosmica_status cosmica_debug_curand_philox(uint32_t n, uint64_t seed, const uint64_t *subseq,
                                           const uint64_t *offset, uint32_t *out, void *stream);

/* The FP64 step's normals for step `step` of particles pid0 .. pid0+n-1 (device double [3 n]). */
cosmica_status cosmica_debug_normals64(uint64_t seed, uint64_t pid0, uint32_t n, uint32_t step,
                                       double *z, void *stream);

/* The mixed step's FP32 normals for step `step` of particles pid0 .. pid0+n-1 (device float
 * [3 n]), built with the mixed kernels' floating-point flags; with words != NULL also the
 * Philox4x32-10 block each particle's normals come from (device uint32 [4 n]).  Box-Muller
 * on that block: u = ((x >> 9) + 1/2) 2^-23 for each word x, z0 = rho0 cos(2 pi u1),
 * z1 = rho0 sin(2 pi u1), z2 = rho2 cos(2 pi u3), rho = sqrt(-2 ln u).  INVALID also for
 * n > 2^28. */
cosmica_status cosmica_debug_normals32(uint64_t seed, uint64_t pid0, uint32_t n, uint32_t step,
                                       float *z, uint32_t *words, void *stream);

/* The FP64 step's deterministic elementary function `which` (0 exp, 1 log, 2 sin, 3 cos,
 * 4 tanh, 5 atan) on device arrays x, y of length n. */
cosmica_status cosmica_debug_fn64(int32_t which, uint32_t n, const double *x, double *y, void *stream);

/* Coefficients of one step at n states (device double [4 n]: r, th, ph, lnP) for the
 * model's parameter set and `species`; precision 0 = FP64 evaluator, 1 = FP32 evaluator.
 * out: device double [n * COSMICA_DEBUG_EVAL_N]. */
cosmica_status cosmica_debug_eval(cosmica_model *model, const cosmica_species *species, int32_t precision,
                                  uint32_t n, const double *states, double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* COSMICA_DEBUG_H */
