/*
 * cosmica.h -- C ABI of libcosmica, a GB300 (sm_103a) implementation of the
 * hot path of COSMICA (Cavallotto, Della Torre, La Vacca, Gervasi,
 * arXiv 2502.06319): backward-in-time Euler-Maruyama integration of the
 * Parker-transport SDEs in momentum form, one GPU thread per quasi-particle,
 * followed by binning of the exit rigidities and the LIS-weighted spectrum.
 *
 * Conventions shared by every entry point
 *   - Ownership: the caller owns every input and output buffer.  The library
 *     owns only the opaque handles it returns (model, batch, server) and the
 *     device scratch inside them.
 *   - Memory: arguments documented "device" must be device pointers of the
 *     current CUDA device; "host" arguments are ordinary host memory.  The
 *     exit-state buffers of cosmica_propagate / cosmica_batch_run may be host
 *     memory too (pinned or pageable): the library then stages through its
 *     own device scratch and copies the result back on the stream.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *     Calls are stream-ordered and do not synchronise the host, except
 *     where a host output is requested (then they synchronise the stream).
 *   - Errors: every call returns a cosmica_status; on failure a thread-local
 *     message is available from cosmica_last_error().  No call aborts, traps
 *     or spins without bound: the only loops on the device are the particle
 *     step loops, each bounded by cosmica_params.max_steps.
 *   - Particle identity: quasi-particle i of a work item has pid =
 *     first_pid + i.  Its Philox stream is keyed by (seed, pid, step) only, so
 *     results do not depend on batching, ordering or launch shape.
 *   - Threads: a model or batch handle holds per-call scratch, so calls on one
 *     handle must not overlap in time (serialise them, or give each thread
 *     its own handle); calls on different handles may run concurrently.  A
 *     server handle may be used from any number of threads (cosmica_server_destroy
 *     excepted: no other call on it may be in progress).  Consecutive
 *     calls on one handle on different streams must be ordered by the caller
 *     (an event or a synchronisation): the later call reuses the handle's
 *     device scratch that the earlier call's kernels may still read.  On one
 *     stream they are ordered already.
 */
#ifndef COSMICA_H
#define COSMICA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define COSMICA_ABI_VERSION 1u
#define COSMICA_MAX_SHELLS 16u

typedef enum {
    COSMICA_OK = 0,
    COSMICA_ERR_INVALID = 1,   /* bad argument; nothing was launched            */
    COSMICA_ERR_OOM = 2,       /* a device or pinned allocation failed          */
    COSMICA_ERR_CUDA = 3,      /* a CUDA runtime call or launch failed          */
    COSMICA_ERR_TIMEOUT = 4,   /* a bounded host wait ran out                   */
    COSMICA_ERR_BUSY = 5       /* result not ready yet (server poll)            */
} cosmica_status;

/* Arithmetic of the step. */
enum {
    COSMICA_PREC_FP64 = 0,        /* FP64 everywhere; built without FMA contraction
                                     and with deterministic elementary functions  */
    COSMICA_PREC_MIXED = 1,       /* FP32 coefficients, tensor root and normals;
                                     compensated FP32 (float-float) accumulation of
                                     r, theta, phi, lnP, s; exact boundary test  */
    COSMICA_PREC_MIXED_F64ACC = 2 /* FP32 coefficients; FP64 accumulation and test */
};

/* Per-path status in cosmica_exit_states.status. */
enum {
    COSMICA_PATH_RUNNING = 0,
    COSMICA_PATH_EXIT = 1,        /* crossed the outer boundary r >= R_out      */
    COSMICA_PATH_STEP_LIMIT = 2,  /* reached max_steps                          */
    COSMICA_PATH_NONFINITE = 3    /* the state became NaN / Inf                 */
};

/*
 * Heliospheric model and integration parameters (Sec. II.B: inner heliosphere
 * with a Parker-spiral field and latitude-dependent wind; the termination
 * shock separates the heliosheath).  The paper defers the SDE coefficients to
 * another publication; the library implements this reading:
 *   wind    V(th) = Vs + (Vf-Vs) (1 + tanh((|lat| - lat_fast)/dlat)) / 2, radial
 *   field   B = A h B0 (1 AU/r)^2 (e_r - Gamma e_ph), Gamma = Omega r sin(th)/V,
 *           B0 chosen so that |B|(1 AU, equator) = B1AU_nT
 *   K       K_par = K0 beta P[GV] g(r) along b, K_perp,r = kperp_r_frac K_par,
 *           K_perp,th = kperp_th_frac K_par; g = 1 - (1-ts_K_factor)(1+tanh((r-R_ts)/dts))/2
 *   drift   v_d = sgn(q A) curl(kappa_A h e_B), kappa_A = beta P / (3 |B|),
 *           h = tanh((th_cs - th)/delta), th_cs = pi/2 + atan(tan(tilt) sin(ph + Omega r/V)),
 *           delta = max(2 r_L / r, dcs_min)
 *   SDE     (Eq. 3, Eq. 5, Eq. 6) dx = (div K - V - v_d) ds + sqrt(2K) dW,
 *           d lnP = 2V/(3r) ds, Euler-Maruyama, backward time s [day]
 *   dt      dt_fixed if > 0, else min(dt_max, eps_adv 2K_rr/A_r^2, eps_diff r^2/K_rr,
 *           eps_diff (r delta)^2/K_th) floored at dt_min (the advective step
 *           is kept small against the diffusive one, Sec. IV.A)
 *   bounds  absorbing at r >= R_out, reflecting at r_in, theta folded at the poles
 * isotropic != 0 selects the spherically symmetric 1-D model of Sec. IV.B:
 *   K = K0 beta P times the identity, uniform wind V_const_kms, no drift.
 * Fill with cosmica_params_default() and override; struct_size and version
 * guard the ABI.
 */
typedef struct {
    uint32_t struct_size;      /* = sizeof(cosmica_params)                 */
    uint32_t version;          /* = COSMICA_ABI_VERSION                    */
    double K0;                 /* AU^2/day                                 */
    double kperp_r_frac;
    double kperp_th_frac;
    double B1AU_nT;
    double V_slow_kms;
    double V_fast_kms;
    double lat_fast_deg;
    double tilt_deg;
    int32_t polarity;          /* +1 or -1: sign of A                      */
    int32_t drift_on;          /* 0/1                                      */
    int32_t hcs_on;            /* 0/1: wavy sheet; 0 = unipolar (h = +1)   */
    int32_t isotropic;         /* 0/1                                      */
    double R_out_AU;
    double R_ts_AU;            /* 0 = no termination shock                 */
    double ts_K_factor;
    double r_in_AU;
    double dt_max_day;
    double dt_fixed_day;       /* > 0: fixed step                          */
    double dt_min_day;
    double eps_adv;
    double eps_diff;
    double V_const_kms;        /* wind of the isotropic model              */
    double dlat_deg;
    double dts_AU;
    double dcs_min_deg;
    double rot_period_day;
    double r0_AU, th0_rad, ph0_rad;   /* detection point (start of the backward paths) */
    uint32_t max_steps;        /* step limit per path (>= 1)               */
    int32_t precision;         /* COSMICA_PREC_*                           */
    int32_t formulation;       /* 0: momentum form (Eq. 5-6, L = 0); 1: energy
                                  form (Eq. 1: kinetic energy T integrated with
                                  A_T = (2/3)(V/r) alpha T and the loss
                                  L = (2V/(3r))(1 + beta^2) accumulated for the
                                  weight of Eq. 4; needs exit->lw)              */
    int32_t reserved0;
    /* Radial shells of the inner heliosphere (Sec. II.B: shells that the wind
     * fills during successive Carrington rotations, each with its own
     * parameters).  n_shells = 0: one region with K0 and tilt_deg above.
     * n_shells = n >= 1: n equal shells between the Sun and the termination
     * shock (the outer boundary when there is none), shell k = 0 innermost;
     * the outermost continues beyond the shock.  K0 and the sheet tilt of
     * shell k are shell_K0[k] and shell_tilt_deg[k] (K0 and tilt_deg above are
     * then unused); across each interior edge R_e they pass from shell e-1's
     * to shell e's value along the cubic smoothstep over [R_e - w, R_e + w],
     * w = shell_blend_AU (needs 0 < 2w < shell width). */
    uint32_t n_shells;         /* 0 .. COSMICA_MAX_SHELLS                   */
    uint32_t reserved1;
    double shell_blend_AU;
    double shell_K0[COSMICA_MAX_SHELLS];        /* AU^2/day, > 0            */
    double shell_tilt_deg[COSMICA_MAX_SHELLS];  /* |tilt| < 89              */
    /* Nose-squashed heliosphere (Sec. II.B: inner heliosphere and heliosheath
     * squashed toward the nose, the Sun's direction of motion through the
     * interstellar medium).  squashed = 1: the termination shock and the outer
     * boundary are spheroids about the nose axis with the Sun on the axis:
     * nose distance R (R_ts_AU, R_out_AU), tail distance R * tail_ratio, flank
     * semi-axis R * flank_ratio (semi-axis R (1 + tail)/2 along the axis,
     * centre R (tail - 1)/2 behind the Sun).  The shock factor uses the shock's
     * distance along the direction of the point; a path exits when it is
     * outside the outer spheroid.  The start point must lie inside it. */
    int32_t squashed;          /* 0: spheres (R_ts_AU, R_out_AU); 1: spheroids */
    int32_t reserved2;
    double nose_th_rad, nose_ph_rad;            /* nose direction            */
    double ts_tail_ratio, ts_flank_ratio;       /* > 0                        */
    double hp_tail_ratio, hp_flank_ratio;       /* > 0                        */
} cosmica_params;

/* Particle species: mass number A, signed charge number Z, rest mass per
 * nucleon m0 [GeV].  Rigidity P = (A/|Z|) sqrt(T (T + 2 m0)) for kinetic
 * energy per nucleon T [GeV/n]. */
typedef struct {
    int32_t A;
    int32_t Z;
    double m0_GeV;
} cosmica_species;

/* Exit states, one entry per quasi-particle, structure of arrays.  Entry g is
 * the g-th particle in work-item order (item 0's particles first).  Written
 * once per particle; caller-owned, device or host memory (all arrays in the
 * same space), each of length n. */
typedef struct {
    double *r, *th, *ph, *lnP, *s;   /* post-step state at exit [AU, rad, rad, ln GV, day] */
    uint32_t *steps;                 /* Euler-Maruyama steps taken               */
    uint8_t *status;                 /* COSMICA_PATH_*                           */
    uint32_t *item;                  /* work item (energy index for propagate)   */
    uint64_t n;
    double *lw;                      /* optional: log of the loss weight
                                        exp(-sum L ds) of Eq. 4 (energy form; 0 for
                                        the momentum form); NULL = not written   */
} cosmica_exit_states;

/* Local interstellar spectrum per GeV/n (Sec. II.B, Eq. 4).
 * kind 0: analytic J = T^-2.7 / (1 + T^-3.7); kind 1: log-log table of n host
 * points (ln T ascending, ln J), linear in between, clamped at the ends. */
typedef struct {
    int32_t kind;
    uint32_t n;
    const double *lnT;
    const double *lnJ;
} cosmica_lis;

/* Exit-rigidity histogram: nbins log-spaced bins on [P_min, P_max] GV. */
typedef struct {
    double P_min_GV;
    double P_max_GV;
    uint32_t nbins;
} cosmica_bins;

/* Histogram layout per work item, (nbins + 3) uint64 counters:
 * [0] underflow, [1 .. nbins] bins, [nbins + 1] overflow, [nbins + 2] failed
 * (step limit or non-finite). */
#define COSMICA_HIST_STRIDE(nbins) ((nbins) + 3u)

typedef struct cosmica_model cosmica_model;

/* Fill *p with the library defaults (the full model of the reading above,
 * 100 AU, adaptive dt, FP64). */
void cosmica_params_default(cosmica_params *p);

/* Create a model from one parameter set (host).  Validates the parameters,
 * uploads them and derives the per-set constants on the device (synchronous).
 * *out receives the handle; destroy it with cosmica_model_destroy.
 * Errors: INVALID (with nothing allocated) for a wrong struct_size or version,
 * a non-positive or non-finite scale (K0, R_out, wind, field, step sizes), a
 * non-finite angle or tolerance, a start point outside (r_in, R_out) x (0, pi)
 * or outside the squashed outer boundary, an unknown precision or formulation,
 * or an invalid shell table; OOM; CUDA. */
cosmica_status cosmica_model_create(const cosmica_params *params, cosmica_model **out);
void cosmica_model_destroy(cosmica_model *model);

/*
 * Propagate quasi-particles backward in time until they leave the heliosphere
 * (Sec. IV.A: one thread per quasi-particle, a propagation kernel evolving
 * each path until a boundary is reached).
 *   species        host, one species for all energies
 *   T_in_GeVn      host [n_energies], kinetic energy per nucleon at the start
 *   n_per_energy   host [n_energies], quasi-particles per energy (0 allowed)
 *   seed           Philox key
 *   out            exit states; out->n must equal sum(n_per_energy); out->item
 *                  receives the energy index
 * Particle g has pid = g.  The FP64 path launches one thread per particle;
 * the mixed paths run the persistent work-queue kernel.
 * Errors: INVALID (sizes, null pointers), OOM, CUDA. */
cosmica_status cosmica_propagate(cosmica_model *model, const cosmica_species *species,
                                 const double *T_in_GeVn, uint32_t n_energies,
                                 const uint32_t *n_per_energy, uint64_t seed,
                                 cosmica_exit_states *out, void *stream);

/* One detection point of an orbit (Sec. IV.A: the detection point may move
 * along a spacecraft orbit; the quasi-particle sample is subdivided among the
 * positions, which integrates the flux over the orbit and the mission time). */
typedef struct {
    double r_AU;      /* heliocentric radius, r_in <= r < R_out                  */
    double th_rad;    /* colatitude, in (0, pi)                                   */
    double ph_rad;    /* longitude (any finite value; kept modulo 2 pi)           */
    double weight;    /* share of the sample (e.g. time spent there), > 0         */
} cosmica_position;

/*
 * cosmica_propagate with the start point moving along an orbit.  The
 * n_per_energy[e] quasi-particles of energy e are split among the positions in
 * proportion to their weights, in position order and contiguously: with
 * W_m = weight[0] + ... + weight[m-1] (summed in this order, W = W_n_positions),
 * position m receives the particles i of energy e with
 *   c_m <= i < c_(m+1),  c_m = floor(n_e * W_m / W)  (FP64, c_n_positions = n_e).
 * Particle identities are those of cosmica_propagate (pid = sum_{e'<e} n_e' + i),
 * exit entry g belongs to the same particle as there, and out->item receives
 * the energy index, so cosmica_spectrum and cosmica_spectrum_unbinned return the
 * orbit-averaged spectrum unchanged.  A single position equal to the parameter
 * set's (r0, th0, ph0) reproduces cosmica_propagate bit for bit.
 *   positions      host [n_positions], n_positions >= 1
 * Errors: INVALID (sizes, null pointers, a position outside the heliosphere or
 * a weight <= 0), OOM, CUDA. */
cosmica_status cosmica_propagate_orbit(cosmica_model *model, const cosmica_species *species,
                                       const double *T_in_GeVn, uint32_t n_energies,
                                       const uint32_t *n_per_energy, const cosmica_position *positions,
                                       uint32_t n_positions, uint64_t seed, cosmica_exit_states *out,
                                       void *stream);

/*
 * Propagation that allocates nothing.  The paper has no counterpart: this is
 * an interface for callers that cannot allocate device memory -- code running
 * under a memory pool it does not own (a framework's caching allocator may
 * hold all free memory, so a raw cudaMalloc fails or fragments the pool),
 * code that must not trigger the device-wide synchronisation of cudaFree
 * while other work is in flight, and hosts that route every device
 * allocation through an approved allocator.
 * Same arguments and results as cosmica_propagate, with the parameter set
 * passed directly instead of a model handle.  The library's scratch for the
 * call (parameter block, species, work items, prefix sums, queue cursor,
 * step counter) is a fixed static device array of about 95 KB that every GPU
 * loading the library holds until the process exits; the call makes no
 * cudaMalloc, cudaFree or other allocating call.  The tables reach the array
 * as kernel parameters, in chunks built in a few KB of the calling thread's
 * stack (no host copies, no large stack frame).
 *   n_energies   at most COSMICA_NOALLOC_MAX_ENERGIES (INVALID otherwise)
 *   out          device memory only (INVALID otherwise)
 * Set-up: each call whose stream is not capturing looks the array's address up
 * (cudaGetSymbolAddress with the device current), so calls after a re-created
 * context (cudaDeviceReset) find the new array; a call on a capturing stream
 * uses the address of the last earlier call on that device (INVALID if there
 * was none).  So make a first call on each device before any stream capture;
 * that first call may also make the CUDA driver load the library's device
 * code (lazy module loading), which allocates on the driver's side, so make
 * it during set-up, before the phase that must not allocate.
 * All calls share the array -- the counters are cleared at the start of each
 * call, the tables overwritten -- so calls whose work overlaps on the GPU
 * race; serialise them.
 */
#define COSMICA_NOALLOC_MAX_ENERGIES 1024u
cosmica_status cosmica_propagate_noalloc(const cosmica_params *params, const cosmica_species *species,
                                         const double *T_in_GeVn, uint32_t n_energies,
                                         const uint32_t *n_per_energy, uint64_t seed,
                                         cosmica_exit_states *out, void *stream);

/*
 * Bin the exit rigidities and form the modulated spectrum (Eq. 4 with L = 0
 * (Eq. 6) and J = f P^2 (Sec. VI), J the intensity per unit kinetic energy,
 * f conserved along each path): for energy e,
 *   J(T0) = P0^2 (1/N) sum_b c_b w_b,  w_b = J_LIS(T_b) / P_b^2
 * at the log-centre P_b of each bin; sigma = sample standard deviation of the
 * summand / sqrt(N).  Only EXIT paths inside [P_min, P_max) enter N.
 *   exit           device exit states (item = energy index)
 *   T_in_GeVn      host [n_energies]
 *   J_out, sigma_out  device [n_energies] (NaN where N = 0)
 *   hist_out       device [n_energies * (nbins + 3)], overwritten
 * The histogram is integer and order-independent, hence deterministic.
 * Errors: INVALID (NULL species/bins/outputs, P_min <= 0 or P_max <= P_min,
 * nbins = 0, exit or outputs not in device memory, a malformed LIS table),
 * OOM, CUDA.  n_energies = 0 is a no-op. */
cosmica_status cosmica_spectrum(const cosmica_exit_states *exit, const cosmica_species *species,
                                const double *T_in_GeVn, uint32_t n_energies,
                                const cosmica_lis *lis, const cosmica_bins *bins,
                                double *J_out, double *sigma_out, uint64_t *hist_out,
                                void *stream);

/*
 * Unbinned Eq. 4 per energy, every exit rigidity weighted exactly:
 *   formulation 0 (momentum form, L = 0):  J(T0) = P0^2 <J_LIS(T_ex) / P_ex^2>
 *   formulation 1 (energy form, Eq. 1):    J(T0) = beta0 <J_LIS(T_ex) exp(lw) / beta_ex>
 * (Eq. 1 is written for the density per unit kinetic energy U = 4 pi J / v; the
 * loss weight exp(lw) = exp(-sum L ds) is read from exit->lw).  sigma = sample
 * standard deviation of the summand / sqrt(N); only EXIT paths enter N.
 *   exit          device exit states; energy e owns the n_per_energy[e] entries
 *                 after those of energies 0..e-1 (the order cosmica_propagate writes)
 *   n_per_energy  host [n_energies]
 *   J_out, sigma_out  device [n_energies] (NaN where N = 0)
 * Sums are reduced in a fixed order, so the result is deterministic.
 * Errors: INVALID (NULL arguments, formulation not 0 or 1, exit->n not the sum
 * of n_per_energy, no exit->lw for formulation 1, buffers not in device
 * memory, a malformed LIS table), OOM, CUDA.  n_energies = 0 is a no-op. */
cosmica_status cosmica_spectrum_unbinned(const cosmica_exit_states *exit, const cosmica_species *species,
                                         const double *T_in_GeVn, uint32_t n_energies,
                                         const uint32_t *n_per_energy, int32_t formulation,
                                         const cosmica_lis *lis, double *J_out, double *sigma_out, void *stream);

/* ---------------- batched persistent launch (many heliospheres) ---------------- */

/* One work item: n quasi-particles of one species at one energy in one
 * parameter set (the paper distributes energy bins over GPUs, Sec. IV.A; here
 * many (set, species, energy) items share one persistent launch). */
typedef struct {
    uint32_t param_idx;       /* into the batch's parameter sets */
    uint32_t species_idx;     /* into the batch's species        */
    double T_GeVn;
    uint32_t n;
    uint32_t exit_item_plus1; /* 0: the item's exit records carry its index in
                                 `items`; k > 0: they carry k - 1 (a shard of a
                                 larger item list keeps that list's numbering, so
                                 its histogram rows are the list's rows)          */
    uint64_t first_pid;
    uint64_t seed;
    double r0_AU;             /* start position of the item's particles (a detection  */
    double th0_rad;           /* point of an orbit); r0_AU = 0 selects the parameter  */
    double ph0_rad;           /* set's r0, th0, ph0                                   */
} cosmica_work_item;

/* Launch shape and scheduling of the persistent kernel.  Passing NULL selects
 * block 128, the most resident blocks, compaction every 64 steps, no graph,
 * most-expensive-first queue order -- except that a launch with fewer than 8
 * particles per resident lane (bound by its slowest paths, which step faster
 * when fewer warps share an SM) takes 4 blocks of 128 per SM.  The same
 * default shapes the launches of cosmica_propagate and
 * cosmica_propagate_orbit. */
typedef struct {
    uint32_t block;           /* threads per block (32..256; 0 = 128)                   */
    uint32_t blocks_per_sm;   /* resident blocks per SM requested (0 = as many as fit)  */
    uint32_t compact_period;  /* once the queue is drained, every this many steps the
                                 active particles of a block are repacked into its lowest
                                 warps (0 = never)                                       */
    uint32_t use_graph;       /* 1: replay the launch as a CUDA graph                   */
    uint32_t queue_order;     /* 0: items in the given order; 1: items with the lowest
                                 K0 beta P first (longest paths first); exit records keep
                                 item order either way                                   */
} cosmica_tuning;

typedef struct cosmica_batch cosmica_batch;

/* Upload n_params parameter sets and n_species species (host) and derive
 * their constants on the device.  All sets must share one precision (taken
 * from params[0].precision) and one formulation.  *out receives the handle;
 * destroy it with cosmica_batch_destroy.  Errors: INVALID (no sets or species,
 * a set or species rejected as by cosmica_model_create, mixed precisions or
 * formulations; nothing allocated), OOM, CUDA. */
cosmica_status cosmica_batch_create(const cosmica_params *params, uint32_t n_params,
                                    const cosmica_species *species, uint32_t n_species,
                                    cosmica_batch **out);
void cosmica_batch_destroy(cosmica_batch *batch);

/* Run every item of `items` (host, n_items) in one persistent launch fed by a
 * device work queue.  Exit entry g belongs to the g-th particle in item order.
 * `tuning` may be NULL.  If steps_out (device, 1 uint64) is not NULL it
 * receives the total number of steps taken.  Errors: INVALID, OOM, CUDA. */
cosmica_status cosmica_batch_run(cosmica_batch *batch, const cosmica_work_item *items,
                                 uint32_t n_items, const cosmica_tuning *tuning,
                                 cosmica_exit_states *out, uint64_t *steps_out, void *stream);

/* Histogram and spectrum per work item of a batch run (same estimator as
 * cosmica_spectrum; item k uses its own species and energy).  J_out,
 * sigma_out: device [n_items]; hist_out: device [n_items * (nbins + 3)].
 * Errors: as cosmica_spectrum, and INVALID for a species index out of range. */
cosmica_status cosmica_batch_spectrum(cosmica_batch *batch, const cosmica_work_item *items,
                                      uint32_t n_items, const cosmica_exit_states *exit,
                                      const cosmica_lis *lis, const cosmica_bins *bins,
                                      double *J_out, double *sigma_out, uint64_t *hist_out,
                                      void *stream);

/* Spectra of work items from a given histogram instead of exit states: the
 * estimator of cosmica_spectrum applied to hist [n_items * (nbins + 3)]
 * (device, the layout cosmica_batch_spectrum writes), item k with its own
 * species and energy.  This is the last step of a workload partitioned over
 * several GPUs (the paper distributes energy bins over GPUs and collects
 * their histograms, Sec. IV.A): every GPU bins its share of the particles into
 * the rows of the whole item list (cosmica_work_item.exit_item_plus1), the
 * histograms are summed across GPUs (an all-reduce of integers, exact), and
 * this call turns the sum into spectra, equal bit for bit to the one-GPU
 * result.  J_out, sigma_out: device [n_items].  Errors: as
 * cosmica_batch_spectrum (hist must be device memory). */
cosmica_status cosmica_batch_spectrum_hist(cosmica_batch *batch, const cosmica_work_item *items,
                                           uint32_t n_items, const cosmica_lis *lis, const cosmica_bins *bins,
                                           const uint64_t *hist, double *J_out, double *sigma_out,
                                           void *stream);

/* Pick a launch shape for this batch by timing candidate shapes (block size,
 * resident blocks, compaction period) and write the fastest to *best (its
 * predicted steps/s in *best_rate if not NULL).  Batches of up to ~30 particles
 * per SM thread slot are timed whole; larger ones on two scaled samples of
 * `items` (host; ~10 and ~30 particles per slot), from which each candidate's
 * time for the whole batch is extrapolated linearly in the particle count.  Results are cached for the
 * process per device and configuration class (precision, drift, termination
 * shock, particle count within a factor of two, kernel variant); a cached
 * class returns at once.  Synchronous; uses the batch's own scratch.  An FP64
 * batch needs no tuning and gets block 128 without compaction.  Errors:
 * INVALID (NULL batch/best, invalid items, no particles), OOM, CUDA. */
cosmica_status cosmica_autotune(cosmica_batch *batch, const cosmica_work_item *items,
                                uint32_t n_items, cosmica_tuning *best, double *best_rate);

/* ---------------- continuous-batching server (spectrum requests) ---------------- */

/* One spectrum request: one heliosphere, one species, n_energies energies.
 * All pointers are host memory, read only during cosmica_server_submit. */
typedef struct {
    cosmica_params params;        /* precision must equal the server's       */
    cosmica_species species;
    const double *T_GeVn;         /* [n_energies]                             */
    const uint32_t *n_per_energy; /* [n_energies]                             */
    uint32_t n_energies;
    uint64_t seed;                /* particle e,i has pid = sum_{e'<e} n_e' + i */
    cosmica_bins bins;
} cosmica_request;

/* Result of a finished request.  The caller provides the host arrays:
 * J, sigma [n_energies] and hist [n_energies * (nbins + 3)] (may be NULL). */
typedef struct {
    double *J;
    double *sigma;
    uint64_t *hist;
    uint64_t steps;               /* SDE steps of the request's paths             */
    double t_submit, t_admit, t_done;   /* seconds on the server's monotonic clock */
} cosmica_result;

typedef struct {
    uint64_t submitted, admitted, completed, rejected;
    uint64_t quanta;              /* persistent launches so far                  */
    uint64_t steps;               /* SDE steps of completed requests             */
    uint64_t in_flight_particles; /* admitted, not yet exited                    */
    uint64_t arena_capacity, arena_used;   /* exit-state slots (particles)     */
    double busy_seconds;          /* wall time with work on the device           */
} cosmica_server_stats;

typedef struct cosmica_server cosmica_server;

/*
 * Create a server on the current device.  mem_budget_bytes bounds the device
 * memory the server may hold for admitted requests (exit states 49 B per
 * particle, histograms, per-slot parameters) plus its fixed suspend/resume
 * buffers; it is allocated once here.  precision: COSMICA_PREC_MIXED or
 * COSMICA_PREC_MIXED_F64ACC.  budget_steps: steps per lane per quantum (0 = 4096).
 * A scheduler thread runs quanta on the server's own stream: between quanta
 * it admits waiting requests (first come, first served) while their memory
 * fits and retires finished ones (histogram + spectrum, copied to the host);
 * in-flight particles stay resident on the device, suspended exactly.
 * Errors: INVALID, OOM, CUDA.
 */
cosmica_status cosmica_server_create(size_t mem_budget_bytes, int32_t precision, uint32_t budget_steps,
                                     cosmica_server **out);

/* Queue a request (non-blocking).  *ticket identifies it.  INVALID if the
 * request can never fit the memory budget or its fields are invalid.  The
 * server runs the momentum form (radial shells and a squashed heliosphere
 * included); requests with formulation = 1 are INVALID (use the batch entry
 * points for the energy form). */
cosmica_status cosmica_server_submit(cosmica_server *srv, const cosmica_request *req, uint64_t *ticket);

/* Non-blocking: OK and *res filled (the ticket is then released) if the
 * request is finished; BUSY if not yet; INVALID for an unknown ticket; CUDA if
 * the server failed (its message in cosmica_last_error). */
cosmica_status cosmica_server_poll(cosmica_server *srv, uint64_t ticket, cosmica_result *res);

/* As poll, waiting at most timeout_ms; TIMEOUT if still not finished. */
cosmica_status cosmica_server_wait(cosmica_server *srv, uint64_t ticket, uint32_t timeout_ms,
                                   cosmica_result *res);

/* Counters of the server so far (host copy).  Errors: INVALID (NULL arguments). */
cosmica_status cosmica_server_stats_get(cosmica_server *srv, cosmica_server_stats *st);

/* Stop the scheduler (finishing the current quantum), free everything. */
void cosmica_server_destroy(cosmica_server *srv);

/* Thread-local text of the last error of this thread ("" if none). */
const char *cosmica_last_error(void);

/* Number of device kernels this library has launched since load (all
 * threads); lets callers count launches in a timed region. */
uint64_t cosmica_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* COSMICA_H */
