/*
 * dmb.h -- C ABI of the GB300 library for the data-parallel hot path of the
 * hybrid dark matter-baryon interaction step of Hainje & Farrar (arXiv 2603.24688).
 *
 * The step (Sec. 2.4, "GIZMO implementation") has three parts:
 *   1. the cross-species pair set {(i, j): |x_i - x_j| < h_i + h_j} (i: DM, j: gas),
 *      the pairs whose overlap integral g_ij (Eq. dm-update-prob, App. D) is non-zero;
 *   2. the mean-field acceleration and heating of every gas particle
 *      (Eqs. gas-dVdt and gas-dTdt, with A and B of Eqs. scrA/scrB, App. B);
 *   3. one Monte Carlo scattering draw per DM particle (Eqs. dm-update-vels,
 *      dm-update-prob, scatter_chi; timestep criterion Eq. prob_criterion).
 *
 * Units: lengths kpc, velocities km/s, masses Msun, time kpc/(km/s), temperatures K.
 * Particle masses m_chi and mu_j are in units of the proton mass.  The cross section
 * is sigma(v) = sigma0 (v / v0)^n, isotropic (sigma = momentum-transfer sigma_bar).
 *
 * Conventions for every entry point:
 *   - array arguments marked "device" are CUDA device pointers owned by the caller;
 *     "host" pointers are ordinary host memory owned by the caller;
 *   - the context owns all scratch (sorted copies, spatial tree, pair lists, overlap
 *     table) and frees it in dmb_destroy;
 *   - work is enqueued on the context's stream; calls that return host values
 *     (n_pairs, sums) synchronise that stream, the others return immediately;
 *   - results are written in the caller's input order (never in the internal sorted
 *     order) and depend only on particle ids, not on that order;
 *   - on failure a call returns a non-zero dmb_status and dmb_last_error() describes
 *     it; the library never exits or aborts.
 */
#ifndef DMB_H
#define DMB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DMB_OK = 0,
  DMB_ERR_ARG = 1,      /* invalid argument or input value (h <= 0, NaN, T < 0, ...) */
  DMB_ERR_CUDA = 2,     /* a CUDA runtime call failed */
  DMB_ERR_OOM = 3,      /* device allocation failed */
  DMB_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up */
  DMB_ERR_DOMAIN = 5,   /* input outside what the selected rate provider covers */
  DMB_ERR_STATE = 6     /* calls made in the wrong order (e.g. neighbours before grid) */
} dmb_status;

typedef enum {
  DMB_RATE_CLOSED = 0,  /* App. B closed forms via 1F1 (integer n >= -4, n != -3) */
  DMB_RATE_QUAD = 1,    /* composite 8-panel x 8-point Gauss-Legendre quadrature of Eqs. scrA/scrB (App. B) */
  DMB_RATE_MLP = 2      /* learned surrogate of the rate integrals (float32 only; train or load first) */
} dmb_rate_mode;

/* Physical and numerical parameters (Sec. 2.4; Table test_params for typical values). */
typedef struct {
  double sigma0_cm2;    /* sigma0 in cm^2 */
  double v0_kms;        /* reference speed of the power law, km/s (> 0) */
  int32_t n;            /* power-law index, n >= -4 */
  int32_t periodic;     /* 1: periodic box [0, box)^3 with minimum-image pairs */
  double m_chi_mp;      /* DM particle mass in m_p (> 0) */
  double box[3];        /* periodic box sides in kpc (used when periodic = 1) */
  int32_t rate_mode;    /* dmb_rate_mode */
  int32_t fp64;         /* 1: all pair arithmetic in float64 (slow on GB300); 0: float32 */
  uint64_t seed;        /* key of the Philox4x32-10 streams */
} dmb_params;

/* DM particles (Eq. macroparticle-DF_DM): M_i, x_i, h_i, v_i.  All device pointers. */
typedef struct {
  int64_t n;
  const double *pos;    /* [n][3] kpc */
  const double *vel;    /* [n][3] km/s */
  const double *mass;   /* [n] Msun */
  const double *h;      /* [n] kernel-support length, kpc (> 0) */
  const uint32_t *id;   /* [n] stable ids, unique within the species; key the RNG */
} dmb_dm;

/* Gas particles (Eq. macroparticle-DF_B): M_j, x_j, h_j, V_j, T_j, mu_j.  Device pointers. */
typedef struct {
  int64_t n;
  const double *pos;    /* [n][3] kpc */
  const double *vel;    /* [n][3] bulk velocity, km/s */
  const double *mass;   /* [n] Msun */
  const double *h;      /* [n] kpc (> 0) */
  const double *T;      /* [n] temperature, K (>= 0) */
  const double *mu;     /* [n] mean molecular mass in m_p (> 0) */
  const uint32_t *id;   /* [n] stable ids, unique within the species */
} dmb_gas;

typedef struct dmb_ctx dmb_ctx;

/* Create a context on the current CUDA device.  stream: a cudaStream_t (NULL: the
 * legacy default stream).  Validates the parameters, builds the overlap table
 * (App. D) on the device.  *out is NULL on failure. */
dmb_status dmb_create(dmb_ctx **out, const dmb_params *p, void *cuda_stream);

/* Free every device buffer of the context.  NULL is accepted. */
dmb_status dmb_destroy(dmb_ctx *ctx);

/* Text of the last error of this context (or of the last failed dmb_create when ctx
 * is NULL).  Valid until the next call on the context. */
const char *dmb_last_error(const dmb_ctx *ctx);

/* Spatial index (the pair search of Sec. 2.4 on a Morton-sorted grid): Morton keys of
 * both species over one shared frame, LSD radix sort, sorted float copies, and a
 * bounding-volume tree over chunks of 32 sorted particles with per-node h_max.
 * Reads positions, velocities, masses, h, T, mu and ids; copies what it needs, so the
 * caller may change its arrays afterwards.  Inputs are checked on the device
 * (finite values, h > 0, M > 0, T >= 0, mu > 0; periodic: h_i + h_j < box/2). */
dmb_status dmb_build_grid(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas);

/* Pair set {(i, j): d_ij < h_i + h_j} (strict; minimum image when periodic) from the
 * grid of the last dmb_build_grid.  Builds gas-major and DM-major pair lists in the
 * context.  n_pairs (host, may be NULL) receives the count (synchronises).  If
 * pairs_out (device, may be NULL) is given it receives min(count, capacity) pairs as
 * [k][2] uint32 (DM input index, gas input index), grouped by gas. */
dmb_status dmb_neighbors(dmb_ctx *ctx, int64_t *n_pairs, uint32_t *pairs_out, int64_t capacity);

/* Gas mean field (Eqs. gas-dVdt, gas-dTdt) over the pairs of the last dmb_neighbors,
 * from the state given to the last dmb_build_grid.  acc: device [N_B][3] float64,
 * (km/s)^2/kpc; dudt: device [N_B] float64, du_j/dt = (3/(2 mu_j)) dT_j/dt in
 * (km/s)^3/kpc.  Per-gas sums are accumulated in float64. */
dmb_status dmb_meanfield_gas(dmb_ctx *ctx, double *acc, double *dudt);

/* DM Monte Carlo (Eqs. dm-update-vels, dm-update-prob, scatter_chi) for time step dt at
 * step index `step` (both key the Philox streams).  One categorical draw per DM
 * particle: partners in ascending gas id, P_ij summed exactly; if sum_j P_ij > 1 the
 * draw is renormalised (the particle scatters surely) and counted.
 *   vel_out     device [N_chi][3] float64: new DM velocities
 *   scattered   device [N_chi] uint8 (may be NULL): 1 if the particle scattered
 *   partner     device [N_chi] uint32 (may be NULL): gas id of the partner, or 0xFFFFFFFF
 *   p_ratio_max device [N_chi] float32 (may be NULL): max_j P_ij / min(0.1,
 *               1e-4 ((m_chi + mu_j)/mu_j)^2), the Eq. prob_criterion ratio
 *   p_total     device [N_chi] float64 (may be NULL): sum_j P_ij */
dmb_status dmb_mc_scatter_dm(dmb_ctx *ctx, uint64_t step, double dt, double *vel_out,
                             uint8_t *scattered, uint32_t *partner, float *p_ratio_max,
                             double *p_total);

/* One whole step: grid, pairs, mean field, Monte Carlo, kicks and float64 sums.
 * Updates in place (device arrays, the caller's): dm->vel (cast away const),
 * gas->vel and gas->T (V_j += a_j dt; u_j += du_j/dt dt clamped at 0; T from u).
 * sums_out (host, 16 doubles, may be NULL; synchronises):
 *   [0:3] sum_i M_i dv_i (DM, realised)   [3:6] sum_j M_j a_j dt (gas)
 *   [6] DM kinetic-energy change          [7] gas kinetic + thermal energy change
 *   [8] sum_i E[dE_i] (App. C)            [9] scatters  [10] renormalised draws
 *   [11] clamped gas u                    [12] pairs    [13] sum_ij P_ij
 *   [14] max p_ratio                      [15] decisions within 1e-6 of a threshold */
dmb_status dmb_step(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, uint64_t step,
                    double dt, double *sums_out);

/* Parameters of one box of a batched step (the values that vary from box to box in a parameter
 * scan; the power law n, v0, seed and precision are the context's). */
typedef struct {
  double box[3];        /* periodic sides, kpc */
  double sigma0_cm2;    /* this box's sigma0 */
  double m_chi_mp;      /* this box's m_chi in m_p */
} dmb_box;

/* One step of many independent periodic boxes at once (the same physics as dmb_step in each
 * box; no pair ever joins two boxes).  The particles of all boxes are given concatenated in
 * any order, with dm_box / gas_box (device, uint32 [n]) naming each particle's box in
 * boxes[0 .. nbox-1] (host).  Every stage runs once over all boxes: the box index is the top
 * field of the Morton key, boxes occupy disjoint slots of one virtual space, and each pair uses
 * its box's sides for the minimum image and its box's sigma0 and m_chi.  Requires a periodic
 * context; h < min(box side)/4 is checked on the device.  sums_out: as dmb_step, over all
 * boxes. */
dmb_status dmb_step_batched(dmb_ctx *ctx, const dmb_dm *dm, const uint32_t *dm_box, const dmb_gas *gas,
                            const uint32_t *gas_box, const dmb_box *boxes, int32_t nbox, uint64_t step, double dt,
                            double *sums_out);

/* Debug/verification: evaluate the device overlap integral used by the pair kernels
 * for k (d, h_i, h_j) triples.  in: device [k][3] float64; out: device [k] float64.
 * Uses the table (float32 mode) or the exact evaluator (fp64 mode). */
dmb_status dmb_debug_overlap(dmb_ctx *ctx, int64_t k, const double *in, double *out);

/* Debug/verification: the device rate provider's normalised integrals for k samples
 * (the provider chosen by params.rate_mode).  in: device [k] float64 x = w^2/(2 varsigma^2);
 * out: device [k][2] float64 (FA, FB) with A = (alpha_n/3)(sigma0/v0^n) varsigma^(n+1) FA and
 * B = alpha_n (sigma0/v0^n) varsigma^(n+3) FB (App. B); for the power law
 * FA = 1F1(-(n+1)/2, 5/2; -x), FB = 1F1(-(n+3)/2, 3/2; -x). */
dmb_status dmb_debug_rates(dmb_ctx *ctx, int64_t k, const double *in, double *out);

/* Debug/verification: Philox4x32-10 on the device.  ctr: device [k][4] uint32,
 * out: device [k][4] uint32 with key = params.seed. */
dmb_status dmb_debug_philox(dmb_ctx *ctx, int64_t k, const uint32_t *ctr, uint32_t *out);

/* ---- hierarchical substeps (power-of-two timestep bins) ----------------------------------
 * Sec. 2.4 limits each DM particle's timestep by the scatter probability (Eq. prob_criterion);
 * with power-of-two timesteps a particle in bin b has dt = 2^b dt_min and is active at substep
 * s when s mod 2^b == 0.  At a substep the active gas particles receive the mean field (Eqs.
 * gas-dVdt, gas-dTdt) of ALL their DM partners and are kicked with their own dt; the active DM
 * particles draw the Monte Carlo (Eqs. dm-update-vels, dm-update-prob, scatter_chi) against ALL
 * their gas partners with their own dt (Philox step = s); every other particle is unchanged.
 * Positions do not change across substeps (drift is not part of the interaction step), so the
 * grid and pairs of dmb_build_grid + dmb_neighbors serve every substep.
 *
 * dmb_set_bins: set-up after dmb_neighbors (synchronises).  dm_bin, gas_bin: device uint8 [n]
 * in caller order, values 0..63 (DMB_ERR_ARG otherwise).  The arrays must stay valid and
 * unchanged while substeps run.  Orders each species by (bin, sorted index) so that every
 * substep's active set is a prefix of it, and allocates all substep scratch.  Single-box
 * contexts only.  A later dmb_build_grid, dmb_neighbors or dmb_step invalidates it. */
dmb_status dmb_set_bins(dmb_ctx *ctx, const uint8_t *dm_bin, const uint8_t *gas_bin);

/* Monte Carlo variant of every later step (dmb_mc_scatter_dm, dmb_step, dmb_step_batched,
 * dmb_substep).  0 (default): one categorical draw per dark-matter particle per step, the form
 * of the derivation (Eqs. dm-update-vels, dm-update-prob).  1: the per-pair Bernoulli form in
 * which Sec. 2.5 applies it: the particle's pairs, in ascending gas id, each scatter when
 * r_ij < P_ij, with P_ij from the velocity after any earlier scatter of the step.  r_ij and the
 * new direction come from the pair's Bernoulli Philox stream: counter (id_i, id_j, step_lo,
 * step_hi & 0x3fffffff | 0x40000000); words 0 and 3 give r_ij with 52 random bits, words 1 and
 * 2 cos theta' and phi' as for the categorical draw.  Steps must stay below 2^62.  At most 64
 * scatters per particle and step.  The outputs keep their meaning: p_total and p_ratio_max
 * from the velocity at the start of the step, partner = the first partner, the new velocity
 * after all kicks.  DMB_ERR_ARG for other values.  Drops captured substep graphs. */
dmb_status dmb_set_mc_variant(dmb_ctx *ctx, int32_t variant);

/* Anisotropic scattering (Sec. 2.4: the Monte Carlo's probability takes the total cross
 * section sigma, the gas exchange rates the momentum-transfer cross section sigma_bar; the
 * power-law runs are isotropic, sigma = sigma_bar).  Sets dsigma/dOmega = sigma(v) (1 + beta
 * cos theta) / (4 pi), theta the angle between the relative velocity before and after the
 * collision: the Monte Carlo (both variants) keeps P_ij with sigma and draws cos theta from the
 * density (1 + beta m) / 2 about the incoming relative velocity (the step's isotropic cosine
 * word mapped through the inverse cumulative distribution, the azimuth word about an
 * orthonormal basis of that direction); the mean field, the expected DM energy change and the
 * gas coefficients take sigma_bar = sigma (1 - beta / 3) (<cos theta> = beta / 3).  beta = 0
 * (the default) is the isotropic step unchanged.  beta in [-1, 1] (dsigma/dOmega >= 0),
 * DMB_ERR_ARG otherwise.  A change drops the grid, the pair lists, the substep tables and the
 * captured graphs (dmb_set_bins again before dmb_substep); dmb_step rebuilds the rest. */
dmb_status dmb_set_anisotropy(dmb_ctx *ctx, double beta);

/* Velocity law of the cross section (Sec. 2.4: the method takes any sigma(v) whose A and B can be
 * computed; the power law has the App. B closed forms).  family 0 (the default): the power law of
 * the parameters, sigma0 (v / v0)^n.  family 1: the screened law sigma(v) = sigma0 / (1 + (v /
 * v_c)^2)^2 with v_c_kms > 0 (scattering through a massive mediator: flat below v_c, falling as
 * v^-4 above it).  With it the Monte Carlo takes sigma(v_rel) in P_ij (Eq. dm-update-prob); the
 * mean field's A and B come from the device quadrature (DMB_RATE_QUAD: the integrand carries
 * sigma_bar(u) / sigma0, the window is split where the law's poles come near it) or from a
 * surrogate trained for this law (DMB_RATE_MLP: dmb_train_surrogate after this call; its second
 * input is then varsigma^2 / v_c^2); the closed forms exist for the power law only, so
 * DMB_RATE_CLOSED gives DMB_ERR_ARG.  The rates keep the n = 0 normalisation,
 * A = (alpha_0 / 3) sigma0 varsigma FA and B = alpha_0 sigma0 varsigma^3 FB, with FA, FB functions
 * of x and q = varsigma^2 / v_c^2.  Composes with dmb_set_anisotropy (sigma_bar = sigma (1 - beta/3)).
 * A change drops the grid, the pair lists, the substep tables and the captured graphs, as
 * dmb_set_anisotropy does.  Other family values or v_c <= 0: DMB_ERR_ARG. */
dmb_status dmb_set_cross_section(dmb_ctx *ctx, int32_t family, double v_c_kms);

/* Debug/verification: the device quadrature of the screened law (see dmb_set_cross_section) at k
 * points, in the context's precision.  in: device [k][2] float64 (x = w^2 / (2 varsigma^2),
 * q = varsigma^2 / v_c^2); out: device [k][2] float64 (FA, FB) of the n = 0 normalisation. */
dmb_status dmb_debug_rates_screened(dmb_ctx *ctx, int64_t k, const double *in, double *out);

/* Timestep feedback (Sec. 2.5, Eq. prob_criterion: a dark-matter particle whose P_ij is too
 * large takes a smaller timestep next).  p_ratio_max: device float [n], max_j P_ij / min(0.1,
 * 1e-4 ((m_chi + mu_j) / mu_j)^2) of each particle at its current dt_i = 2^bin dt_min, as
 * dmb_mc_scatter_dm writes it; dm_bin: device uint8 [n], updated in place.  P_ij is proportional
 * to dt, so the ratio at bin b' is ratio 2^(b' - b).  A particle with ratio > 1 (or not finite)
 * moves to the largest bin b' <= b with ratio 2^(b' - b) <= 1 (at least 0); one with ratio < 1/4
 * moves up one bin if b < max_bin and substep (the next substep) is a multiple of 2^(b+1); all
 * others keep their bins.  The paper gives the criterion, not this bin arithmetic: the rule is
 * this library's reading.  active (device uint8 [n] or NULL = all): only particles with a
 * nonzero flag move.  n in [0, 2^31) and max_bin in [0, 63] (DMB_ERR_ARG otherwise).  n_changed (host, may be NULL):
 * the number of bins that moved; when given the call synchronises.  The new bins take effect
 * through dmb_set_bins. */
dmb_status dmb_rebin_dm(dmb_ctx *ctx, const float *p_ratio_max, uint8_t *dm_bin, int64_t n, int32_t max_bin,
                        uint64_t substep, const uint8_t *active, int64_t *n_changed);

/* Host-side sizes of substep s (no GPU work): out5 = {active DM, active gas, mean-field row
 * segments, pairs of the active gas rows, pairs of the active DM rows}. */
dmb_status dmb_substep_info(dmb_ctx *ctx, uint64_t substep, int64_t *out5);

/* One substep s with dt_min (see above).  dm, gas: the same particles (and arrays) as the
 * grid was built from; updates dm->vel, gas->vel and gas->T in place (device) and keeps the
 * library's sorted copies of the updated particles current.  Between substeps the caller
 * changes the particle state only through dmb_substep (otherwise: dmb_build_grid again).
 * Stream-ordered, no allocation, no host synchronisation unless sums_out (host, 16 doubles,
 * as dmb_step with [12] = half the pair evaluations of the substep) is given.
 * With dmb_set_graph(ctx, 1) each distinct active set is captured once into a CUDA graph
 * (on a stream of the library's, ordered after the context stream by events) and replayed;
 * the results are the same as without graphs. */
dmb_status dmb_substep(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, uint64_t substep,
                       double dt_min, double *sums_out);

/* on = 1: dmb_substep replays captured CUDA graphs; 0: launches directly. */
dmb_status dmb_set_graph(dmb_ctx *ctx, int on);

/* Engine of the surrogate's pair pass: 0 (default) 128-pair tiles on the tcgen05 tensor cores
 * with the accumulators in tensor memory; 1 the warp-level mma.sync pass (kept for
 * comparison).  Both evaluate the same network; captured substep graphs are dropped. */
dmb_status dmb_set_surrogate_engine(dmb_ctx *ctx, int32_t engine);

/* Raw outputs of the network for n input rows on the tcgen05 engine (same contract as
 * dmb_surrogate_infer; synchronises to report a timed-out tensor-core wait as DMB_ERR_TIMEOUT). */
dmb_status dmb_surrogate_infer_tc(dmb_ctx *ctx, const float *X, int64_t n, float *Y);

/* ---- launch shapes and their autotuner (no counterpart in the paper: the shapes are how this
 * library maps the work onto the GPU; the physics does not depend on them) --------------------
 * shapes[5] = {search work unit (target leaves per unit, 4..1024; default 64),
 *              mean-field segment (pairs per warp task, 128..65536; default 2048),
 *              mean-field blocks per SM (grid cap, 1..64; default 32),
 *              Monte Carlo blocks per SM (1..64; default 32),
 *              surrogate warpgroups per CTA (2..4; default 4; with 2 the activations are
 *              kept in tensor memory)}.
 * dmb_autotune: builds the grid of (dm, gas) and times, with CUDA events on the context stream,
 * each candidate of one shape at a time in the order of the array (the search with units
 * {16, 32, 64, 128}; the mean field with segments {512, 1024, 2048, 4096} x blocks {8, 16, 32}
 * and, with a trained surrogate, warpgroups {2, 3, 4}; the Monte Carlo with blocks {4, 8, 16, 32}),
 * keeps the fastest of each and leaves the grid and pairs of (dm, gas) built.  The caller's
 * arrays are only read.  shapes_out (host [5]) and report (host, up to 23 doubles: the candidate
 * times in ms in the order above) may be NULL.  Synchronises.  Single-box contexts.
 * dmb_set_shapes / dmb_get_shapes: set or read them (setting invalidates pairs and substep tables). */
dmb_status dmb_autotune(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, int32_t *shapes_out, double *report);
dmb_status dmb_set_shapes(dmb_ctx *ctx, const int32_t *shapes);
dmb_status dmb_get_shapes(dmb_ctx *ctx, int32_t *shapes_out);

/* Persisted launch shapes: dmb_save_shapes writes the context's shapes (dmb_get_shapes) under
 * `key` into the JSON file at `path` ({"key": [5 integers], ...}; other keys are kept; the file is
 * replaced atomically); dmb_load_shapes sets them from the entry of `key` (DMB_ERR_STATE when the
 * file or the key is absent, DMB_ERR_ARG for a malformed or out-of-range entry).  Keys are made of
 * [A-Za-z0-9._+-] (a workload name, say).  Host-only; no GPU work. */
dmb_status dmb_save_shapes(dmb_ctx *ctx, const char *path, const char *key);
dmb_status dmb_load_shapes(dmb_ctx *ctx, const char *path, const char *key);

/* Stage timing of dmb_step with CUDA events recorded on the context stream (adds one
 * event synchronisation per step).  on = 0 disables it.  Resets the accumulators. */
dmb_status dmb_set_timing(dmb_ctx *ctx, int on);

/* Accumulated stage times since dmb_set_timing or the last call, in ms (host [8]):
 * [0] grid (frame, keys, sort, gather, tree)  [1] pair search (count, scan, emit, both
 * directions)  [2] mean field  [3] Monte Carlo  [4] kicks and sums  [5] the surrogate's pair
 * pass (part of [2]; 0 for the other rate providers)  [6..7] 0.
 * steps_out (host, may be NULL): steps timed.  Resets the accumulators. */
dmb_status dmb_stage_times(dmb_ctx *ctx, double *ms_out, int64_t *steps_out);

/* Work counters of the last dmb_neighbors (host [16] uint64).  [0..3] gas-major search,
 * [4..7] DM-major search, each: tree nodes visited (stage 1), target leaves tiled
 * (stage 2 count pass), candidate pair tests after the ballot filter (count pass), 0.
 * Synchronises. */
dmb_status dmb_search_stats(dmb_ctx *ctx, uint64_t *out16);

/* ---- learned surrogate of the rate integrals (rate_mode = DMB_RATE_MLP) ------------------
 * A 4 -> 128 -> 128 -> 128 -> 2 MLP (squared-ReLU activations max(z, 0)^2; bf16 tensor-core
 * hidden layers, float32 accumulation) standing in for FA, FB of Eqs. scrA/scrB (the App. B normalisation).  Inputs
 * log10(s)/2, log10(tau)/2, log10(m_chi/m_p), n/4 with s = w/varsigma, tau = varsigma^2/v0^2;
 * outputs the residuals of log FA, log FB against envelopes with the exact small- and large-x
 * limits.  The paper has no surrogate: it evaluates 1F1 (Sec. 2.4); quadrature is the
 * reference it is trained on and the fallback outside the training box
 * (s in [1e-2, 1e2], tau in [1e-3, 1e2], m_chi in [0.5, 10] m_p). */

/* Train on the device: nsamples points drawn with Philox(seed), targets from the float64 device
 * quadrature, 10% held out; Adam with a cosine schedule, batch 4096, `epochs` passes.
 * report (host [8], may be NULL): last-batch loss, max and mean relative validation errors of
 * FA and FB ([1],[2],[3],[4]), seconds, optimiser steps, samples.  Synchronises. */
dmb_status dmb_train_surrogate(dmb_ctx *ctx, int64_t nsamples, int32_t epochs, uint64_t seed, double *report);

/* How a float32 step with one categorical draw per DM particle (dmb_step, dmb_step_batched) runs
 * its pair physics: on = 1: one pass over the gas-major pairs evaluates each pair's geometry and
 * overlap once for both the mean field and P_ij of the Monte Carlo, and a second pass per DM row
 * sums and selects from those P_ij (read through each DM-major entry's gas-major position, which
 * the pair search then also writes); on = 0 (the default, faster on the galaxy workloads): the
 * mean field and the Monte Carlo run as separate passes over their own row orders.  The results
 * are the same bit for bit.  Other values: DMB_ERR_ARG.  (The standalone calls, the float64 mode, the per-pair Bernoulli variant
 * and the substeps always use the separate passes.) */
dmb_status dmb_set_fusion(dmb_ctx *ctx, int32_t on);

/* Where the float32 mean field with the learned surrogate (DMB_RATE_MLP on the tensor-core
 * engine) sums its pairs (Eqs. gas-dVdt, gas-dTdt): mode = 0 (the default, faster on the galaxy
 * workloads): the surrogate's tensor-core kernel stores every pair's (FA, FB) and the mean-field
 * kernel reads them back, summing in segments of the autotuned length.  mode = 1: inside the
 * surrogate's kernel, which forms each pair's overlap while its last MMA runs and its rates after
 * the output layer, sums the pair terms per gas row over each warp's 32 pairs and leaves the
 * float64 sum over those partial sums to one thread per gas row; no rate is stored.  The two
 * modes differ only in the order of the float32 additions.  The fused pair pass of
 * dmb_set_fusion(ctx, 1) always reads stored rates.  Other values: DMB_ERR_ARG. */
dmb_status dmb_set_surrogate_epilogue(dmb_ctx *ctx, int32_t mode);

/* Pair weights of a float32 pair set: the search's emit pass forms every pair's overlap g_ij
 * (Eqs. gas-dVdt, dm-update-prob; the canonical displacement and the overlap table, the same
 * arithmetic as the interaction kernels) and stores M_i g_ij beside each gas-major entry and g_ij
 * beside each DM-major entry; the mean field and the Monte Carlo then read them instead of
 * gathering positions and evaluating the table.  Results are the same bit for bit.  The search
 * pays for them (about the time the two kernels save), so they pay off when a pair set serves
 * many passes.  mode = -1 (the default): stored when the pair set is kept for later calls, i.e.
 * by dmb_neighbors (the pair set of dmb_set_bins / dmb_substep and of the standalone
 * dmb_meanfield_gas / dmb_mc_scatter_dm), not by the search inside dmb_step or dmb_step_batched;
 * 0: never; 1: always.  Other values: DMB_ERR_ARG.  float64 contexts never store them. */
dmb_status dmb_set_pair_weights(dmb_ctx *ctx, int32_t mode);

/* Which power-law indices the next dmb_train_surrogate covers: 0 (the default) the scan's
 * {-4, -2, 0, 2} and the context's n, one network for all of them; 1 the context's n only (the
 * network's fourth input is then constant, and all of its capacity serves that n).  Other values:
 * DMB_ERR_ARG.  The screened law always trains its single normalisation. */
dmb_status dmb_set_surrogate_scope(dmb_ctx *ctx, int32_t scope);

/* Copy the float32 parameter block to host memory (count receives its length; host_out may be
 * NULL to query it).  Layout: W1[128][4] b1 W2[128][128] b2 W3[128][128] b3 W4[2][128] b4. */
dmb_status dmb_surrogate_params(dmb_ctx *ctx, float *host_out, int64_t *count);

/* Load a parameter block (host, count floats) as the context's surrogate. */
dmb_status dmb_load_surrogate(dmb_ctx *ctx, const float *host_params, int64_t count);

/* Raw network outputs for n inputs.  X: device [n][4] float32; Y: device [n][2] float32. */
dmb_status dmb_surrogate_infer(dmb_ctx *ctx, const float *X, int64_t n, float *Y);

/* Loss and gradient of the mean squared error on a batch (checks the backward kernels).
 * X: device [B][4], Y: device [B][2] targets, grad: device [count] float32 (dL/dp for
 * L = sum over the batch and both outputs of (y - target)^2 / B); loss: host, may be NULL. */
dmb_status dmb_surrogate_grad(dmb_ctx *ctx, const float *X, const float *Y, int32_t B, float *grad, double *loss);

/* Number of pairs of the last mean-field call that fell back to quadrature (outside the
 * training box).  Synchronises. */
dmb_status dmb_surrogate_fallbacks(dmb_ctx *ctx, int64_t *out);

/* dmb_surrogate_grad without any device allocation (the paper has no counterpart: it is a
 * service of this library).  dmb_surrogate_grad allocates its work buffers on every call; this
 * variant is for callers that cannot call cudaMalloc/cudaFree at that point - inside CUDA-graph
 * capture, under an external allocator that owns all device memory, or in loops where an
 * allocation's implicit synchronisation is not acceptable.  Its work buffers live in one fixed
 * device array of about 16 MB, reserved on every GPU that loads the library until the process
 * exits, so B is limited to 4096 (larger B returns DMB_ERR_ARG).  Same arguments, results and
 * kernels as dmb_surrogate_grad.  The first call on a device looks the array up (setup); make it
 * before any stream capture.  All calls on a device share the array: calls whose work overlaps on
 * the GPU (different streams or contexts without ordering) race and give wrong results.  When
 * loss is non-NULL the call synchronises the context's stream.  The current CUDA device must be
 * the one the context was created on (DMB_ERR_STATE otherwise); the array's address is looked up
 * once per device, so a cudaDeviceReset after the first call is not supported. */
dmb_status dmb_surrogate_grad_noalloc(dmb_ctx *ctx, const float *X, const float *Y, int32_t B, float *grad,
                                      double *loss);

/* Fault injection for the timeout path of the tensor-core surrogate (failure detection; the
 * paper has no counterpart).  With on = 1 the next tensor-core surrogate launch of this context
 * (dmb_surrogate_infer_tc, or the surrogate pass of a mean field) leaves out the completion
 * commit of one MMA (warpgroup 0 of the first CTA, its first layer-1 MMA) and limits its waits
 * to 1 ms, so that bounded wait runs out.  The kernel then commits again, waits (bounded) for
 * the MMAs it has in flight, frees its tensor memory and ends normally; the call that
 * synchronises on it returns DMB_ERR_TIMEOUT and the context stays usable.  Applies to one
 * launch; on = 0 cancels it; other values: DMB_ERR_ARG.  No GPU fault is involved. */
dmb_status dmb_debug_tc_timeout(dmb_ctx *ctx, int32_t on);

/* Number of kernel launches the context has issued since creation (bench accounting). */
int64_t dmb_launch_count(const dmb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DMB_H */
