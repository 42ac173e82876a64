// Pair search, mean field and Monte Carlo kernels.
#pragma once
#include <cuda_bf16.h>

#include "grid.cuh"
#include "mlp.cuh"

// Surrogate handles for the mean-field kernel (rate_mode = DMB_RATE_MLP).
struct MlpRun {
  const float *p;                  // float32 parameters
  const __nv_bfloat16 *w2, *w3;    // bf16 copies of the 128 x 128 layers
  MlpDomain dom;
  unsigned long long *fallback_count;
  const float2 *rates;             // per gas-major pair (FA, FB) from launch_mlp_pair_rates
};

#define SR_UNIT 64   // default target leaves per work unit of the tile stage
#define MF_SEG 2048  // default pairs per mean-field work segment (long rows are split)

// Launch shapes: defaults, or the choice of the autotuner (dmb_autotune).
struct Shapes {
  int unit = SR_UNIT;   // target leaves per search work unit
  int seg = MF_SEG;     // pairs per mean-field segment
  int mf_bps = 32;      // mean-field blocks per SM (grid cap of the persistent loop)
  int mc_bps = 32;      // Monte Carlo blocks per SM
  int tc_wg = 4;        // warpgroups (128-pair tiles in flight) per surrogate CTA: 2 to 4
};

template <typename R>
cudaError_t launch_leaf_pairs(SpeciesView<R> Q, SpeciesView<R> O, BoxSplit bx, const Frame *frame, bool emit,
                              uint32_t *item_cnt, const int64_t *item_ptr, uint32_t *items, uint32_t *status,
                              unsigned long long *stats, cudaStream_t s, int64_t *launches);
cudaError_t launch_unit_counts(const int64_t *item_ptr, int nleaf, int unit, uint32_t *unit_cnt, cudaStream_t s,
                               int64_t *launches);
cudaError_t launch_unit_map(const int64_t *item_ptr, const int64_t *unit_ptr, int nleaf, int unit, uint32_t *unit_leaf,
                            int64_t *unit_item0, cudaStream_t s, int64_t *launches);
// The transposed (target-major) lists written by the tile stage as it finds the pairs: the
// count pass adds each tile's pairs to cnt[target]; the emit pass claims positions with
// cursor[target] and writes the query index at ptr[target] + position (row order within a
// target follows the tiles' completion, so consumers must not depend on it).
struct TransposeOut {
  uint32_t *cnt = nullptr;       // [targets] (count pass)
  uint32_t *cursor = nullptr;    // [targets], zeroed (emit pass)
  const int64_t *ptr = nullptr;  // [targets + 1] row starts (emit pass)
  uint32_t *rows = nullptr;      // [pairs] (emit pass)
  uint32_t *gidx = nullptr;      // [pairs] (emit pass, may be null): the pair's query-major position
};

// Pair weights of a float32 search, written by the emit pass from the tile masks: the overlap
// g_ij (Eqs. gas-dVdt, dm-update-prob) at every target-major entry and the target's mass times
// g_ij at every query-major entry.  The emit pass forms them from the canonical displacement and
// the overlap table exactly as the mean-field and Monte Carlo kernels would, which then read them
// instead of gathering positions.
struct PairWeights {
  float *q = nullptr;             // [pairs] query-major: M_target g_ij
  float *t = nullptr;             // [pairs] target-major: g_ij
  const float4 *gtab = nullptr;   // overlap table
};

// tmask (optional, [items][32] uint32): the count pass stores each tile's pair masks (entry k:
// the query lanes paired with target k of the item's leaf) and the emit pass reads them instead
// of testing the distances again.  pw (emit pass with tmask, float32 only): the pair weights.
template <typename R>
cudaError_t launch_tile(SpeciesView<R> Q, SpeciesView<R> O, BoxSplit bx, const Frame *frame, bool emit,
                        const uint32_t *unit_leaf, const int64_t *unit_item0, const int64_t *item_ptr,
                        const uint32_t *items, int64_t n_units, int unit, uint32_t *unit_cnt, const int64_t *row_ptr,
                        uint32_t *rows, TransposeOut tr, uint32_t *tmask, uint32_t *status, unsigned long long *stats,
                        cudaStream_t s, int64_t *launches, const int64_t *n_units_dev = nullptr,
                        PairWeights pw = PairWeights());
// Capacity check of a captured step (the host sized the buffers before capture and reads no
// count back): totals [k] against cap [k], written to need[slot[k]]; on overflow gate = 1, the
// status gets DMB_BAD_OVERFLOW and the offset arrays zero[k] (zero_n[k] entries) are cleared.
struct CapCheck {
  const int64_t *total[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t cap[4] = {0, 0, 0, 0};
  int slot[4] = {0, 0, 0, 0};
  int64_t *zero[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t zero_n[4] = {0, 0, 0, 0};
  int64_t *need = nullptr;
  uint32_t *gate = nullptr;
  uint32_t *status = nullptr;
};
cudaError_t launch_cap_check(const CapCheck &c, cudaStream_t s, int64_t *launches);

cudaError_t launch_unit_prefix(const int64_t *unit_ptr, int nleaf, int64_t nq, uint32_t *unit_cnt, uint32_t *counts,
                               cudaStream_t s, int64_t *launches);


cudaError_t launch_seg_counts(const int64_t *row_ptr, int64_t n, int seg, uint32_t *cnt, cudaStream_t s,
                              int64_t *launches);
cudaError_t launch_seg_map(const int64_t *row_ptr, const int64_t *seg_ptr, int64_t n, int seg, uint32_t *seg_row,
                           int64_t *seg_begin, cudaStream_t s, int64_t *launches);

// Mean-field row segments: segment u covers pairs [begin[u], min(begin[u] + seg_len, end of row)).
// Without a row list the rows are all gas particles in sorted order and seg_ptr is indexed by
// the sorted gas index; with a list (the active gas of a substep) row k is gas list[k] and
// seg_ptr is indexed by k.
struct SegView {
  const int64_t *seg_ptr;     // [rows + 1]: segments of row k are [seg_ptr[k], seg_ptr[k+1])
  const uint32_t *seg_row;    // [n_seg]: sorted gas index of the segment's row
  const int64_t *seg_begin;   // [n_seg]
  const uint32_t *list = nullptr;   // sorted gas index of row k, or null (row k is gas k)
  int64_t n_rows = -1;        // rows when list is set
  int64_t n_seg = -1;         // segments to process; < 0: seg_ptr[N_B] read on the device
  int seg_len = MF_SEG;       // pairs per segment the table was built with
};

struct MfOut {
  double *acc;      // [N_B][3] caller order
  double *dudt;     // [N_B] caller order
  double *e_exp;    // [N_B] sorted order: M_j (cB sum tFB - cA sum tFA v_i.w) (no dt); may be null
};

// part: scratch [n_seg][6] in the pair precision (per-segment sums before the float64 finish)
// wq: float32 steps, M_i g_ij of every gas-major pair (PairWeights::q of the search); the float64
// path forms g_ij from the positions with the exact evaluator and takes null
template <typename R>
cudaError_t launch_meanfield(SpeciesView<R> G, SpeciesView<R> D, BoxSplit bx, const int64_t *row_ptr,
                             const uint32_t *rows, SegView sv, int64_t n_seg_max, const float4 *gtab, RunConst rc,
                             MfOut out, R *part, MlpRun mr, int blocks_per_sm, cudaStream_t s, int64_t *launches,
                             const float *wq);

struct McArgs {
  double dt;
  unsigned long long step, seed;
  int id_bits;                // bits needed for the largest gas id
  const double *vel_in;       // caller DM velocities [N][3]
  double *vel_out;            // [N][3] (may alias vel_in)
  uint8_t *scattered;         // may be null
  uint32_t *partner;          // may be null
  float *p_ratio;             // may be null
  double *p_total;            // may be null
  double *block_sums;         // [finish blocks][8]: sum M dv (3), dKE, scatters, clamps, band, sum P
  double *block_max;          // [finish blocks]: max p_ratio
  // hierarchical substeps: the rows are the DM of `list` (sorted indices, n_list of them), each
  // with its own dt = dt 2^bin (bin in caller order); the step number is read on the device;
  // the finish also refreshes the sorted velocity copy of the particles it updates
  const uint32_t *list = nullptr;
  int64_t n_list = 0;
  const uint8_t *bin = nullptr;
  const unsigned long long *step_dev = nullptr;
  void *v_sorted = nullptr;   // Vec<R>::v4 [N_chi] or null
  int v_sorted_fp64 = 0;
  // 0: one categorical draw per DM particle; 1: the per-pair Bernoulli variant (k_mc_bernoulli)
  int variant = 0;
  // dsigma/dOmega proportional to 1 + beta cos theta (0: isotropic)
  double beta = 0.0;
  // float32 steps: g_ij of every DM-major pair (PairWeights::t of the search), read by the
  // categorical draw instead of the positions; null in float64 (g from the exact evaluator)
  const float *g = nullptr;
};

// Sets the surrogate pass's shared-memory attribute (done before any graph capture).
cudaError_t prepare_mlp_pair_rates();
cudaError_t launch_mlp_pair_rates(SpeciesView<float> G, SpeciesView<float> D, const int64_t *row_ptr,
                                  const uint32_t *rows, SegView sv, int64_t n_seg_max, RunConst rc, MlpRun mr,
                                  float2 *rates, cudaStream_t s, int64_t *launches);

// Per-DM result of the Monte Carlo kernel (sorted order), finished in float64 by k_mc_finish.
struct McRec {
  unsigned long long c_lo, c_hi;  // sum_j P_ij, 128-bit fixed point with 64 fractional bits
  float rmax;                     // max_j P_ij / P_cap
  uint32_t flags;                 // 1 scattered, 2 renormalised (sum > 1), 4 within 1e-6 of a threshold
  uint32_t partner;               // gas id or 0xffffffff
  double dv[3];                   // velocity change
};

template <typename R>
cudaError_t launch_mc(SpeciesView<R> D, SpeciesView<R> G, BoxSplit bx, const int64_t *row_ptr, const uint32_t *rows,
                      const float4 *gtab, RunConst rc, McArgs a, R *pcache, McRec *rec, int finish_blocks,
                      int blocks_per_sm, cudaStream_t s, int64_t *launches);

// The fused pass of a float32 step with one categorical draw per DM particle (no row lists): the
// mean field of every gas row (part, then the float64 finish into out) and P_ij of every pair at
// its gas-major position (pg); then the Monte Carlo per DM row from pg through gidx (the DM-major
// rows' gas-major positions) and its float64 finish.  The results are those of launch_meanfield
// and launch_mc.
cudaError_t launch_pairs_fused(SpeciesView<float> G, SpeciesView<float> D, BoxSplit bx, const int64_t *row_ptr,
                               const uint32_t *rows, SegView sv, int64_t n_seg_max, const float4 *gtab, RunConst rc,
                               MfOut out, float *part, MlpRun mr, McArgs a, float *pg, int blocks_per_sm,
                               cudaStream_t s, int64_t *launches);
cudaError_t launch_mc_select(SpeciesView<float> D, SpeciesView<float> G, BoxSplit bx, const int64_t *row_ptr,
                             const uint32_t *rows, const uint32_t *gidx, const float *pg, const float4 *gtab,
                             RunConst rc, McArgs a, McRec *rec, int finish_blocks, int blocks_per_sm, cudaStream_t s,
                             int64_t *launches);

// Overlap table build (float64 exact evaluator at the nodes) and debug evaluators.
cudaError_t launch_gtable(float4 *T, cudaStream_t s, int64_t *launches);
cudaError_t launch_debug_overlap(const float4 *T, int fp64, int64_t k, const double *in, double *out, cudaStream_t s);
cudaError_t launch_debug_rates(int fp64, int n, int mode, double alpha, int64_t k, const double *in, double *out,
                               cudaStream_t s);
cudaError_t launch_debug_rates_screened(int fp64, double alpha0, int64_t k, const double *in, double *out,
                                        cudaStream_t s);
cudaError_t launch_debug_philox(int64_t k, const uint32_t *ctr, uint32_t *out, unsigned long long seed,
                                cudaStream_t s);
