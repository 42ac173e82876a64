// Pair search, mean field and Monte Carlo kernels.
#pragma once
#include "grid.cuh"

#define SR_UNIT 64   // target leaves per work unit of the tile stage

template <typename R>
cudaError_t launch_leaf_pairs(SpeciesView<R> Q, SpeciesView<R> O, BoxSplit bx, const Frame *frame, bool emit,
                              uint32_t *item_cnt, const int64_t *item_ptr, uint32_t *items, uint32_t *status,
                              unsigned long long *stats, cudaStream_t s, int64_t *launches);
cudaError_t launch_unit_counts(const int64_t *item_ptr, int nleaf, uint32_t *unit_cnt, cudaStream_t s,
                               int64_t *launches);
cudaError_t launch_unit_map(const int64_t *item_ptr, const int64_t *unit_ptr, int nleaf, uint32_t *unit_leaf,
                            int64_t *unit_item0, cudaStream_t s, int64_t *launches);
template <typename R>
cudaError_t launch_tile(SpeciesView<R> Q, SpeciesView<R> O, BoxSplit bx, const Frame *frame, bool emit,
                        const uint32_t *unit_leaf, const int64_t *unit_item0, const int64_t *item_ptr,
                        const uint32_t *items, int64_t n_units, uint32_t *unit_cnt, const int64_t *row_ptr,
                        uint32_t *rows, uint32_t *status, unsigned long long *stats, cudaStream_t s,
                        int64_t *launches);
cudaError_t launch_unit_prefix(const int64_t *unit_ptr, int nleaf, int64_t nq, uint32_t *unit_cnt, uint32_t *counts,
                               cudaStream_t s, int64_t *launches);

struct MfOut {
  double *acc;      // [N_B][3] caller order
  double *dudt;     // [N_B] caller order
  double *e_exp;    // [N_B] sorted order: M_j (cB sum tFB - cA sum tFA v_i.w) (no dt); may be null
};

template <typename R>
cudaError_t launch_meanfield(SpeciesView<R> G, SpeciesView<R> D, BoxSplit bx, const int64_t *row_ptr,
                             const uint32_t *rows, const float4 *gtab, RunConst rc, MfOut out, cudaStream_t s,
                             int64_t *launches);

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
  double *block_sums;         // [gridDim][8]: sum M dv (3), dKE, scatters, clamps, band, sum P
  double *block_max;          // [gridDim]: max p_ratio
};

template <typename R>
cudaError_t launch_mc(SpeciesView<R> D, SpeciesView<R> G, BoxSplit bx, const int64_t *row_ptr, const uint32_t *rows,
                      const float4 *gtab, RunConst rc, McArgs a, R *pcache, int blocks, cudaStream_t s,
                      int64_t *launches);

// Overlap table build (float64 exact evaluator at the nodes) and debug evaluators.
cudaError_t launch_gtable(float4 *T, cudaStream_t s, int64_t *launches);
cudaError_t launch_debug_overlap(const float4 *T, int fp64, int64_t k, const double *in, double *out, cudaStream_t s);
cudaError_t launch_debug_rates(int fp64, int n, int64_t k, const double *in, double *out, cudaStream_t s);
cudaError_t launch_debug_philox(int64_t k, const uint32_t *ctr, uint32_t *out, unsigned long long seed,
                                cudaStream_t s);
