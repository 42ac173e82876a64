// Tensor-core (tcgen05) inference of the learned rate surrogate: arguments and launchers.
#pragma once
#include <cuda_bf16.h>

#include "grid.cuh"
#include "mlp.cuh"


struct TcArgs {
  // network: float32 parameter block and the bf16 [out][in] copies of the 128 x 128 layers
  const float *p;
  const __nv_bfloat16 *w2, *w3;
  int64_t n;                       // rows
  // rows given directly: X [n][4] network inputs -> Y [n][2] raw outputs
  const float *X;
  float *Y;
  // rows = gas-major pairs: row q of the processing order lies in row k (largest k with
  // R_ptr[k] <= q) of n_rows rows; k is gas list[k] (or gas k when list is null) and the
  // pair index is p = row_ptr[gas] + q - R_ptr[k] (or q when list is null)
  const int64_t *R_ptr;
  int64_t n_rows;
  const uint32_t *list;
  const int64_t *row_ptr;
  const uint32_t *rows;            // DM index of pair p (sorted)
  const float4 *G_V, *D_V;         // sorted velocity copies (v, varsigma)
  const uint32_t *prow;            // row k of every q (set by the launcher)
  MlpDomain dom;
  RunConst rc;
  float2 *rates;                   // [pairs] (FA, FB)
  unsigned long long *fallback_count;
  uint32_t *status;                // DMB_BAD_TIMEOUT if a tensor-core wait gave up
  // limit of every wait on an MMA completion, ns (0: the default, about two seconds)
  unsigned long long wait_ns;
  // fault injection for the timeout path: warpgroup 0 of CTA 0 omits the commit of its first
  // layer-1 MMA, so its wait runs out; the launcher then uses a 1 ms limit
  int skip_commit;
  // captured steps: the row count lives on the device (n is then a capacity); null otherwise
  const int64_t *n_dev;
  // the mean field in the epilogue (mlp_tc_meanfield): sorted positions (hi, h) and (lo, M) of
  // both species, the gas box index (batched boxes, else null), the periodic boxes, the overlap
  // table, and the per-segment sums [slots][6] (slot = q / 32 + k for the rows of row k in the
  // 32 processing positions of one warp)
  const float4 *G_P, *G_L, *D_P, *D_L;
  const uint16_t *G_bid;
  BoxSplit bx;
  const float4 *gtab;
  float *part;
};

// Shared-memory attributes (call once before any graph capture).
cudaError_t mlp_tc_prepare();
// Raw network outputs of X (debug / validation entry).
// nwg: warpgroups (independent 128-row tiles in flight) per CTA, 2 to 4; with 2 the
// activations stay in tensor memory as the MMAs' A operand.
cudaError_t mlp_tc_infer(TcArgs a, int nwg, cudaStream_t s, int64_t *launches);
// Rates of the pairs in processing order; prow: scratch of n uint32 (the row of every q).
cudaError_t mlp_tc_pair_rates(TcArgs a, uint32_t *prow, int nwg, cudaStream_t s, int64_t *launches);
// The gas mean field (Eqs. gas-dVdt, gas-dTdt) of the same pairs with the rates never stored:
// each row's pair terms M_i g_ij (FA w, FA w^2, FB, FA v_i.w) are formed in the epilogue, summed
// per gas row over each warp's 32 rows (a segmented shuffle reduction in a fixed order) into
// a.part, and a float64 pass over the rows writes acc and du/dt (caller order, through perm) and
// the expected DM energy change e_exp (sorted order, may be null).  Rows without pairs get zeros.
// part holds (n >> 5) + n_rows + 1 slots of 6 floats.
cudaError_t mlp_tc_meanfield(TcArgs a, uint32_t *prow, int nwg, const float4 *G_K, const uint32_t *G_perm,
                             double *acc, double *dudt, double *e_exp, cudaStream_t s, int64_t *launches);
