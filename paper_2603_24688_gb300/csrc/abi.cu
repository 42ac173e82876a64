// C ABI: context, buffers and the launch sequences of the hybrid interaction step.
#include <ctype.h>
#include <math.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>

#include <chrono>
#include <random>
#include <vector>

#include "active.cuh"
#include "internal.cuh"
#include "mlp_host.cuh"
#include "mlp_tc.cuh"
#include "pairs.cuh"
#include "sort_scan.cuh"
#include "step.cuh"

namespace {

// Physical constants (CODATA 2018 / IAU); code units kpc, km/s, Msun.
const double kKB = 1.380649e-16;          // erg/K
const double kMP = 1.67262192369e-24;     // g
const double kKPC = 3.0856775814913673e21;  // cm
const double kMSUN = 1.98841e33;          // g

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

std::string g_create_error;

}  // namespace

struct SpeciesBufs {
  DevBuf keys0, keys1, vals0, vals1, P, L, V, K, sid, bmin, bmax, bid, leaf_box;
  int64_t n = 0;
  int levels = 0, nodes = 0;
  int off[DMB_MAX_LEVELS] = {0}, cnt[DMB_MAX_LEVELS] = {0};
};

// Pair-search scratch of one direction (queries of one species against the other's tree).
struct SearchBufs {
  DevBuf item_cnt, item_ptr, items, unit_cnt_leaf, unit_ptr, unit_leaf, unit_item0, unit_cnt, counts, row_ptr, rows,
      tmask;
  // float32 pair weights beside rows (PairWeights): gas-major M_i g_ij, DM-major g_ij
  DevBuf w;
  int64_t n_items = 0, n_units = 0, n_pairs = 0;
};

struct dmb_ctx {
  dmb_params p;
  cudaStream_t stream = nullptr;
  std::string err;
  RunConst rc;
  BoxSplit bx;
  int64_t launches = 0;
  // device state
  DevBuf frame, status, frame_part, gtab;
  SpeciesBufs dm, gas;
  DevBuf hist, hist_scan, scan_tmp;
  SearchBufs sg, sd;   // gas-major (gas queries, DM tree) and DM-major searches
  DevBuf pcache, mf_part, mc_rec, seg_cnt, seg_ptr, seg_row, seg_begin, t_cursor;
  // learned surrogate of the rate integrals
  DevBuf mlp_p, mlp_m, mlp_v, mlp_w2, mlp_w3, mlp_w2t, mlp_w3t, mlp_fallback, mlp_rates;
  bool mlp_ready = false;
  int mlp_engine = 0;            // 0: tcgen05 tiles (mlp_tc.cu), 1: warp-level mma.sync pass
  DevBuf tc_tiles;               // row of every pair of the surrogate's pass
  // dmb_set_surrogate_epilogue: 1 the tensor-core kernel forms the mean field in its epilogue
  // (per-warp row sums in tc_part), 0 (faster) it stores each pair's rates for the mean-field kernel
  int tc_epilogue = 0;
  DevBuf tc_part;
  bool tc_skip_commit = false;   // dmb_debug_tc_timeout: inject one timed-out wait into the next launch
  int device = 0;                // the CUDA device the context was created on
  // batched boxes (dmb_step_batched): caller box index arrays of the current build and tables
  const uint32_t *dm_box = nullptr, *gas_box = nullptr;
  int nbox = 0;
  double stride = 0.0;
  DevBuf box_sides, box_params;
  std::vector<int> mlp_n;        // power-law indices the network was trained for
  int mlp_family = 0;            // velocity law the network was trained for (0 power, 1 screened)
  int mlp_scope = 0;             // dmb_set_surrogate_scope: 0 the scan's indices and n, 1 n only
  int xsec = 0;                  // dmb_set_cross_section: 0 power law, 1 screened law
  double v_c = 0.0;              // its v_c, km/s
  double mlp_box[6] = {-2.0, 2.0, -3.0, 2.0, -0.30102999566398120, 1.0};   // log10 ranges of s, tau, m_chi
  int64_t n_seg_max = 0;
  int seg_len = MF_SEG, act_seg_len = MF_SEG;   // segment lengths the two segment tables were built with
  Shapes shp;                                   // launch shapes (defaults or dmb_autotune's choice)
  DevBuf mf_acc, mf_dudt, e_exp, mc_blocks, mc_max, kick_blocks, sums;
  DevBuf scratch_vel, search_stats, rebin_cnt;
  uint32_t *h_status = nullptr;   // pinned
  int64_t *h_tot = nullptr;       // pinned [8]
  double *h_sums = nullptr;       // pinned [16]
  // state
  bool grid_ready = false, pairs_ready = false;
  int64_t n_pairs = 0;
  const double *dm_vel = nullptr;   // caller DM velocities of the last build
  // hierarchical substeps (dmb_set_bins, dmb_substep): species lists ordered by (bin, sorted
  // index), the segment table of the gas list, and per bin boundary b (the active set of bins < b):
  // tab[0] DM count, tab[1] gas count, tab[2] gas segments, tab[3] pairs of the gas rows,
  // tab[4] pairs of the DM rows
  DevBuf act_dm, act_gas, act_start, act_seg_ptr, act_seg_row, act_seg_begin, act_len, act_segs, act_gpairs,
      act_dpairs, act_pick, step_dev, bin_keys, bin_keys1, bin_vals1;
  const uint8_t *dm_bin = nullptr, *gas_bin = nullptr;
  bool bins_ready = false;
  int64_t bin_tab[5][DMB_NBINS + 1];
  int64_t act_seg_total = 0;
  // CUDA graphs of substeps, one per (active-set boundary, dt, caller arrays)
  struct GraphEntry {
    int lim;
    double dt;
    const void *key[6];
    cudaGraphExec_t exec;
    int64_t launches;
  };
  bool use_graph = false;
  // the captured batched step (dmb_step_batched with dmb_set_graph(ctx, 1)): the graph of one
  // step for one set of caller arrays and boxes, and the buffer capacities it was sized for
  struct BatchCaps {
    int64_t items = 0, units = 0, pairs = 0, segs = 0;
  };
  struct BatchGraph {
    bool valid = false;
    const void *key[14] = {};
    int64_t nd = 0, ng = 0;
    double dt = 0.0;
    std::vector<dmb_box> boxes;
    BatchCaps caps;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
  } bgraph;
  bool capturing = false;           // a batched step is being captured: no allocation, no readback
  const int64_t *pairs_dev = nullptr;   // device pair total while capturing (surrogate row count)
  const uint32_t *gate_dev = nullptr;   // device overflow gate while capturing (kick)
  bool frame_ready = false;         // the batched frame was uploaded by dmb_step_batched
  uint64_t batch_next_step = ~0ull; // device step counter value after the last batched graph
  DevBuf gate, cap_need;
  DevBuf gidx;                      // gas-major position of every DM-major pair (the fused pass)
  bool fuse = false;                // dmb_set_fusion: one pass for the mean field and the Monte Carlo
  // dmb_set_pair_weights: -1 (auto) the float32 search stores pair weights when its pair set is
  // kept for later calls (dmb_neighbors); 0 never; 1 always.  w_ready: the current set has them.
  int weights_mode = -1;
  bool w_ready = false;
  int mc_variant = 0;             // dmb_set_mc_variant
  double mc_beta = 0.0;           // dmb_set_anisotropy
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  std::vector<GraphEntry> graphs;
  uint64_t graph_next_step = ~0ull;   // device step counter value, when known
  // optional stage timing with CUDA events on the context stream
  bool timing = false;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t sev[2] = {nullptr, nullptr};   // around the surrogate's pair pass (stage [5])
  bool sev_pending = false;
  double stage_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int64_t timed_steps = 0;
};

namespace {

dmb_status fail(dmb_ctx *c, dmb_status s, const std::string &msg) {
  if (c) c->err = msg; else g_create_error = msg;
  return s;
}

dmb_status cuda_fail(dmb_ctx *c, cudaError_t e, const char *where) {
  return fail(c, DMB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                    \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

bool ensure(DevBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return true;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  const size_t want = bytes + bytes / 8;   // a little slack so slowly growing sizes do not reallocate
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  b.bytes = want;
  return true;
}

void release(DevBuf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

template <typename T> T *ptr(const DevBuf &b) { return reinterpret_cast<T *>(b.p); }

int next_pow2(int64_t x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

template <typename R>
SpeciesView<R> view(const SpeciesBufs &s, bool batched = false) {
  SpeciesView<R> v;
  v.bid = batched ? ptr<uint16_t>(s.bid) : nullptr;
  v.leaf_box = batched ? ptr<int2>(s.leaf_box) : nullptr;
  v.n = s.n;
  v.P = ptr<typename Vec<R>::v4>(s.P);
  v.L = ptr<typename Vec<R>::v4>(s.L);
  v.V = ptr<typename Vec<R>::v4>(s.V);
  v.K = ptr<typename Vec<R>::v4>(s.K);
  v.id = ptr<uint32_t>(s.sid);
  v.perm = ptr<uint32_t>(s.vals0);
  v.bmin = ptr<float4>(s.bmin);
  v.bmax = ptr<float4>(s.bmax);
  v.levels = s.levels;
  for (int k = 0; k < DMB_MAX_LEVELS; ++k) { v.off[k] = s.off[k]; v.cnt[k] = s.cnt[k]; }
  return v;
}

void clear_graphs(dmb_ctx *ctx) {
  for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();
  ctx->graph_next_step = ~0ull;
}

// drops the captured batched step (its kernels hold the buffers and constants of its capture)
void clear_batch_graph(dmb_ctx *ctx) {
  if (ctx->bgraph.exec) cudaGraphExecDestroy(ctx->bgraph.exec);
  ctx->bgraph.exec = nullptr;
  ctx->bgraph.valid = false;
  ctx->batch_next_step = ~0ull;
}

// the grid or the pair lists change: substep tables and captured graphs are stale (the batched
// step's own capture rebuilds them inside the graph, which is why it keeps its graph)
void invalidate_substeps(dmb_ctx *ctx) {
  ctx->bins_ready = false;
  clear_graphs(ctx);
  if (!ctx->capturing) clear_batch_graph(ctx);
}

dmb_status ensure_species(dmb_ctx *ctx, SpeciesBufs &s, int64_t n, bool gas) {
  const size_t v4b = ctx->p.fp64 ? 32 : 16;
  s.n = n;
  s.nodes = tree_layout(n, &s.levels, s.off, s.cnt);
  bool ok = ensure(s.keys0, n * 8) && ensure(s.keys1, n * 8) && ensure(s.vals0, n * 4) && ensure(s.vals1, n * 4) &&
            ensure(s.P, n * v4b) && ensure(s.L, n * v4b) && ensure(s.V, n * v4b) && ensure(s.sid, n * 4) &&
            ensure(s.bmin, (size_t)s.nodes * 16) && ensure(s.bmax, (size_t)s.nodes * 16) && ensure(s.bid, n * 2 + 16) &&
            ensure(s.leaf_box, (size_t)s.cnt[0] * 8 + 16);
  if (gas) ok = ok && ensure(s.K, n * v4b);
  else ok = ok && ensure(s.K, 64);
  if (!ok) return fail(ctx, DMB_ERR_OOM, "device allocation failed for particle buffers");
  return DMB_OK;
}

dmb_status ensure_sort_scratch(dmb_ctx *ctx, int64_t n) {
  const int64_t hist_n = radix_hist_elems(n);
  const int64_t tmp_n = scan_tmp_elems(hist_n > n + 1 ? hist_n : n + 1);
  if (!ensure(ctx->hist, hist_n * 4) || !ensure(ctx->hist_scan, (hist_n + 1) * 8) || !ensure(ctx->scan_tmp, tmp_n * 8))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for sort scratch");
  return DMB_OK;
}

dmb_status check_status(dmb_ctx *ctx) {
  CK(cudaMemcpyAsync(ctx->h_status, ctx->status.p, 4, cudaMemcpyDeviceToHost, ctx->stream), "status readback");
  CK(cudaStreamSynchronize(ctx->stream), "synchronise");
  const uint32_t st = *ctx->h_status;
  if (st == 0) return DMB_OK;
  CK(cudaMemsetAsync(ctx->status.p, 0, 4, ctx->stream), "status reset");
  std::string m = "device input checks failed:";
  if (st & DMB_BAD_VALUE) m += " non-finite or out-of-range value (need finite x, v; h, M, mu > 0; T >= 0);";
  if (st & DMB_BAD_PERIODIC) m += " periodic box smaller than 2 (max h_dm + max h_gas);";
  if (st & DMB_BAD_DOMAIN) m += " rate provider outside its domain;";
  if (st & DMB_BAD_OVERFLOW) m += " internal list overflow;";
  if (st & DMB_BAD_TIMEOUT) m += " a tensor-core wait timed out;";
  return fail(ctx, (st & DMB_BAD_TIMEOUT) ? DMB_ERR_TIMEOUT : (st & DMB_BAD_DOMAIN) ? DMB_ERR_DOMAIN : DMB_ERR_ARG, m);
}

// ---- build_grid ------------------------------------------------------------------------
template <typename R>
dmb_status build_grid_impl(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas) {
  cudaStream_t s = ctx->stream;
  int64_t *L = &ctx->launches;
  dmb_status st;
  invalidate_substeps(ctx);
  if ((st = ensure_species(ctx, ctx->dm, dm->n, false)) != DMB_OK) return st;
  if ((st = ensure_species(ctx, ctx->gas, gas->n, true)) != DMB_OK) return st;
  if ((st = ensure_sort_scratch(ctx, dm->n > gas->n ? dm->n : gas->n)) != DMB_OK) return st;
  const bool batched = ctx->nbox > 0;
  const int64_t ntot = dm->n + gas->n;
  int bits = (int)fmin(21.0, fmax(10.0, ceil(log2((double)(ntot > 1 ? ntot : 2)) / 3.0) + 7.0));
  int box_bits = 0;
  if (batched) {
    // the frame of the virtual space (boxes side by side along x) was set up by dmb_step_batched
    while ((1 << box_bits) < ctx->nbox) ++box_bits;
    bits = (int)fmin((double)bits, floor((63.0 - box_bits) / 3.0));
    if (!ctx->frame_ready) return fail(ctx, DMB_ERR_STATE, "batched frame missing");
  } else {
    CK(launch_frame(dm->pos, dm->h, dm->n, gas->pos, gas->h, gas->n, ctx->p.periodic, ctx->p.box,
                    ptr<double>(ctx->frame_part), (int64_t)(ctx->frame_part.bytes / 8), ptr<Frame>(ctx->frame),
                    ptr<uint32_t>(ctx->status), s, L), "frame");
  }
  const Frame *fr = ptr<Frame>(ctx->frame);
  SpeciesBufs *sp[2] = {&ctx->dm, &ctx->gas};
  const double *pos[2] = {dm->pos, gas->pos};
  const double *vel[2] = {dm->vel, gas->vel};
  const double *mass[2] = {dm->mass, gas->mass};
  const double *hh[2] = {dm->h, gas->h};
  const double *T[2] = {nullptr, gas->T};
  const double *mu[2] = {nullptr, gas->mu};
  const uint32_t *id[2] = {dm->id, gas->id};
  const uint32_t *box_of[2] = {ctx->dm_box, ctx->gas_box};
  for (int k = 0; k < 2; ++k) {
    SpeciesBufs &b = *sp[k];
    BatchArgs ba;
    ba.box_of = batched ? box_of[k] : nullptr;
    ba.bp = batched ? ptr<BoxParamDev>(ctx->box_params) : nullptr;
    ba.box_bits = box_bits;
    if (b.n > 0) {
      CK(launch_morton(pos[k], b.n, ctx->p.periodic, ctx->p.box, fr, ba, ptr<uint64_t>(b.keys0), ptr<uint32_t>(b.vals0),
                       s, L), "morton");
      CK(radix_sort_pairs(ptr<uint64_t>(b.keys0), ptr<uint32_t>(b.vals0), ptr<uint64_t>(b.keys1),
                          ptr<uint32_t>(b.vals1), b.n, 3 * bits + box_bits, ptr<uint32_t>(ctx->hist),
                          ptr<int64_t>(ctx->hist_scan), ptr<int64_t>(ctx->scan_tmp), s, L), "radix sort");
      CK(launch_gather<R>(pos[k], vel[k], mass[k], hh[k], T[k], mu[k], id[k], b.n, ptr<uint32_t>(b.vals0),
                          ctx->p.periodic, ctx->p.box, fr, ctx->rc, ba, ptr<typename Vec<R>::v4>(b.P),
                          ptr<typename Vec<R>::v4>(b.L), ptr<typename Vec<R>::v4>(b.V),
                          ptr<typename Vec<R>::v4>(b.K), ptr<uint32_t>(b.sid), ptr<uint16_t>(b.bid),
                          ptr<uint32_t>(ctx->status), s, L), "gather");
    }
    CK(launch_tree<R>(ptr<typename Vec<R>::v4>(b.P), ptr<typename Vec<R>::v4>(b.L), b.n, fr, ptr<float4>(b.bmin),
                      ptr<float4>(b.bmax), b.levels, b.off, b.cnt, batched ? ptr<uint16_t>(b.bid) : nullptr,
                      ptr<int2>(b.leaf_box), s, L), "tree");
  }
  ctx->dm_vel = dm->vel;
  ctx->grid_ready = true;
  ctx->pairs_ready = false;
  ctx->w_ready = false;
  return DMB_OK;
}

// ---- neighbours --------------------------------------------------------------------------
// Stage 1 (candidate leaves) and the unit layout for one direction; needs no host sizes.
template <typename R>
dmb_status search_stage1_count(dmb_ctx *ctx, SearchBufs &sb, SpeciesView<R> Q, SpeciesView<R> O,
                               unsigned long long *stats) {
  cudaStream_t s = ctx->stream;
  int64_t *L = &ctx->launches;
  const int nleaf = Q.cnt[0];
  if (!ensure(sb.item_cnt, (size_t)nleaf * 4) || !ensure(sb.item_ptr, (size_t)(nleaf + 1) * 8) ||
      !ensure(sb.unit_cnt_leaf, (size_t)nleaf * 4) || !ensure(sb.unit_ptr, (size_t)(nleaf + 1) * 8) ||
      !ensure(sb.counts, (size_t)(Q.n + 1) * 4) || !ensure(sb.row_ptr, (size_t)(Q.n + 1) * 8))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for search offsets");
  const Frame *fr = ptr<Frame>(ctx->frame);
  uint32_t *status = ptr<uint32_t>(ctx->status);
  CK(launch_leaf_pairs<R>(Q, O, ctx->bx, fr, false, ptr<uint32_t>(sb.item_cnt), nullptr, nullptr, status, stats, s, L),
     "leaf pairs (count)");
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(sb.item_cnt), ptr<int64_t>(sb.item_ptr), nleaf, ptr<int64_t>(ctx->scan_tmp),
                            s, L), "scan");
  CK(launch_unit_counts(ptr<int64_t>(sb.item_ptr), nleaf, ctx->shp.unit, ptr<uint32_t>(sb.unit_cnt_leaf), s, L),
     "unit counts");
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(sb.unit_cnt_leaf), ptr<int64_t>(sb.unit_ptr), nleaf,
                            ptr<int64_t>(ctx->scan_tmp), s, L), "scan");
  return DMB_OK;
}

template <typename R>
dmb_status search_stage2_count(dmb_ctx *ctx, SearchBufs &sb, SpeciesView<R> Q, SpeciesView<R> O,
                               unsigned long long *stats, TransposeOut tr) {
  cudaStream_t s = ctx->stream;
  int64_t *L = &ctx->launches;
  const int nleaf = Q.cnt[0];
  if (!ensure(sb.items, (size_t)sb.n_items * 4) || !ensure(sb.unit_leaf, (size_t)sb.n_units * 4) ||
      !ensure(sb.unit_item0, (size_t)sb.n_units * 8) || !ensure(sb.unit_cnt, (size_t)sb.n_units * 32 * 4) ||
      !ensure(sb.tmask, (size_t)sb.n_items * 32 * 4))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for search lists");
  const Frame *fr = ptr<Frame>(ctx->frame);
  uint32_t *status = ptr<uint32_t>(ctx->status);
  CK(launch_leaf_pairs<R>(Q, O, ctx->bx, fr, true, nullptr, ptr<int64_t>(sb.item_ptr), ptr<uint32_t>(sb.items), status,
                          nullptr, s, L), "leaf pairs (emit)");
  CK(launch_unit_map(ptr<int64_t>(sb.item_ptr), ptr<int64_t>(sb.unit_ptr), nleaf, ctx->shp.unit, ptr<uint32_t>(sb.unit_leaf),
                     ptr<int64_t>(sb.unit_item0), s, L), "unit map");
  CK(launch_tile<R>(Q, O, ctx->bx, fr, false, ptr<uint32_t>(sb.unit_leaf), ptr<int64_t>(sb.unit_item0),
                    ptr<int64_t>(sb.item_ptr), ptr<uint32_t>(sb.items), sb.n_units, ctx->shp.unit,
                    ptr<uint32_t>(sb.unit_cnt), nullptr, nullptr, tr, ptr<uint32_t>(sb.tmask), status, stats, s, L),
     "tile (count)");
  CK(launch_unit_prefix(ptr<int64_t>(sb.unit_ptr), nleaf, Q.n, ptr<uint32_t>(sb.unit_cnt), ptr<uint32_t>(sb.counts), s,
                        L), "unit prefix");
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(sb.counts), ptr<int64_t>(sb.row_ptr), Q.n, ptr<int64_t>(ctx->scan_tmp), s, L),
     "scan");
  return DMB_OK;
}

template <typename R>
dmb_status search_stage2_emit(dmb_ctx *ctx, SearchBufs &sb, SpeciesView<R> Q, SpeciesView<R> O, TransposeOut tr,
                              PairWeights pw) {
  if (!ensure(sb.rows, (size_t)sb.n_pairs * 4)) return fail(ctx, DMB_ERR_OOM, "device allocation failed for pair lists");
  CK(launch_tile<R>(Q, O, ctx->bx, ptr<Frame>(ctx->frame), true, ptr<uint32_t>(sb.unit_leaf),
                    ptr<int64_t>(sb.unit_item0), ptr<int64_t>(sb.item_ptr), ptr<uint32_t>(sb.items), sb.n_units,
                    ctx->shp.unit, ptr<uint32_t>(sb.unit_cnt), ptr<int64_t>(sb.row_ptr), ptr<uint32_t>(sb.rows), tr,
                    ptr<uint32_t>(sb.tmask), ptr<uint32_t>(ctx->status), nullptr, ctx->stream, &ctx->launches, nullptr,
                    pw),
     "tile (emit)");
  return DMB_OK;
}

// The pair weights of a float32 search (none in float64, whose kernels evaluate g exactly).
template <typename R>
PairWeights pair_weights(dmb_ctx *ctx) {
  PairWeights pw;
  if (sizeof(R) == 4) {
    pw.q = ptr<float>(ctx->sg.w);
    pw.t = ptr<float>(ctx->sd.w);
    pw.gtab = ptr<float4>(ctx->gtab);
  }
  return pw;
}
// The weights the mean field and the Monte Carlo read: those of the current pair set, if any.
template <typename R>
PairWeights ready_weights(dmb_ctx *ctx) {
  return ctx->w_ready ? pair_weights<R>(ctx) : PairWeights();
}
// Whether a search stores weights: reuse = the pair set outlives the call that searched it.
template <typename R>
bool want_weights(const dmb_ctx *ctx, bool reuse) {
  return sizeof(R) == 4 && (ctx->weights_mode == 1 || (ctx->weights_mode == -1 && reuse));
}

// Mean-field segments of the gas rows (upper bound N_B + pairs / seg, no readback).
dmb_status build_segments(dmb_ctx *ctx, const SearchBufs &sg, int64_t ng) {
  cudaStream_t s = ctx->stream;
  int64_t *L = &ctx->launches;
  const int seg = ctx->shp.seg;
  const int64_t nmax = ng + sg.n_pairs / seg + 1;
  if (!ensure(ctx->seg_cnt, (size_t)(ng + 1) * 4) || !ensure(ctx->seg_ptr, (size_t)(ng + 1) * 8) ||
      !ensure(ctx->seg_row, (size_t)nmax * 4) || !ensure(ctx->seg_begin, (size_t)nmax * 8))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for mean-field segments");
  CK(launch_seg_counts(ptr<int64_t>(sg.row_ptr), ng, seg, ptr<uint32_t>(ctx->seg_cnt), s, L), "segments");
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(ctx->seg_cnt), ptr<int64_t>(ctx->seg_ptr), ng, ptr<int64_t>(ctx->scan_tmp),
                            s, L), "scan");
  CK(launch_seg_map(ptr<int64_t>(sg.row_ptr), ptr<int64_t>(ctx->seg_ptr), ng, seg, ptr<uint32_t>(ctx->seg_row),
                    ptr<int64_t>(ctx->seg_begin), s, L), "segment map");
  ctx->n_seg_max = nmax;
  ctx->seg_len = seg;
  return DMB_OK;
}

template <typename R>
dmb_status neighbors_impl(dmb_ctx *ctx, bool reuse = false) {
  cudaStream_t s = ctx->stream;
  const SpeciesView<R> D = view<R>(ctx->dm, ctx->nbox > 0), G = view<R>(ctx->gas, ctx->nbox > 0);
  const int64_t nmax = D.n > G.n ? D.n : G.n;
  dmb_status st;
  invalidate_substeps(ctx);
  if ((st = ensure_sort_scratch(ctx, nmax + 1)) != DMB_OK) return st;
  unsigned long long *sst = ptr<unsigned long long>(ctx->search_stats);
  CK(cudaMemsetAsync(sst, 0, 16 * 8, s), "stats reset");
  SearchBufs &sg = ctx->sg, &sd = ctx->sd;
  // gas-major search: stage 1 counts, one readback of the list sizes
  if ((st = search_stage1_count<R>(ctx, sg, G, D, sst)) != DMB_OK) return st;
  CK(cudaMemcpyAsync(ctx->h_tot + 0, ptr<int64_t>(sg.item_ptr) + G.cnt[0], 8, cudaMemcpyDeviceToHost, s), "readback");
  CK(cudaMemcpyAsync(ctx->h_tot + 1, ptr<int64_t>(sg.unit_ptr) + G.cnt[0], 8, cudaMemcpyDeviceToHost, s), "readback");
  if ((st = check_status(ctx)) != DMB_OK) return st;
  sg.n_items = ctx->h_tot[0];
  sg.n_units = ctx->h_tot[1];
  // stage 2 counts in both directions (the DM-major counts from per-tile column sums), then
  // the pair total
  const int64_t nd = D.n;
  if (!ensure(sd.counts, (size_t)(nd + 1) * 4) || !ensure(sd.row_ptr, (size_t)(nd + 1) * 8) ||
      !ensure(ctx->t_cursor, (size_t)(nd + 1) * 4))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for DM-major lists");
  CK(cudaMemsetAsync(sd.counts.p, 0, (size_t)(nd + 1) * 4, s), "memset");
  TransposeOut trc;
  trc.cnt = ptr<uint32_t>(sd.counts);
  if ((st = search_stage2_count<R>(ctx, sg, G, D, sst, trc)) != DMB_OK) return st;
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(sd.counts), ptr<int64_t>(sd.row_ptr), nd, ptr<int64_t>(ctx->scan_tmp), s,
                            &ctx->launches), "scan");
  CK(cudaMemcpyAsync(ctx->h_tot + 4, ptr<int64_t>(sg.row_ptr) + G.n, 8, cudaMemcpyDeviceToHost, s), "readback");
  CK(cudaMemcpyAsync(ctx->h_tot + 5, ptr<int64_t>(sd.row_ptr) + nd, 8, cudaMemcpyDeviceToHost, s), "readback");
  if ((st = check_status(ctx)) != DMB_OK) return st;
  sg.n_pairs = G.n > 0 ? ctx->h_tot[4] : 0;
  sd.n_pairs = nd > 0 ? ctx->h_tot[5] : 0;
  if (sd.n_pairs != sg.n_pairs) return fail(ctx, DMB_ERR_CUDA, "pair counts of the two directions differ");
  // emit both directions: gas-major rows in search order, DM-major rows by claimed positions
  const bool w = want_weights<R>(ctx, reuse);
  if (!ensure(sd.rows, (size_t)sg.n_pairs * 4) || (ctx->fuse && !ensure(ctx->gidx, (size_t)sg.n_pairs * 4)) ||
      (w && (!ensure(sg.w, (size_t)sg.n_pairs * 4 + 16) || !ensure(sd.w, (size_t)sg.n_pairs * 4 + 16))))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for DM-major lists");
  CK(cudaMemsetAsync(ctx->t_cursor.p, 0, (size_t)(nd + 1) * 4, s), "memset");
  TransposeOut tre;
  tre.cursor = ptr<uint32_t>(ctx->t_cursor);
  tre.ptr = ptr<int64_t>(sd.row_ptr);
  tre.rows = ptr<uint32_t>(sd.rows);
  tre.gidx = ctx->fuse ? ptr<uint32_t>(ctx->gidx) : nullptr;   // only the fused step reads them
  if ((st = search_stage2_emit<R>(ctx, sg, G, D, tre, w ? pair_weights<R>(ctx) : PairWeights())) != DMB_OK)
    return st;
  ctx->w_ready = w;
  if ((st = build_segments(ctx, sg, G.n)) != DMB_OK) return st;
  if (!ensure(ctx->pcache, (size_t)sd.n_pairs * (ctx->p.fp64 ? 8 : 4)))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for the probability cache");
  ctx->n_pairs = sg.n_pairs;
  ctx->pairs_ready = true;
  return DMB_OK;
}

// The pair search of a captured batched step: the launches of neighbors_impl with every buffer
// sized in advance to the capacities of ctx->bgraph.caps and no count read back.  After each
// scan a capacity check compares the device total with its capacity; on overflow it clears
// the offsets (every later kernel sees empty rows), raises the gate (the kick changes nothing)
// and records the totals, from which the host regrows the buffers and repeats the step.
template <typename R>
dmb_status neighbors_capped(dmb_ctx *ctx) {
  cudaStream_t s = ctx->stream;
  int64_t *L = &ctx->launches;
  const dmb_ctx::BatchCaps &cap = ctx->bgraph.caps;
  const SpeciesView<R> D = view<R>(ctx->dm, true), G = view<R>(ctx->gas, true);
  SearchBufs &sg = ctx->sg, &sd = ctx->sd;
  const int nleaf = G.cnt[0];
  const int64_t nd = D.n, ng = G.n;
  const Frame *fr = ptr<Frame>(ctx->frame);
  uint32_t *status = ptr<uint32_t>(ctx->status);
  CapCheck base;
  base.need = ptr<int64_t>(ctx->cap_need);
  base.gate = ptr<uint32_t>(ctx->gate);
  base.status = status;
  int64_t *item_ptr = ptr<int64_t>(sg.item_ptr), *unit_ptr = ptr<int64_t>(sg.unit_ptr);
  // stage 1: candidate leaves per query leaf and the work units
  CK(launch_leaf_pairs<R>(G, D, ctx->bx, fr, false, ptr<uint32_t>(sg.item_cnt), nullptr, nullptr, status, nullptr, s,
                          L), "leaf pairs (count)");
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(sg.item_cnt), item_ptr, nleaf, ptr<int64_t>(ctx->scan_tmp), s, L), "scan");
  CK(launch_unit_counts(item_ptr, nleaf, ctx->shp.unit, ptr<uint32_t>(sg.unit_cnt_leaf), s, L), "unit counts");
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(sg.unit_cnt_leaf), unit_ptr, nleaf, ptr<int64_t>(ctx->scan_tmp), s, L),
     "scan");
  CapCheck c1 = base;
  c1.total[0] = item_ptr + nleaf; c1.cap[0] = cap.items; c1.slot[0] = 0; c1.zero[0] = item_ptr; c1.zero_n[0] = nleaf + 1;
  c1.total[1] = unit_ptr + nleaf; c1.cap[1] = cap.units; c1.slot[1] = 1; c1.zero[1] = unit_ptr; c1.zero_n[1] = nleaf + 1;
  CK(launch_cap_check(c1, s, L), "capacity check");
  // stage 2, count pass (both directions' counts)
  CK(cudaMemsetAsync(sd.counts.p, 0, (size_t)(nd + 1) * 4, s), "memset");
  TransposeOut trc;
  trc.cnt = ptr<uint32_t>(sd.counts);
  CK(launch_leaf_pairs<R>(G, D, ctx->bx, fr, true, nullptr, item_ptr, ptr<uint32_t>(sg.items), status, nullptr, s, L),
     "leaf pairs (emit)");
  CK(launch_unit_map(item_ptr, unit_ptr, nleaf, ctx->shp.unit, ptr<uint32_t>(sg.unit_leaf), ptr<int64_t>(sg.unit_item0),
                     s, L), "unit map");
  CK(launch_tile<R>(G, D, ctx->bx, fr, false, ptr<uint32_t>(sg.unit_leaf), ptr<int64_t>(sg.unit_item0), item_ptr,
                    ptr<uint32_t>(sg.items), cap.units, ctx->shp.unit, ptr<uint32_t>(sg.unit_cnt), nullptr, nullptr,
                    trc, ptr<uint32_t>(sg.tmask), status, nullptr, s, L, unit_ptr + nleaf), "tile (count)");
  CK(launch_unit_prefix(unit_ptr, nleaf, ng, ptr<uint32_t>(sg.unit_cnt), ptr<uint32_t>(sg.counts), s, L),
     "unit prefix");
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(sg.counts), ptr<int64_t>(sg.row_ptr), ng, ptr<int64_t>(ctx->scan_tmp), s, L),
     "scan");
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(sd.counts), ptr<int64_t>(sd.row_ptr), nd, ptr<int64_t>(ctx->scan_tmp), s, L),
     "scan");
  CapCheck c2 = base;
  c2.total[0] = ptr<int64_t>(sg.row_ptr) + ng; c2.cap[0] = cap.pairs; c2.slot[0] = 2;
  c2.zero[0] = ptr<int64_t>(sg.row_ptr); c2.zero_n[0] = ng + 1;
  c2.total[1] = ptr<int64_t>(sd.row_ptr) + nd; c2.cap[1] = cap.pairs; c2.slot[1] = 2;
  c2.zero[1] = ptr<int64_t>(sd.row_ptr); c2.zero_n[1] = nd + 1;
  CK(launch_cap_check(c2, s, L), "capacity check");
  // emit pass: gas-major rows and the DM-major rows by claimed positions
  CK(cudaMemsetAsync(ctx->t_cursor.p, 0, (size_t)(nd + 1) * 4, s), "memset");
  TransposeOut tre;
  tre.cursor = ptr<uint32_t>(ctx->t_cursor);
  tre.ptr = ptr<int64_t>(sd.row_ptr);
  tre.rows = ptr<uint32_t>(sd.rows);
  tre.gidx = ctx->fuse ? ptr<uint32_t>(ctx->gidx) : nullptr;
  CK(launch_tile<R>(G, D, ctx->bx, fr, true, ptr<uint32_t>(sg.unit_leaf), ptr<int64_t>(sg.unit_item0), item_ptr,
                    ptr<uint32_t>(sg.items), cap.units, ctx->shp.unit, ptr<uint32_t>(sg.unit_cnt),
                    ptr<int64_t>(sg.row_ptr), ptr<uint32_t>(sg.rows), tre, ptr<uint32_t>(sg.tmask), status, nullptr, s,
                    L, unit_ptr + nleaf, want_weights<R>(ctx, false) ? pair_weights<R>(ctx) : PairWeights()),
     "tile (emit)");
  ctx->w_ready = want_weights<R>(ctx, false);
  // mean-field segments
  const int seg = ctx->shp.seg;
  CK(launch_seg_counts(ptr<int64_t>(sg.row_ptr), ng, seg, ptr<uint32_t>(ctx->seg_cnt), s, L), "segments");
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(ctx->seg_cnt), ptr<int64_t>(ctx->seg_ptr), ng, ptr<int64_t>(ctx->scan_tmp),
                            s, L), "scan");
  CapCheck c3 = base;
  c3.total[0] = ptr<int64_t>(ctx->seg_ptr) + ng; c3.cap[0] = cap.segs; c3.slot[0] = 3;
  c3.zero[0] = ptr<int64_t>(ctx->seg_ptr); c3.zero_n[0] = ng + 1;
  CK(launch_cap_check(c3, s, L), "capacity check");
  CK(launch_seg_map(ptr<int64_t>(sg.row_ptr), ptr<int64_t>(ctx->seg_ptr), ng, seg, ptr<uint32_t>(ctx->seg_row),
                    ptr<int64_t>(ctx->seg_begin), s, L), "segment map");
  ctx->n_seg_max = cap.segs;
  ctx->seg_len = seg;
  sg.n_items = cap.items;
  sg.n_units = cap.units;
  sg.n_pairs = sd.n_pairs = ctx->n_pairs = cap.pairs;
  ctx->pairs_ready = true;
  return DMB_OK;
}

// ---- surrogate helpers ---------------------------------------------------------------------
double alpha_of(int n) { return pow(2.0, (n + 5) / 2.0) * tgamma(3.0 + n / 2.0) / sqrt(M_PI); }

// Envelope E(x) = (1 + p x + q x^2 + r x^3)^m of F = 1F1(a, b; -x) with e = -a != 0 (FA: a = -(n+1)/2,
// b = 5/2; FB: a = -(n+3)/2, b = 3/2), m = e/3: r carries the large-x limit F -> Gamma(b)/Gamma(b+e) x^-e
// (DLMF 13.7.2), p and q the first two Taylor coefficients F = 1 + (e/b) x + e(e-1)/(2b(b+1)) x^2 + ...
// (DLMF 13.2.2), so the network's target log F - log E vanishes at both ends as O(x^3) and O(1/x);
// q is kept >= 0 so that the cubic stays positive.  e = 0: E = 1.  env = {p, q, r, m}.
void envelope_of(double a, double b, double env[4]) {
  const double e = -a;
  if (e == 0.0) {
    env[0] = env[1] = env[2] = env[3] = 0.0;
    return;
  }
  const double m = e / 3.0, k1 = e / b, k2 = e * (e - 1.0) / (2.0 * b * (b + 1.0));
  const double pc = k1 / m;
  env[0] = pc;
  env[1] = fmax((k2 - 0.5 * k1 * k1) / m + 0.5 * pc * pc, 0.0);
  env[2] = pow(tgamma(b) / tgamma(b + e), 1.0 / m);
  env[3] = m;
}
void envelope(int n, double envA[4], double envB[4]) {
  envelope_of(-(n + 1) / 2.0, 2.5, envA);
  envelope_of(-(n + 3) / 2.0, 1.5, envB);
}

dmb_status ensure_mlp(dmb_ctx *ctx) {
  const size_t np = MLP_NPARAM * 4, nw = MLP_H * MLP_H * 2;
  if (!ensure(ctx->mlp_p, np) || !ensure(ctx->mlp_m, np) || !ensure(ctx->mlp_v, np) || !ensure(ctx->mlp_w2, nw) ||
      !ensure(ctx->mlp_w3, nw) || !ensure(ctx->mlp_w2t, nw) || !ensure(ctx->mlp_w3t, nw) ||
      !ensure(ctx->mlp_fallback, 16))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for the surrogate");
  return DMB_OK;
}

MlpDev mlp_dev(dmb_ctx *ctx) {
  MlpDev d;
  d.p = ptr<float>(ctx->mlp_p);
  d.m = ptr<float>(ctx->mlp_m);
  d.v = ptr<float>(ctx->mlp_v);
  d.w2 = ptr<__nv_bfloat16>(ctx->mlp_w2);
  d.w3 = ptr<__nv_bfloat16>(ctx->mlp_w3);
  d.w2t = ptr<__nv_bfloat16>(ctx->mlp_w2t);
  d.w3t = ptr<__nv_bfloat16>(ctx->mlp_w3t);
  return d;
}

// whether the loaded network was trained for the context's velocity law (and power-law index)
bool surrogate_covers(const dmb_ctx *ctx) {
  if (ctx->mlp_family != ctx->xsec) return false;
  if (ctx->xsec == 1) return true;
  bool known = false;
  for (int k : ctx->mlp_n) known = known || k == ctx->p.n;
  return known;
}

MlpRun mlp_run(dmb_ctx *ctx) {
  MlpRun r;
  r.p = ptr<float>(ctx->mlp_p);
  r.w2 = ptr<__nv_bfloat16>(ctx->mlp_w2);
  r.w3 = ptr<__nv_bfloat16>(ctx->mlp_w3);
  r.fallback_count = ptr<unsigned long long>(ctx->mlp_fallback);
  MlpDomain &d = r.dom;
  d.s2_lo = (float)pow(10.0, 2.0 * ctx->mlp_box[0]);
  d.s2_hi = (float)pow(10.0, 2.0 * ctx->mlp_box[1]);
  d.tau_lo = (float)pow(10.0, ctx->mlp_box[2]);
  d.tau_hi = (float)pow(10.0, ctx->mlp_box[3]);
  d.m_lo = (float)pow(10.0, ctx->mlp_box[4]);
  d.m_hi = (float)pow(10.0, ctx->mlp_box[5]);
  double envA[4], envB[4];
  envelope(ctx->rc.n, envA, envB);
  for (int k = 0; k < 4; ++k) {
    d.envA[k] = (float)envA[k];
    d.envB[k] = (float)envB[k];
  }
  // the second input: varsigma^2 / v0^2 for the power law, varsigma^2 / v_c^2 for the screened law
  d.inv_v0sq = ctx->xsec == 1 ? (float)(1.0 / (ctx->v_c * ctx->v_c)) : (float)(1.0 / (ctx->p.v0_kms * ctx->p.v0_kms));
  d.log_m = (float)log10(ctx->p.m_chi_mp);
  d.n4 = (float)(0.25 * ctx->rc.n);
  d.scr = ctx->xsec == 1 ? 1 : 0;
  return r;
}

// Surrogate rates of the gas-major pairs in processing order q < n_q: rows k < n_rows of the
// prefix R_ptr (gas list[k], or gas k without a list); sv is the same rows' segment view.
dmb_status surrogate_rates(dmb_ctx *ctx, const MlpRun &mr, const SegView &sv, const int64_t *R_ptr, int64_t n_rows,
                           const uint32_t *list, int64_t n_q) {
  if (n_q <= 0 || n_rows <= 0) return DMB_OK;
  cudaStream_t s = ctx->stream;
  if (ctx->mlp_engine == 0) {
    TcArgs a = {};
    a.p = mr.p;
    a.w2 = mr.w2;
    a.w3 = mr.w3;
    a.n = n_q;
    a.R_ptr = R_ptr;
    a.n_rows = n_rows;
    a.list = list;
    a.row_ptr = ptr<int64_t>(ctx->sg.row_ptr);
    a.rows = ptr<uint32_t>(ctx->sg.rows);
    a.G_V = ptr<float4>(ctx->gas.V);
    a.D_V = ptr<float4>(ctx->dm.V);
    a.dom = mr.dom;
    a.rc = ctx->rc;
    a.rates = ptr<float2>(ctx->mlp_rates);
    a.fallback_count = mr.fallback_count;
    a.status = ptr<uint32_t>(ctx->status);
    a.skip_commit = ctx->tc_skip_commit ? 1 : 0;
    ctx->tc_skip_commit = false;
    a.n_dev = ctx->capturing ? ctx->pairs_dev : nullptr;
    if (!ensure(ctx->tc_tiles, (size_t)n_q * 4)) return fail(ctx, DMB_ERR_OOM, "surrogate pair rows");
    CK(mlp_tc_pair_rates(a, ptr<uint32_t>(ctx->tc_tiles), ctx->shp.tc_wg, s, &ctx->launches),
       "surrogate rates (tensor cores)");
  } else {
    CK(launch_mlp_pair_rates(view<float>(ctx->gas, ctx->nbox > 0), view<float>(ctx->dm, ctx->nbox > 0),
                             ptr<int64_t>(ctx->sg.row_ptr), ptr<uint32_t>(ctx->sg.rows), sv,
                             sv.n_seg >= 0 ? sv.n_seg : ctx->n_seg_max, ctx->rc, mr, ptr<float2>(ctx->mlp_rates), s,
                             &ctx->launches), "surrogate rates");
  }
  return DMB_OK;
}

// Whether a float32 mean field with the surrogate runs in the tensor-core kernel's epilogue.
template <typename R>
bool surrogate_epilogue(const dmb_ctx *ctx) {
  return sizeof(R) == 4 && ctx->rc.rate_mode == DMB_RATE_MLP && ctx->mlp_engine == 0 && ctx->tc_epilogue == 1;
}

// The gas mean field of rows k < n_rows of the prefix R_ptr (gas list[k], or gas k without a
// list) with the surrogate's rates formed and used inside the tensor-core kernel (no rates
// stored), then the float64 finish into o.
dmb_status surrogate_meanfield(dmb_ctx *ctx, const MlpRun &mr, const int64_t *R_ptr, int64_t n_rows,
                               const uint32_t *list, int64_t n_q, const MfOut &o) {
  if (n_rows <= 0) return DMB_OK;
  TcArgs a = {};
  a.p = mr.p;
  a.w2 = mr.w2;
  a.w3 = mr.w3;
  a.n = n_q;
  a.R_ptr = R_ptr;
  a.n_rows = n_rows;
  a.list = list;
  a.row_ptr = ptr<int64_t>(ctx->sg.row_ptr);
  a.rows = ptr<uint32_t>(ctx->sg.rows);
  a.G_V = ptr<float4>(ctx->gas.V);
  a.D_V = ptr<float4>(ctx->dm.V);
  a.dom = mr.dom;
  a.rc = ctx->rc;
  a.fallback_count = mr.fallback_count;
  a.status = ptr<uint32_t>(ctx->status);
  a.skip_commit = ctx->tc_skip_commit ? 1 : 0;
  ctx->tc_skip_commit = false;
  a.n_dev = ctx->capturing ? ctx->pairs_dev : nullptr;
  const SpeciesView<float> G = view<float>(ctx->gas, ctx->nbox > 0), D = view<float>(ctx->dm, ctx->nbox > 0);
  a.G_P = G.P;
  a.G_L = G.L;
  a.D_P = D.P;
  a.D_L = D.L;
  a.G_bid = G.bid;
  a.bx = ctx->bx;
  a.gtab = ptr<float4>(ctx->gtab);
  const int64_t nq = n_q > 0 ? n_q : 0;
  if (!ensure(ctx->tc_tiles, (size_t)nq * 4 + 16) || !ensure(ctx->tc_part, ((size_t)(nq >> 5) + n_rows + 1) * 24))
    return fail(ctx, DMB_ERR_OOM, "surrogate mean-field scratch");
  a.part = ptr<float>(ctx->tc_part);
  CK(mlp_tc_meanfield(a, ptr<uint32_t>(ctx->tc_tiles), ctx->shp.tc_wg, G.K, G.perm, o.acc, o.dudt, o.e_exp,
                      ctx->stream, &ctx->launches),
     "surrogate mean field (tensor cores)");
  return DMB_OK;
}

template <typename R>
dmb_status meanfield_impl(dmb_ctx *ctx, double *acc, double *dudt, double *e_exp) {
  const SpeciesView<R> D = view<R>(ctx->dm, ctx->nbox > 0), G = view<R>(ctx->gas, ctx->nbox > 0);
  MfOut o;
  o.acc = acc;
  o.dudt = dudt;
  o.e_exp = e_exp;
  if (!ensure(ctx->mf_part, (size_t)ctx->n_seg_max * 6 * sizeof(R))) return fail(ctx, DMB_ERR_OOM, "mean-field scratch");
  SegView sv;
  sv.seg_ptr = ptr<int64_t>(ctx->seg_ptr);
  sv.seg_row = ptr<uint32_t>(ctx->seg_row);
  sv.seg_begin = ptr<int64_t>(ctx->seg_begin);
  sv.seg_len = ctx->seg_len;
  MlpRun mr = {};
  if (ctx->rc.rate_mode == DMB_RATE_MLP) {
    if (!ctx->mlp_ready) return fail(ctx, DMB_ERR_STATE, "surrogate rate provider selected but no trained network");
    if (!surrogate_covers(ctx))
      return fail(ctx, DMB_ERR_DOMAIN, "the surrogate was not trained for this cross section (law or power-law index)");
    mr = mlp_run(ctx);
    CK(cudaMemsetAsync(ctx->mlp_fallback.p, 0, 8, ctx->stream), "memset");
    const bool tm = ctx->timing && !ctx->capturing;
    if (surrogate_epilogue<R>(ctx)) {
      if (tm) CK(cudaEventRecord(ctx->sev[0], ctx->stream), "event");
      const dmb_status st =
          surrogate_meanfield(ctx, mr, ptr<int64_t>(ctx->sg.row_ptr), ctx->gas.n, nullptr, ctx->sg.n_pairs, o);
      if (st != DMB_OK) return st;
      if (tm) {
        CK(cudaEventRecord(ctx->sev[1], ctx->stream), "event");
        ctx->sev_pending = true;
      }
      return DMB_OK;
    }
    if (!ensure(ctx->mlp_rates, (size_t)ctx->sg.n_pairs * 8 + 8)) return fail(ctx, DMB_ERR_OOM, "surrogate rates");
    mr.rates = ptr<float2>(ctx->mlp_rates);
    if (sizeof(R) == 4) {
      if (tm) CK(cudaEventRecord(ctx->sev[0], ctx->stream), "event");
      const dmb_status st = surrogate_rates(ctx, mr, sv, ptr<int64_t>(ctx->sg.row_ptr), ctx->gas.n, nullptr,
                                            ctx->sg.n_pairs);
      if (st != DMB_OK) return st;
      if (tm) {
        CK(cudaEventRecord(ctx->sev[1], ctx->stream), "event");
        ctx->sev_pending = true;
      }
    }
  }
  CK(launch_meanfield<R>(G, D, ctx->bx, ptr<int64_t>(ctx->sg.row_ptr), ptr<uint32_t>(ctx->sg.rows), sv,
                         ctx->n_seg_max, ptr<float4>(ctx->gtab), ctx->rc, o, ptr<R>(ctx->mf_part), mr,
                         ctx->shp.mf_bps, ctx->stream, &ctx->launches, ready_weights<R>(ctx).q), "meanfield");
  return DMB_OK;
}

int mc_blocks_for(int64_t n) {   // blocks of the float64 finish kernel (256 threads)
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b > 0 ? b : 1);
}

template <typename R>
dmb_status mc_impl(dmb_ctx *ctx, uint64_t step, double dt, double *vel_out, uint8_t *scat, uint32_t *partner,
                   float *pratio, double *ptot) {
  const SpeciesView<R> D = view<R>(ctx->dm, ctx->nbox > 0), G = view<R>(ctx->gas, ctx->nbox > 0);
  const int nb = mc_blocks_for(D.n);
  if (!ensure(ctx->mc_blocks, (size_t)nb * 8 * 8) || !ensure(ctx->mc_max, (size_t)nb * 8))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for MC partials");
  McArgs a;
  a.variant = ctx->mc_variant;
  a.beta = ctx->mc_beta;
  a.dt = dt;
  a.step = step;
  a.seed = ctx->p.seed;
  a.id_bits = 32;
  a.vel_in = ctx->dm_vel;
  a.vel_out = vel_out;
  a.scattered = scat;
  a.partner = partner;
  a.p_ratio = pratio;
  a.p_total = ptot;
  a.block_sums = ptr<double>(ctx->mc_blocks);
  a.block_max = ptr<double>(ctx->mc_max);
  if (ctx->capturing) a.step_dev = ptr<unsigned long long>(ctx->step_dev);   // set before each replay
  if (!ensure(ctx->mc_rec, (size_t)D.n * sizeof(McRec))) return fail(ctx, DMB_ERR_OOM, "MC scratch");
  a.g = ready_weights<R>(ctx).t;
  if (D.n > 0)
    CK(launch_mc<R>(D, G, ctx->bx, ptr<int64_t>(ctx->sd.row_ptr), ptr<uint32_t>(ctx->sd.rows),
                    ptr<float4>(ctx->gtab), ctx->rc, a, ptr<R>(ctx->pcache), ptr<McRec>(ctx->mc_rec), nb,
                    ctx->shp.mc_bps, ctx->stream, &ctx->launches), "mc");
  return DMB_OK;
}

// The mean field and the Monte Carlo of a float32 step with one categorical draw per DM particle
// in one pass over the gas-major pairs (launch_pairs_fused), then the Monte Carlo's sums and
// selection per DM row (launch_mc_select): the results of meanfield_impl and mc_impl, each pair's
// geometry and overlap evaluated once.  ev_mid (may be null) is recorded between the two.
dmb_status step_pairs_fused(dmb_ctx *ctx, uint64_t step, double dt, double *vel_out, cudaEvent_t ev_mid) {
  const SpeciesView<float> D = view<float>(ctx->dm, ctx->nbox > 0), G = view<float>(ctx->gas, ctx->nbox > 0);
  MfOut o;
  o.acc = ptr<double>(ctx->mf_acc);
  o.dudt = ptr<double>(ctx->mf_dudt);
  o.e_exp = ptr<double>(ctx->e_exp);
  if (!ensure(ctx->mf_part, (size_t)ctx->n_seg_max * 6 * 4)) return fail(ctx, DMB_ERR_OOM, "mean-field scratch");
  SegView sv;
  sv.seg_ptr = ptr<int64_t>(ctx->seg_ptr);
  sv.seg_row = ptr<uint32_t>(ctx->seg_row);
  sv.seg_begin = ptr<int64_t>(ctx->seg_begin);
  sv.seg_len = ctx->seg_len;
  MlpRun mr = {};
  if (ctx->rc.rate_mode == DMB_RATE_MLP) {
    if (!ctx->mlp_ready) return fail(ctx, DMB_ERR_STATE, "surrogate rate provider selected but no trained network");
    if (!surrogate_covers(ctx))
      return fail(ctx, DMB_ERR_DOMAIN, "the surrogate was not trained for this cross section (law or power-law index)");
    mr = mlp_run(ctx);
    CK(cudaMemsetAsync(ctx->mlp_fallback.p, 0, 8, ctx->stream), "memset");
    if (!ensure(ctx->mlp_rates, (size_t)ctx->sg.n_pairs * 8 + 8)) return fail(ctx, DMB_ERR_OOM, "surrogate rates");
    mr.rates = ptr<float2>(ctx->mlp_rates);
    const bool tm = ctx->timing && !ctx->capturing;
    if (tm) CK(cudaEventRecord(ctx->sev[0], ctx->stream), "event");
    const dmb_status st = surrogate_rates(ctx, mr, sv, ptr<int64_t>(ctx->sg.row_ptr), ctx->gas.n, nullptr,
                                          ctx->sg.n_pairs);
    if (st != DMB_OK) return st;
    if (tm) {
      CK(cudaEventRecord(ctx->sev[1], ctx->stream), "event");
      ctx->sev_pending = true;
    }
  }
  const int nb = mc_blocks_for(D.n);
  if (!ensure(ctx->mc_blocks, (size_t)nb * 8 * 8) || !ensure(ctx->mc_max, (size_t)nb * 8) ||
      !ensure(ctx->mc_rec, (size_t)D.n * sizeof(McRec)) || !ensure(ctx->pcache, (size_t)ctx->sd.n_pairs * 4))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for MC partials");
  McArgs a;
  a.variant = 0;
  a.beta = ctx->mc_beta;
  a.dt = dt;
  a.step = step;
  a.seed = ctx->p.seed;
  a.id_bits = 32;
  a.vel_in = ctx->dm_vel;
  a.vel_out = vel_out;
  a.scattered = nullptr;
  a.partner = nullptr;
  a.p_ratio = nullptr;
  a.p_total = nullptr;
  a.block_sums = ptr<double>(ctx->mc_blocks);
  a.block_max = ptr<double>(ctx->mc_max);
  if (ctx->capturing) a.step_dev = ptr<unsigned long long>(ctx->step_dev);
  CK(launch_pairs_fused(G, D, ctx->bx, ptr<int64_t>(ctx->sg.row_ptr), ptr<uint32_t>(ctx->sg.rows), sv, ctx->n_seg_max,
                        ptr<float4>(ctx->gtab), ctx->rc, o, ptr<float>(ctx->mf_part), mr, a, ptr<float>(ctx->pcache),
                        ctx->shp.mf_bps, ctx->stream, &ctx->launches), "fused pair pass");
  if (ev_mid) CK(cudaEventRecord(ev_mid, ctx->stream), "event");
  if (D.n > 0)
    CK(launch_mc_select(D, G, ctx->bx, ptr<int64_t>(ctx->sd.row_ptr), ptr<uint32_t>(ctx->sd.rows),
                        ptr<uint32_t>(ctx->gidx), ptr<float>(ctx->pcache), ptr<float4>(ctx->gtab), ctx->rc, a,
                        ptr<McRec>(ctx->mc_rec), nb, ctx->shp.mc_bps, ctx->stream, &ctx->launches), "mc select");
  return DMB_OK;
}

dmb_status check_dm(dmb_ctx *ctx, const dmb_dm *dm) {
  if (!dm) return fail(ctx, DMB_ERR_ARG, "dm is NULL");
  if (dm->n < 0 || dm->n > 0x7fffffffLL) return fail(ctx, DMB_ERR_ARG, "dm->n out of range");
  if (dm->n > 0 && (!dm->pos || !dm->vel || !dm->mass || !dm->h || !dm->id))
    return fail(ctx, DMB_ERR_ARG, "dm has a NULL array");
  return DMB_OK;
}
dmb_status check_gas(dmb_ctx *ctx, const dmb_gas *g) {
  if (!g) return fail(ctx, DMB_ERR_ARG, "gas is NULL");
  if (g->n < 0 || g->n > 0x7fffffffLL) return fail(ctx, DMB_ERR_ARG, "gas->n out of range");
  if (g->n > 0 && (!g->pos || !g->vel || !g->mass || !g->h || !g->T || !g->mu || !g->id))
    return fail(ctx, DMB_ERR_ARG, "gas has a NULL array");
  return DMB_OK;
}

// ---- hierarchical substeps -------------------------------------------------------------------
int substep_lim(uint64_t substep) {   // active bins are b < lim: s mod 2^b == 0
  if (substep == 0) return DMB_NBINS;
  const int nu = __builtin_ctzll(substep);
  return nu + 1 < DMB_NBINS ? nu + 1 : DMB_NBINS;
}

template <typename R>
dmb_status set_bins_impl(dmb_ctx *ctx, const uint8_t *dm_bin, const uint8_t *gas_bin) {
  cudaStream_t s = ctx->stream;
  int64_t *L = &ctx->launches;
  const int64_t nd = ctx->dm.n, ng = ctx->gas.n, nmax = nd > ng ? nd : ng;
  dmb_status st;
  if ((st = ensure_sort_scratch(ctx, nmax + 1)) != DMB_OK) return st;
  bool ok = ensure(ctx->bin_keys, (size_t)nmax * 8) && ensure(ctx->bin_keys1, (size_t)nmax * 8) &&
            ensure(ctx->bin_vals1, (size_t)nmax * 4) && ensure(ctx->act_dm, (size_t)nd * 4) &&
            ensure(ctx->act_gas, (size_t)ng * 4) && ensure(ctx->act_start, 2 * (DMB_NBINS + 1) * 8) &&
            ensure(ctx->act_len, (size_t)nmax * 4) && ensure(ctx->act_segs, (size_t)ng * 4) &&
            ensure(ctx->act_seg_ptr, (size_t)(ng + 1) * 8) && ensure(ctx->act_gpairs, (size_t)(ng + 1) * 8) &&
            ensure(ctx->act_dpairs, (size_t)(nd + 1) * 8) && ensure(ctx->act_pick, 3 * (DMB_NBINS + 1) * 8) &&
            ensure(ctx->step_dev, 8);
  if (!ok) return fail(ctx, DMB_ERR_OOM, "device allocation failed for the substep tables");
  int64_t *start = ptr<int64_t>(ctx->act_start);
  const uint8_t *bins[2] = {dm_bin, gas_bin};
  DevBuf *lists[2] = {&ctx->act_dm, &ctx->act_gas};
  const SpeciesBufs *sp[2] = {&ctx->dm, &ctx->gas};
  for (int k = 0; k < 2; ++k) {
    const int64_t n = sp[k]->n;
    if (n > 0) {
      // stable sort of the sorted indices by bin: within a bin the Morton order is kept
      CK(launch_bin_keys(bins[k], ptr<uint32_t>(sp[k]->vals0), n, ptr<uint64_t>(ctx->bin_keys),
                         ptr<uint32_t>(*lists[k]), ptr<uint32_t>(ctx->status), s, L), "bin keys");
      CK(radix_sort_pairs(ptr<uint64_t>(ctx->bin_keys), ptr<uint32_t>(*lists[k]), ptr<uint64_t>(ctx->bin_keys1),
                          ptr<uint32_t>(ctx->bin_vals1), n, 8, ptr<uint32_t>(ctx->hist), ptr<int64_t>(ctx->hist_scan),
                          ptr<int64_t>(ctx->scan_tmp), s, L), "bin sort");
    }
    CK(launch_bin_bounds(ptr<uint64_t>(ctx->bin_keys), n, start + k * (DMB_NBINS + 1), s, L), "bin bounds");
  }
  // gas rows: pairs and segments in list order; DM rows: pairs in list order
  ctx->act_seg_len = ctx->shp.seg;
  CK(launch_list_counts(ptr<uint32_t>(ctx->act_gas), ng, ptr<int64_t>(ctx->sg.row_ptr), ctx->act_seg_len,
                        ptr<uint32_t>(ctx->act_len), ptr<uint32_t>(ctx->act_segs), s, L), "list counts");
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(ctx->act_segs), ptr<int64_t>(ctx->act_seg_ptr), ng,
                            ptr<int64_t>(ctx->scan_tmp), s, L), "scan");
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(ctx->act_len), ptr<int64_t>(ctx->act_gpairs), ng,
                            ptr<int64_t>(ctx->scan_tmp), s, L), "scan");
  CK(launch_list_counts(ptr<uint32_t>(ctx->act_dm), nd, ptr<int64_t>(ctx->sd.row_ptr), 0,
                        ptr<uint32_t>(ctx->act_len), nullptr, s, L), "list counts");
  CK(exclusive_scan_u32_i64(ptr<uint32_t>(ctx->act_len), ptr<int64_t>(ctx->act_dpairs), nd,
                            ptr<int64_t>(ctx->scan_tmp), s, L), "scan");
  int64_t *pick = ptr<int64_t>(ctx->act_pick);
  CK(launch_pick(ptr<int64_t>(ctx->act_seg_ptr), start + (DMB_NBINS + 1), pick, s, L), "pick");
  CK(launch_pick(ptr<int64_t>(ctx->act_gpairs), start + (DMB_NBINS + 1), pick + (DMB_NBINS + 1), s, L), "pick");
  CK(launch_pick(ptr<int64_t>(ctx->act_dpairs), start, pick + 2 * (DMB_NBINS + 1), s, L), "pick");
  CK(cudaMemcpyAsync(&ctx->bin_tab[0][0], start, 2 * (DMB_NBINS + 1) * 8, cudaMemcpyDeviceToHost, s), "readback");
  CK(cudaMemcpyAsync(&ctx->bin_tab[2][0], pick, 3 * (DMB_NBINS + 1) * 8, cudaMemcpyDeviceToHost, s), "readback");
  if ((st = check_status(ctx)) != DMB_OK) return st;
  ctx->act_seg_total = ctx->bin_tab[2][DMB_NBINS];
  if (!ensure(ctx->act_seg_row, (size_t)ctx->act_seg_total * 4) ||
      !ensure(ctx->act_seg_begin, (size_t)ctx->act_seg_total * 8))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for the substep segments");
  CK(launch_list_seg_map(ptr<uint32_t>(ctx->act_gas), ng, ptr<int64_t>(ctx->sg.row_ptr),
                         ptr<int64_t>(ctx->act_seg_ptr), ctx->act_seg_len, ptr<uint32_t>(ctx->act_seg_row),
                         ptr<int64_t>(ctx->act_seg_begin), s, L), "segment map");
  // every buffer a substep touches, at its largest size: a substep (and its capture) allocates nothing
  ok = ensure(ctx->mf_part, (size_t)ctx->act_seg_total * 6 * sizeof(R)) && ensure(ctx->mf_acc, (size_t)ng * 24) &&
       ensure(ctx->mf_dudt, (size_t)ng * 8) && ensure(ctx->e_exp, (size_t)ng * 8) &&
       ensure(ctx->mc_rec, (size_t)nd * sizeof(McRec)) && ensure(ctx->mc_blocks, (size_t)mc_blocks_for(nd) * 8 * 8) &&
       ensure(ctx->mc_max, (size_t)mc_blocks_for(nd) * 8) && ensure(ctx->kick_blocks, (size_t)152 * 4 * KICK_NSUM * 8);
  if (ok && ctx->rc.rate_mode == DMB_RATE_MLP)
    ok = ensure_mlp(ctx) == DMB_OK && ensure(ctx->mlp_rates, (size_t)ctx->sg.n_pairs * 8 + 8);
  if (!ok) return fail(ctx, DMB_ERR_OOM, "device allocation failed for substep scratch");
  if (ctx->rc.rate_mode == DMB_RATE_MLP) {
    CK(prepare_mlp_pair_rates(), "surrogate kernel attributes");
    CK(mlp_tc_prepare(), "surrogate kernel attributes");
    if (!ensure(ctx->tc_tiles, (size_t)ctx->bin_tab[3][DMB_NBINS] * 4 + 16) ||
        !ensure(ctx->tc_part, ((size_t)(ctx->bin_tab[3][DMB_NBINS] >> 5) + (size_t)ctx->gas.n + 1) * 24))
      return fail(ctx, DMB_ERR_OOM, "surrogate pair rows");
  }
  CK(cudaStreamSynchronize(s), "synchronise");
  ctx->dm_bin = dm_bin;
  ctx->gas_bin = gas_bin;
  ctx->bins_ready = true;
  return DMB_OK;
}

// The launches of one substep (no allocation, no host synchronisation: capturable).
template <typename R>
dmb_status substep_body(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, int lim, uint64_t substep,
                        double dt_min, bool step_on_device) {
  cudaStream_t s = ctx->stream;
  int64_t *L = &ctx->launches;
  const SpeciesView<R> D = view<R>(ctx->dm), G = view<R>(ctx->gas);
  const int64_t nda = ctx->bin_tab[0][lim], nga = ctx->bin_tab[1][lim], nseg = ctx->bin_tab[2][lim];
  const double pair_evals = 0.5 * (double)(ctx->bin_tab[3][lim] + ctx->bin_tab[4][lim]);
  // mean field of the active gas rows against all their DM partners
  SegView sv;
  sv.seg_ptr = ptr<int64_t>(ctx->act_seg_ptr);
  sv.seg_row = ptr<uint32_t>(ctx->act_seg_row);
  sv.seg_begin = ptr<int64_t>(ctx->act_seg_begin);
  sv.seg_len = ctx->act_seg_len;
  sv.list = ptr<uint32_t>(ctx->act_gas);
  sv.n_rows = nga;
  sv.n_seg = nseg;
  MfOut o;
  o.acc = ptr<double>(ctx->mf_acc);
  o.dudt = ptr<double>(ctx->mf_dudt);
  o.e_exp = ptr<double>(ctx->e_exp);
  MlpRun mr = {};
  if (ctx->rc.rate_mode == DMB_RATE_MLP) {
    mr = mlp_run(ctx);
    mr.rates = ptr<float2>(ctx->mlp_rates);
    CK(cudaMemsetAsync(ctx->mlp_fallback.p, 0, 8, s), "memset");
    if (surrogate_epilogue<R>(ctx)) {
      const dmb_status st = surrogate_meanfield(ctx, mr, ptr<int64_t>(ctx->act_gpairs), nga,
                                                ptr<uint32_t>(ctx->act_gas), ctx->bin_tab[3][lim], o);
      if (st != DMB_OK) return st;
    } else if (sizeof(R) == 4 && nseg > 0) {
      const dmb_status st = surrogate_rates(ctx, mr, sv, ptr<int64_t>(ctx->act_gpairs), nga,
                                            ptr<uint32_t>(ctx->act_gas), ctx->bin_tab[3][lim]);
      if (st != DMB_OK) return st;
    }
  }
  if (nga > 0 && !surrogate_epilogue<R>(ctx))
    CK(launch_meanfield<R>(G, D, ctx->bx, ptr<int64_t>(ctx->sg.row_ptr), ptr<uint32_t>(ctx->sg.rows), sv, nseg,
                           ptr<float4>(ctx->gtab), ctx->rc, o, ptr<R>(ctx->mf_part), mr, ctx->shp.mf_bps, s, L,
                           ready_weights<R>(ctx).q),
       "meanfield");
  // Monte Carlo of the active DM against all their gas partners, each with its own dt
  const int nb = mc_blocks_for(nda);
  McArgs a;
  a.variant = ctx->mc_variant;
  a.beta = ctx->mc_beta;
  a.dt = dt_min;
  a.step = substep;
  a.seed = ctx->p.seed;
  a.id_bits = 32;
  a.vel_in = dm->vel;
  a.vel_out = const_cast<double *>(dm->vel);
  a.scattered = nullptr;
  a.partner = nullptr;
  a.p_ratio = nullptr;
  a.p_total = nullptr;
  a.block_sums = ptr<double>(ctx->mc_blocks);
  a.block_max = ptr<double>(ctx->mc_max);
  a.list = ptr<uint32_t>(ctx->act_dm);
  a.n_list = nda;
  a.bin = ctx->dm_bin;
  a.step_dev = step_on_device ? ptr<unsigned long long>(ctx->step_dev) : nullptr;
  a.v_sorted = ctx->dm.V.p;
  a.v_sorted_fp64 = ctx->p.fp64 ? 1 : 0;
  a.g = ready_weights<R>(ctx).t;
  if (nda > 0)
    CK(launch_mc<R>(D, G, ctx->bx, ptr<int64_t>(ctx->sd.row_ptr), ptr<uint32_t>(ctx->sd.rows),
                    ptr<float4>(ctx->gtab), ctx->rc, a, ptr<R>(ctx->pcache), ptr<McRec>(ctx->mc_rec), nb,
                    ctx->shp.mc_bps, s, L), "mc");
  // kick of the active gas (refreshing its sorted copies) and the sums
  const int kb = 152 * 4;
  CK(launch_kick_gas_list<R>(const_cast<double *>(gas->vel), const_cast<double *>(gas->T), gas->mu, gas->mass,
                             ptr<double>(ctx->mf_acc), ptr<double>(ctx->mf_dudt), ptr<double>(ctx->e_exp),
                             ptr<uint32_t>(ctx->act_gas), nga, G.perm, ctx->gas_bin, dt_min, ctx->rc,
                             ptr<typename Vec<R>::v4>(ctx->gas.V), ptr<typename Vec<R>::v4>(ctx->gas.K),
                             ptr<double>(ctx->kick_blocks), kb, s, L), "kick");
  CK(launch_final_sums(ptr<double>(ctx->mc_blocks), ptr<double>(ctx->mc_max), nda > 0 ? nb : 0,
                       ptr<double>(ctx->kick_blocks), kb, dt_min, pair_evals, ptr<double>(ctx->sums), s, L), "sums");
  return DMB_OK;
}

dmb_status substep_graph(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, int lim, uint64_t substep,
                         double dt_min) {
  if (!ctx->gstream) {
    CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking), "graph stream");
    for (int k = 0; k < 2; ++k) CK(cudaEventCreateWithFlags(&ctx->gev[k], cudaEventDisableTiming), "graph event");
  }
  const void *key[6] = {dm->vel, gas->vel, gas->T, gas->mu, gas->mass, ctx->dm_bin};
  dmb_ctx::GraphEntry *ent = nullptr;
  for (auto &g : ctx->graphs)
    if (g.lim == lim && g.dt == dt_min && memcmp(g.key, key, sizeof(key)) == 0) ent = &g;
  if (!ent) {
    // capture the substep's launches on the context's own stream; the graph ends by advancing
    // the device step counter, so consecutive substeps need no host write
    cudaStream_t saved = ctx->stream;
    const int64_t l0 = ctx->launches;
    ctx->stream = ctx->gstream;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
    dmb_status st = DMB_ERR_CUDA;
    if (e == cudaSuccess) {
      st = ctx->p.fp64 ? substep_body<double>(ctx, dm, gas, lim, substep, dt_min, true)
                       : substep_body<float>(ctx, dm, gas, lim, substep, dt_min, true);
      if (st == DMB_OK) {
        const cudaError_t ei = launch_step_advance(ptr<unsigned long long>(ctx->step_dev), ctx->gstream, &ctx->launches);
        if (ei != cudaSuccess) st = cuda_fail(ctx, ei, "step counter");
      }
      const cudaError_t e2 = cudaStreamEndCapture(ctx->gstream, &g);
      if (st == DMB_OK && e2 != cudaSuccess) st = cuda_fail(ctx, e2, "graph capture");
    } else {
      st = cuda_fail(ctx, e, "graph capture");
    }
    ctx->stream = saved;
    const int64_t nl = ctx->launches - l0;
    ctx->launches = l0;
    if (st != DMB_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    dmb_ctx::GraphEntry ne;
    ne.lim = lim;
    ne.dt = dt_min;
    memcpy(ne.key, key, sizeof(key));
    ne.launches = nl;
    e = cudaGraphInstantiate(&ne.exec, g, 0);
    cudaGraphDestroy(g);
    CK(e, "graph instantiate");
    ctx->graphs.push_back(ne);
    ent = &ctx->graphs.back();
  }
  CK(cudaEventRecord(ctx->gev[0], ctx->stream), "event");
  CK(cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0), "event wait");
  if (ctx->graph_next_step != substep) {
    CK(launch_step_set(ptr<unsigned long long>(ctx->step_dev), substep, ctx->gstream, &ctx->launches), "step counter");
  }
  CK(cudaGraphLaunch(ent->exec, ctx->gstream), "graph launch");
  ctx->launches += ent->launches;
  ctx->graph_next_step = substep + 1;
  ctx->batch_next_step = ~0ull;
  CK(cudaEventRecord(ctx->gev[1], ctx->gstream), "event");
  CK(cudaStreamWaitEvent(ctx->stream, ctx->gev[1], 0), "event wait");
  return DMB_OK;
}

}  // namespace

// ---- accessors for entry points defined in other translation units -----------------------
bool dmb_internal_surrogate(dmb_ctx *ctx, MlpDev *dev, cudaStream_t *stream) {
  if (!ctx || !ctx->mlp_ready) return false;
  *dev = mlp_dev(ctx);
  *stream = ctx->stream;
  return true;
}

int dmb_internal_device(const dmb_ctx *ctx) { return ctx ? ctx->device : -1; }

dmb_status dmb_internal_fail(dmb_ctx *ctx, dmb_status s, const char *msg) { return fail(ctx, s, msg); }

// ======================================================================================
extern "C" {

dmb_status dmb_create(dmb_ctx **out, const dmb_params *p, void *cuda_stream) {
  if (!out) return fail(nullptr, DMB_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!p) return fail(nullptr, DMB_ERR_ARG, "params is NULL");
  if (!(p->sigma0_cm2 >= 0.0) || !isfinite(p->sigma0_cm2)) return fail(nullptr, DMB_ERR_ARG, "sigma0 must be finite and >= 0");
  if (!(p->v0_kms > 0.0) || !isfinite(p->v0_kms)) return fail(nullptr, DMB_ERR_ARG, "v0 must be > 0");
  if (p->n < -4 || p->n > 16) return fail(nullptr, DMB_ERR_ARG, "power-law index n must be in [-4, 16]");
  if (!(p->m_chi_mp > 0.0) || !isfinite(p->m_chi_mp)) return fail(nullptr, DMB_ERR_ARG, "m_chi must be > 0");
  if (p->rate_mode != DMB_RATE_CLOSED && p->rate_mode != DMB_RATE_QUAD && p->rate_mode != DMB_RATE_MLP)
    return fail(nullptr, DMB_ERR_ARG, "unknown rate provider");
  if (p->rate_mode == DMB_RATE_MLP && p->fp64)
    return fail(nullptr, DMB_ERR_ARG, "the surrogate rate provider runs in float32 only");
  if (p->periodic)
    for (int k = 0; k < 3; ++k)
      if (!(p->box[k] > 0.0) || !isfinite(p->box[k])) return fail(nullptr, DMB_ERR_ARG, "periodic box sides must be > 0");
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, DMB_ERR_CUDA, "no current CUDA device");
  }
  dmb_ctx *ctx = new dmb_ctx();
  ctx->p = *p;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  const double sig_kpc2 = p->sigma0_cm2 / (kKPC * kKPC);
  ctx->rc.S = sig_kpc2 * (kMSUN / kMP);
  ctx->rc.m_chi = p->m_chi_mp;
  ctx->rc.v0 = p->v0_kms;
  ctx->rc.n = p->n;
  ctx->rc.alpha = pow(2.0, (p->n + 5) / 2.0) * tgamma(3.0 + p->n / 2.0) / sqrt(M_PI);
  ctx->rc.kT_over_mp = kKB / kMP / 1e10;
  ctx->rc.rate_mode = p->rate_mode;
  ctx->bx.periodic = p->periodic ? 1 : 0;
  for (int k = 0; k < 3; ++k) {
    const double Lk = p->periodic ? p->box[k] : 0.0;
    ctx->bx.L[k] = Lk;
    ctx->bx.Lhi[k] = (float)Lk;
    ctx->bx.Llo[k] = (float)(Lk - (double)ctx->bx.Lhi[k]);
  }
  ctx->bx.pad = 0.0f;
  bool ok = ensure(ctx->frame, sizeof(Frame)) && ensure(ctx->status, 16) && ensure(ctx->frame_part, 1024 * 8 * 8) &&
            ensure(ctx->gtab, (size_t)DMB_GT_NQ * DMB_GT_CELLS * 16) && ensure(ctx->sums, 16 * 8) &&
            ensure(ctx->search_stats, 16 * 8);
  if (!ok) {
    dmb_destroy(ctx);
    return fail(nullptr, DMB_ERR_OOM, "device allocation failed at context creation");
  }
  if (cudaMallocHost(&ctx->h_status, 64) != cudaSuccess || cudaMallocHost(&ctx->h_tot, 64) != cudaSuccess ||
      cudaMallocHost(&ctx->h_sums, 16 * 8) != cudaSuccess) {
    cudaGetLastError();
    dmb_destroy(ctx);
    return fail(nullptr, DMB_ERR_OOM, "pinned host allocation failed");
  }
  cudaError_t e = cudaMemsetAsync(ctx->status.p, 0, 16, ctx->stream);
  if (e == cudaSuccess) e = launch_gtable(ptr<float4>(ctx->gtab), ctx->stream, &ctx->launches);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    std::string m = std::string("context setup: ") + cudaGetErrorString(e);
    dmb_destroy(ctx);
    return fail(nullptr, DMB_ERR_CUDA, m);
  }
  *out = ctx;
  return DMB_OK;
}

dmb_status dmb_destroy(dmb_ctx *ctx) {
  if (!ctx) return DMB_OK;
  if (ctx->stream || true) cudaStreamSynchronize(ctx->stream);
  if (ctx->gstream) cudaStreamSynchronize(ctx->gstream);
  clear_graphs(ctx);
  clear_batch_graph(ctx);
  for (int k = 0; k < 2; ++k)
    if (ctx->gev[k]) cudaEventDestroy(ctx->gev[k]);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  for (SearchBufs *sb : {&ctx->sg, &ctx->sd}) {
    DevBuf *q[] = {&sb->item_cnt, &sb->item_ptr, &sb->items, &sb->unit_cnt_leaf, &sb->unit_ptr, &sb->unit_leaf,
                   &sb->unit_item0, &sb->unit_cnt, &sb->counts, &sb->row_ptr, &sb->rows, &sb->tmask};
    for (DevBuf *b : q) release(*b);
  }
  DevBuf *bufs[] = {&ctx->frame, &ctx->status, &ctx->frame_part, &ctx->gtab, &ctx->hist, &ctx->hist_scan,
                    &ctx->scan_tmp, &ctx->pcache, &ctx->mf_part, &ctx->mc_rec, &ctx->seg_cnt, &ctx->seg_ptr,
                    &ctx->seg_row, &ctx->seg_begin, &ctx->t_cursor, &ctx->mlp_p, &ctx->mlp_m, &ctx->mlp_v,
                    &ctx->mlp_w2, &ctx->mlp_w3, &ctx->mlp_w2t, &ctx->mlp_w3t, &ctx->mlp_fallback, &ctx->mlp_rates,
                    &ctx->box_sides, &ctx->box_params, &ctx->mf_acc, &ctx->mf_dudt, &ctx->e_exp, &ctx->mc_blocks, &ctx->mc_max,
                    &ctx->kick_blocks, &ctx->sums, &ctx->scratch_vel, &ctx->search_stats, &ctx->act_dm,
                    &ctx->act_gas, &ctx->act_start, &ctx->act_seg_ptr, &ctx->act_seg_row, &ctx->act_seg_begin,
                    &ctx->act_len, &ctx->act_segs, &ctx->act_gpairs, &ctx->act_dpairs, &ctx->act_pick,
                    &ctx->step_dev, &ctx->bin_keys, &ctx->bin_keys1, &ctx->bin_vals1, &ctx->tc_tiles,
                    &ctx->rebin_cnt, &ctx->gate, &ctx->cap_need, &ctx->gidx};
  for (DevBuf *b : bufs) release(*b);
  SpeciesBufs *sp[2] = {&ctx->dm, &ctx->gas};
  for (SpeciesBufs *s : sp) {
    DevBuf *sb[] = {&s->keys0, &s->keys1, &s->vals0, &s->vals1, &s->P, &s->L, &s->V, &s->K, &s->sid, &s->bmin, &s->bmax,
                    &s->bid, &s->leaf_box};
    for (DevBuf *b : sb) release(*b);
  }
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->h_tot) cudaFreeHost(ctx->h_tot);
  if (ctx->h_sums) cudaFreeHost(ctx->h_sums);
  for (int k = 0; k < 6; ++k)
    if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
  for (int k = 0; k < 2; ++k)
    if (ctx->sev[k]) cudaEventDestroy(ctx->sev[k]);
  delete ctx;
  return DMB_OK;
}

const char *dmb_last_error(const dmb_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int64_t dmb_launch_count(const dmb_ctx *ctx) { return ctx ? ctx->launches : 0; }

static dmb_status build_grid_checked(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas) {
  dmb_status st;
  if ((st = check_dm(ctx, dm)) != DMB_OK || (st = check_gas(ctx, gas)) != DMB_OK) return st;
  return ctx->p.fp64 ? build_grid_impl<double>(ctx, dm, gas) : build_grid_impl<float>(ctx, dm, gas);
}

dmb_status dmb_build_grid(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  ctx->nbox = 0;
  ctx->dm_box = ctx->gas_box = nullptr;
  ctx->bx.boxes = nullptr;
  return build_grid_checked(ctx, dm, gas);
}

dmb_status dmb_neighbors(dmb_ctx *ctx, int64_t *n_pairs, uint32_t *pairs_out, int64_t capacity) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!ctx->grid_ready) return fail(ctx, DMB_ERR_STATE, "dmb_neighbors before dmb_build_grid");
  dmb_status st = ctx->p.fp64 ? neighbors_impl<double>(ctx, true) : neighbors_impl<float>(ctx, true);
  if (st != DMB_OK) return st;
  if (n_pairs) *n_pairs = ctx->n_pairs;
  if (pairs_out && capacity > 0)
    CK(launch_pairs_out(ptr<int64_t>(ctx->sg.row_ptr), ptr<uint32_t>(ctx->sg.rows), ptr<uint32_t>(ctx->gas.vals0),
                        ptr<uint32_t>(ctx->dm.vals0), ctx->gas.n, capacity, pairs_out, ctx->stream, &ctx->launches),
       "pairs out");
  return DMB_OK;
}

dmb_status dmb_meanfield_gas(dmb_ctx *ctx, double *acc, double *dudt) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!ctx->pairs_ready) return fail(ctx, DMB_ERR_STATE, "dmb_meanfield_gas before dmb_neighbors");
  if (ctx->gas.n > 0 && (!acc || !dudt)) return fail(ctx, DMB_ERR_ARG, "acc/dudt is NULL");
  return ctx->p.fp64 ? meanfield_impl<double>(ctx, acc, dudt, nullptr) : meanfield_impl<float>(ctx, acc, dudt, nullptr);
}

dmb_status dmb_mc_scatter_dm(dmb_ctx *ctx, uint64_t step, double dt, double *vel_out, uint8_t *scattered,
                             uint32_t *partner, float *p_ratio_max, double *p_total) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!ctx->pairs_ready) return fail(ctx, DMB_ERR_STATE, "dmb_mc_scatter_dm before dmb_neighbors");
  if (!(dt >= 0.0) || !isfinite(dt)) return fail(ctx, DMB_ERR_ARG, "dt must be finite and >= 0");
  if (ctx->dm.n > 0 && !vel_out) return fail(ctx, DMB_ERR_ARG, "vel_out is NULL");
  return ctx->p.fp64 ? mc_impl<double>(ctx, step, dt, vel_out, scattered, partner, p_ratio_max, p_total)
                     : mc_impl<float>(ctx, step, dt, vel_out, scattered, partner, p_ratio_max, p_total);
}

static dmb_status step_body(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, uint64_t step, double dt,
                            double *sums_out);
static dmb_status step_batched_graph(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, const dmb_box *boxes,
                                     int nbox, uint64_t step, double dt, double *sums_out);

dmb_status dmb_step(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, uint64_t step, double dt, double *sums_out) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!(dt >= 0.0) || !isfinite(dt)) return fail(ctx, DMB_ERR_ARG, "dt must be finite and >= 0");
  ctx->nbox = 0;
  ctx->dm_box = ctx->gas_box = nullptr;
  ctx->bx.boxes = nullptr;
  return step_body(ctx, dm, gas, step, dt, sums_out);
}

dmb_status dmb_step_batched(dmb_ctx *ctx, const dmb_dm *dm, const uint32_t *dm_box, const dmb_gas *gas,
                            const uint32_t *gas_box, const dmb_box *boxes, int32_t nbox, uint64_t step, double dt,
                            double *sums_out) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!(dt >= 0.0) || !isfinite(dt)) return fail(ctx, DMB_ERR_ARG, "dt must be finite and >= 0");
  if (!ctx->p.periodic) return fail(ctx, DMB_ERR_ARG, "batched boxes need a periodic context");
  if (nbox < 1 || nbox > 65535 || !boxes) return fail(ctx, DMB_ERR_ARG, "nbox must be in [1, 65535] with a box table");
  if ((dm && dm->n > 0 && !dm_box) || (gas && gas->n > 0 && !gas_box))
    return fail(ctx, DMB_ERR_ARG, "box index arrays are required");
  std::vector<BoxSide> sides(nbox);
  std::vector<BoxParamDev> bp(nbox);
  double Lmax = 0.0;
  for (int b = 0; b < nbox; ++b) {
    for (int k = 0; k < 3; ++k) {
      const double L = boxes[b].box[k];
      if (!(L > 0.0) || !isfinite(L)) return fail(ctx, DMB_ERR_ARG, "box sides must be > 0");
      Lmax = fmax(Lmax, L);
    }
    if (!(boxes[b].sigma0_cm2 >= 0.0) || !(boxes[b].m_chi_mp > 0.0))
      return fail(ctx, DMB_ERR_ARG, "box sigma0 must be >= 0 and m_chi > 0");
  }
  // slots of width 3 Lmax: particles of different boxes are >= 2 Lmax apart, so even after a
  // minimum-image shift by one side (<= Lmax) they stay >= Lmax > h_i + h_j apart, and a box's
  // periodic images searched by the tree stay inside its own slot
  ctx->stride = 3.0 * Lmax;
  for (int b = 0; b < nbox; ++b) {
    for (int k = 0; k < 3; ++k) {
      const double L = boxes[b].box[k];
      sides[b].L[k] = L;
      sides[b].Lhi[k] = (float)L;
      sides[b].Llo[k] = (float)(L - (double)sides[b].Lhi[k]);
      bp[b].L[k] = L;
    }
    bp[b].S = boxes[b].sigma0_cm2 / (kKPC * kKPC) * (kMSUN / kMP);
    bp[b].m_chi = boxes[b].m_chi_mp;
    bp[b].offset_x = b * ctx->stride;
  }
  if (!ensure(ctx->box_sides, sizeof(BoxSide) * nbox) || !ensure(ctx->box_params, sizeof(BoxParamDev) * nbox))
    return fail(ctx, DMB_ERR_OOM, "box tables");
  CK(cudaMemcpy(ctx->box_sides.p, sides.data(), sizeof(BoxSide) * nbox, cudaMemcpyHostToDevice), "box table");
  CK(cudaMemcpy(ctx->box_params.p, bp.data(), sizeof(BoxParamDev) * nbox, cudaMemcpyHostToDevice), "box table");
  // frame of the virtual space: boxes side by side along x, each in a slot of width `stride`
  {
    const int64_t ntot = (dm ? dm->n : 0) + (gas ? gas->n : 0);
    int box_bits = 0;
    while ((1 << box_bits) < nbox) ++box_bits;
    int bits = (int)fmin(21.0, fmax(10.0, ceil(log2((double)(ntot > 1 ? ntot : 2)) / 3.0) + 7.0));
    bits = (int)fmin((double)bits, floor((63.0 - box_bits) / 3.0));
    Frame f;
    for (int c = 0; c < 3; ++c) f.origin[c] = 0.0;
    f.span = fmax(nbox * ctx->stride, Lmax);
    int e;
    frexp(f.span, &e);
    f.delta = ldexp(1.0, e - 23);
    f.inv_delta = ldexp(1.0, 23 - e);
    f.bits = bits;
    f.key_scale = ldexp(1.0, bits) / (Lmax * (1.0 + 1e-12));
    f.pad = (float)(4.0 * ldexp(1.0, e) * 1.1920928955078125e-07);
    f.hmax_dm = f.hmax_gas = 0.0;
    CK(cudaMemcpy(ctx->frame.p, &f, sizeof(Frame), cudaMemcpyHostToDevice), "frame");
  }
  ctx->frame_ready = true;
  ctx->nbox = nbox;
  ctx->dm_box = dm_box;
  ctx->gas_box = gas_box;
  ctx->bx.boxes = ptr<BoxSide>(ctx->box_sides);
  dmb_status st;
  if (ctx->use_graph && dm && gas) {
    st = (dm->n > 0 && gas->n > 0) ? step_batched_graph(ctx, dm, gas, boxes, nbox, step, dt, sums_out)
                                   : step_body(ctx, dm, gas, step, dt, sums_out);
  } else {
    st = step_body(ctx, dm, gas, step, dt, sums_out);
  }
  ctx->frame_ready = false;
  ctx->nbox = 0;
  ctx->dm_box = ctx->gas_box = nullptr;
  ctx->bx.boxes = nullptr;
  return st;
}

static dmb_status step_body(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, uint64_t step, double dt,
                            double *sums_out) {
  dmb_status st;
  const bool tm = ctx->timing && !ctx->capturing;
  if (tm) CK(cudaEventRecord(ctx->ev[0], ctx->stream), "event");
  if ((st = build_grid_checked(ctx, dm, gas)) != DMB_OK) return st;
  if (tm) CK(cudaEventRecord(ctx->ev[1], ctx->stream), "event");
  if (ctx->capturing) {
    st = ctx->p.fp64 ? neighbors_capped<double>(ctx) : neighbors_capped<float>(ctx);
    if (st != DMB_OK) return st;
  } else if ((st = ctx->p.fp64 ? neighbors_impl<double>(ctx) : neighbors_impl<float>(ctx)) != DMB_OK) {
    return st;   // the step's own pair set: no weights unless dmb_set_pair_weights(ctx, 1)
  }
  if (tm) CK(cudaEventRecord(ctx->ev[2], ctx->stream), "event");
  const int64_t ng = gas->n, nd = dm->n;
  if (!ensure(ctx->mf_acc, ng * 24) || !ensure(ctx->mf_dudt, ng * 8) || !ensure(ctx->e_exp, ng * 8))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for mean-field scratch");
  if (!ctx->p.fp64 && ctx->mc_variant == 0 && ctx->fuse) {
    // DM velocities are updated in place: the MC reads v_i and writes v_i' for the same particle
    st = step_pairs_fused(ctx, step, dt, const_cast<double *>(dm->vel), tm ? ctx->ev[3] : nullptr);
    if (st != DMB_OK) return st;
  } else {
    st = ctx->p.fp64 ? meanfield_impl<double>(ctx, ptr<double>(ctx->mf_acc), ptr<double>(ctx->mf_dudt), ptr<double>(ctx->e_exp))
                     : meanfield_impl<float>(ctx, ptr<double>(ctx->mf_acc), ptr<double>(ctx->mf_dudt), ptr<double>(ctx->e_exp));
    if (st != DMB_OK) return st;
    if (tm) CK(cudaEventRecord(ctx->ev[3], ctx->stream), "event");
    st = ctx->p.fp64 ? mc_impl<double>(ctx, step, dt, const_cast<double *>(dm->vel), nullptr, nullptr, nullptr, nullptr)
                     : mc_impl<float>(ctx, step, dt, const_cast<double *>(dm->vel), nullptr, nullptr, nullptr, nullptr);
    if (st != DMB_OK) return st;
  }
  if (tm) CK(cudaEventRecord(ctx->ev[4], ctx->stream), "event");
  const int kb = 152 * 4;
  if (!ensure(ctx->kick_blocks, (size_t)kb * KICK_NSUM * 8)) return fail(ctx, DMB_ERR_OOM, "kick partials");
  CK(launch_kick_gas(const_cast<double *>(gas->vel), const_cast<double *>(gas->T), gas->mu, gas->mass,
                     ptr<double>(ctx->mf_acc), ptr<double>(ctx->mf_dudt), ptr<double>(ctx->e_exp), ng, dt,
                     ctx->rc.kT_over_mp, ptr<double>(ctx->kick_blocks), kb, ctx->stream, &ctx->launches,
                     ctx->capturing ? ctx->gate_dev : nullptr), "kick");
  if (nd <= 0) {
    CK(cudaMemsetAsync(ctx->mc_blocks.p ? ctx->mc_blocks.p : ctx->sums.p, 0, 8, ctx->stream), "memset");
  }
  const int mnb = nd > 0 ? mc_blocks_for(nd) : 0;
  if (nd <= 0 && !ensure(ctx->mc_blocks, 64)) return fail(ctx, DMB_ERR_OOM, "mc partials");
  if (nd <= 0 && !ensure(ctx->mc_max, 64)) return fail(ctx, DMB_ERR_OOM, "mc partials");
  CK(launch_final_sums(ptr<double>(ctx->mc_blocks), ptr<double>(ctx->mc_max), mnb, ptr<double>(ctx->kick_blocks), kb,
                       dt, (double)ctx->n_pairs, ptr<double>(ctx->sums), ctx->stream, &ctx->launches,
                       ctx->capturing ? ctx->pairs_dev : nullptr), "sums");
  ctx->grid_ready = false;   // the state moved on: rebuild before the next standalone call
  ctx->pairs_ready = false;
  if (tm) {
    CK(cudaEventRecord(ctx->ev[5], ctx->stream), "event");
    CK(cudaEventSynchronize(ctx->ev[5]), "event sync");
    for (int k = 0; k < 5; ++k) {
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, ctx->ev[k], ctx->ev[k + 1]), "event time");
      ctx->stage_ms[k] += ms;
    }
    if (ctx->sev_pending) {
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, ctx->sev[0], ctx->sev[1]), "event time");
      ctx->stage_ms[5] += ms;
      ctx->sev_pending = false;
    }
    ctx->timed_steps += 1;
  }
  if (sums_out) {
    CK(cudaMemcpyAsync(ctx->h_sums, ctx->sums.p, 16 * 8, cudaMemcpyDeviceToHost, ctx->stream), "sums readback");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    memcpy(sums_out, ctx->h_sums, 16 * 8);
  }
  return DMB_OK;
}

// Buffers of a captured batched step at the capacities (every other buffer depends only on the
// particle counts and was sized by the eager step before the capture).
static dmb_status presize_batch(dmb_ctx *ctx) {
  const dmb_ctx::BatchCaps &c = ctx->bgraph.caps;
  SearchBufs &sg = ctx->sg, &sd = ctx->sd;
  const size_t rb = ctx->p.fp64 ? 8 : 4;
  bool ok = ensure(sg.items, (size_t)c.items * 4) && ensure(sg.tmask, (size_t)c.items * 32 * 4) &&
            ensure(sg.unit_leaf, (size_t)c.units * 4) && ensure(sg.unit_item0, (size_t)c.units * 8) &&
            ensure(sg.unit_cnt, (size_t)c.units * 32 * 4) && ensure(sg.rows, (size_t)c.pairs * 4) &&
            ensure(sd.rows, (size_t)c.pairs * 4) && (!ctx->fuse || ensure(ctx->gidx, (size_t)c.pairs * 4)) &&
            (ctx->p.fp64 || ctx->weights_mode != 1 ||
             (ensure(sg.w, (size_t)c.pairs * 4 + 16) && ensure(sd.w, (size_t)c.pairs * 4 + 16))) &&
            ensure(ctx->pcache, (size_t)c.pairs * rb) &&
            ensure(ctx->seg_row, (size_t)c.segs * 4) && ensure(ctx->seg_begin, (size_t)c.segs * 8) &&
            ensure(ctx->mf_part, (size_t)c.segs * 6 * rb) && ensure(ctx->gate, 16) && ensure(ctx->cap_need, 64) &&
            ensure(ctx->step_dev, 8);
  if (ok && ctx->rc.rate_mode == DMB_RATE_MLP)
    ok = ensure(ctx->mlp_rates, (size_t)c.pairs * 8 + 8) && ensure(ctx->tc_tiles, (size_t)c.pairs * 4 + 16) &&
         ensure(ctx->tc_part, ((size_t)(c.pairs >> 5) + (size_t)ctx->gas.n + 1) * 24);
  if (!ok) return fail(ctx, DMB_ERR_OOM, "device allocation failed for the captured batched step");
  return DMB_OK;
}

// dmb_step_batched under dmb_set_graph(ctx, 1).  The first call for a set of caller arrays and
// boxes (or after an overflow) runs the step directly, then sizes every list buffer to 1.25 x the
// sizes it found and captures the whole step (grid, search, mean field, Monte Carlo, kicks, sums,
// and the advance of the device step counter) into one CUDA graph on the library's stream.  Later
// calls replay it with one graph launch and read back the status, the list totals and the sums.
// If a list outgrew its capacity the replayed step changed nothing (the capacity checks cleared
// the lists and gated the kick): the buffers are regrown and the step runs again directly.
static dmb_status step_batched_graph(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, const dmb_box *boxes,
                                     int nbox, uint64_t step, double dt, double *sums_out) {
  dmb_ctx::BatchGraph &bg = ctx->bgraph;
  const void *key[14] = {dm->pos, dm->vel, dm->mass, dm->h, dm->id, gas->pos, gas->vel, gas->mass,
                         gas->h, gas->T, gas->mu, gas->id, ctx->dm_box, ctx->gas_box};
  if (!ctx->gstream) {
    CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking), "graph stream");
    for (int k = 0; k < 2; ++k) CK(cudaEventCreateWithFlags(&ctx->gev[k], cudaEventDisableTiming), "graph event");
  }
  const bool hit = bg.valid && bg.exec && bg.nd == dm->n && bg.ng == gas->n && bg.dt == dt &&
                   memcmp(bg.key, key, sizeof(key)) == 0 && (int)bg.boxes.size() == nbox &&
                   memcmp(bg.boxes.data(), boxes, sizeof(dmb_box) * (size_t)nbox) == 0;
  int64_t grow[4] = {0, 0, 0, 0};
  if (hit) {
    CK(cudaEventRecord(ctx->gev[0], ctx->stream), "event");
    CK(cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0), "event wait");
    if (ctx->batch_next_step != step)
      CK(launch_step_set(ptr<unsigned long long>(ctx->step_dev), step, ctx->gstream, &ctx->launches), "step counter");
    CK(cudaGraphLaunch(bg.exec, ctx->gstream), "graph launch");
    ctx->launches += bg.launches;
    ctx->batch_next_step = step + 1;
    ctx->graph_next_step = ~0ull;
    CK(cudaEventRecord(ctx->gev[1], ctx->gstream), "event");
    CK(cudaStreamWaitEvent(ctx->stream, ctx->gev[1], 0), "event wait");
    // the outcome: status word, list totals and sums, with one synchronisation
    CK(cudaMemcpyAsync(ctx->h_status, ctx->status.p, 4, cudaMemcpyDeviceToHost, ctx->stream), "status readback");
    CK(cudaMemcpyAsync(ctx->h_tot, ctx->cap_need.p, 4 * 8, cudaMemcpyDeviceToHost, ctx->stream), "totals readback");
    CK(cudaMemcpyAsync(ctx->h_sums, ctx->sums.p, 16 * 8, cudaMemcpyDeviceToHost, ctx->stream), "sums readback");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    const uint32_t stw = *ctx->h_status;
    if (stw == 0u) {
      if (sums_out) memcpy(sums_out, ctx->h_sums, 16 * 8);
      return DMB_OK;
    }
    if (stw != DMB_BAD_OVERFLOW) return check_status(ctx);   // bad inputs: reported as the direct step would
    // a list outgrew its buffer: nothing was applied; regrow from the totals and run directly
    CK(cudaMemsetAsync(ctx->status.p, 0, 4, ctx->stream), "status reset");
    for (int k = 0; k < 4; ++k) grow[k] = ctx->h_tot[k];
    clear_batch_graph(ctx);
  }
  // the step itself, directly
  dmb_status st = step_body(ctx, dm, gas, step, dt, sums_out);
  if (st != DMB_OK) return st;
  // capacities for the replays: the sizes just found (or the overflowing totals) plus a quarter
  clear_batch_graph(ctx);
  const SearchBufs &sg = ctx->sg;
  auto cap = [](int64_t a, int64_t b) { return (a > b ? a : b) + (a > b ? a : b) / 4 + 4096; };
  dmb_ctx::BatchCaps c;
  c.items = cap(sg.n_items, grow[0]);
  c.units = cap(sg.n_units, grow[1]);
  c.pairs = cap(sg.n_pairs, grow[2]);
  c.segs = gas->n + c.pairs / ctx->shp.seg + 1;   // every row has at most len / seg + 1 segments
  bg.caps = c;
  if ((st = presize_batch(ctx)) != DMB_OK) return st;
  // capture on the library's stream
  cudaStream_t saved = ctx->stream;
  const int64_t l0 = ctx->launches;
  ctx->stream = ctx->gstream;
  ctx->capturing = true;
  ctx->pairs_dev = ptr<int64_t>(ctx->sg.row_ptr) + gas->n;
  ctx->gate_dev = ptr<uint32_t>(ctx->gate);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
  st = DMB_ERR_CUDA;
  if (e == cudaSuccess) {
    e = cudaMemsetAsync(ctx->gate.p, 0, 4, ctx->gstream);
    if (e == cudaSuccess) {
      st = step_body(ctx, dm, gas, step, dt, nullptr);
      if (st == DMB_OK) {
        const cudaError_t ei = launch_step_advance(ptr<unsigned long long>(ctx->step_dev), ctx->gstream, &ctx->launches);
        if (ei != cudaSuccess) st = cuda_fail(ctx, ei, "step counter");
      }
    } else {
      st = cuda_fail(ctx, e, "graph capture");
    }
    const cudaError_t e2 = cudaStreamEndCapture(ctx->gstream, &g);
    if (st == DMB_OK && e2 != cudaSuccess) st = cuda_fail(ctx, e2, "graph capture");
  } else {
    st = cuda_fail(ctx, e, "graph capture");
  }
  ctx->stream = saved;
  ctx->capturing = false;
  ctx->pairs_dev = nullptr;
  ctx->gate_dev = nullptr;
  bg.launches = ctx->launches - l0;
  ctx->launches = l0;
  if (st != DMB_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  e = cudaGraphInstantiate(&bg.exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    bg.exec = nullptr;
    return cuda_fail(ctx, e, "graph instantiate");
  }
  bg.valid = true;
  memcpy(bg.key, key, sizeof(key));
  bg.nd = dm->n;
  bg.ng = gas->n;
  bg.dt = dt;
  bg.boxes.assign(boxes, boxes + nbox);
  ctx->batch_next_step = ~0ull;
  return DMB_OK;
}

dmb_status dmb_set_bins(dmb_ctx *ctx, const uint8_t *dm_bin, const uint8_t *gas_bin) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!ctx->pairs_ready) return fail(ctx, DMB_ERR_STATE, "dmb_set_bins before dmb_neighbors");
  if (ctx->nbox > 0) return fail(ctx, DMB_ERR_ARG, "substeps run on a single box");
  if ((ctx->dm.n > 0 && !dm_bin) || (ctx->gas.n > 0 && !gas_bin)) return fail(ctx, DMB_ERR_ARG, "bin array is NULL");
  invalidate_substeps(ctx);
  return ctx->p.fp64 ? set_bins_impl<double>(ctx, dm_bin, gas_bin) : set_bins_impl<float>(ctx, dm_bin, gas_bin);
}

dmb_status dmb_rebin_dm(dmb_ctx *ctx, const float *p_ratio_max, uint8_t *dm_bin, int64_t n, int32_t max_bin,
                        uint64_t substep, const uint8_t *active, int64_t *n_changed) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (n < 0 || n > 0x7fffffffLL || (n > 0 && (!p_ratio_max || !dm_bin)))
    return fail(ctx, DMB_ERR_ARG, "NULL array or n outside [0, 2^31)");
  if (max_bin < 0 || max_bin >= DMB_NBINS) return fail(ctx, DMB_ERR_ARG, "max_bin must be in [0, 63]");
  if (!ensure(ctx->rebin_cnt, 8)) return fail(ctx, DMB_ERR_OOM, "device allocation failed");
  cudaStream_t s = ctx->stream;
  unsigned long long *cnt = ptr<unsigned long long>(ctx->rebin_cnt);
  CK(cudaMemsetAsync(cnt, 0, 8, s), "memset");
  CK(launch_rebin(p_ratio_max, dm_bin, n, max_bin, (unsigned long long)substep, active, cnt, s, &ctx->launches),
     "rebin");
  if (n_changed) {
    unsigned long long h = 0;
    CK(cudaMemcpyAsync(&h, cnt, 8, cudaMemcpyDeviceToHost, s), "readback");
    CK(cudaStreamSynchronize(s), "synchronise");
    *n_changed = (int64_t)h;
  }
  return DMB_OK;
}

dmb_status dmb_substep_info(dmb_ctx *ctx, uint64_t substep, int64_t *out5) {
  if (!ctx || !out5) return fail(ctx, DMB_ERR_ARG, "NULL argument");
  if (!ctx->bins_ready) return fail(ctx, DMB_ERR_STATE, "dmb_substep_info before dmb_set_bins");
  const int lim = substep_lim(substep);
  for (int k = 0; k < 5; ++k) out5[k] = ctx->bin_tab[k][lim];
  return DMB_OK;
}

dmb_status dmb_set_mc_variant(dmb_ctx *ctx, int32_t variant) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (variant != 0 && variant != 1) return fail(ctx, DMB_ERR_ARG, "variant must be 0 or 1");
  if (variant != ctx->mc_variant) {   // captured steps hold the old kernel
    clear_graphs(ctx);
    clear_batch_graph(ctx);
  }
  ctx->mc_variant = variant;
  return DMB_OK;
}

dmb_status dmb_set_fusion(dmb_ctx *ctx, int32_t on) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (on != 0 && on != 1) return fail(ctx, DMB_ERR_ARG, "on must be 0 or 1");
  if ((on == 1) != ctx->fuse) {
    clear_batch_graph(ctx);     // the captured step holds the other kernels
    ctx->pairs_ready = false;   // the search writes the pairs' gas-major positions only when fused
  }
  ctx->fuse = on == 1;
  return DMB_OK;
}

dmb_status dmb_set_pair_weights(dmb_ctx *ctx, int32_t mode) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (mode < -1 || mode > 1) return fail(ctx, DMB_ERR_ARG, "mode must be -1, 0 or 1");
  if (mode != ctx->weights_mode) {
    clear_batch_graph(ctx);     // the captured step holds the other kernels
    invalidate_substeps(ctx);
    ctx->pairs_ready = false;   // the next search decides again
    ctx->w_ready = false;
  }
  ctx->weights_mode = mode;
  return DMB_OK;
}

dmb_status dmb_set_surrogate_epilogue(dmb_ctx *ctx, int32_t mode) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (mode != 0 && mode != 1) return fail(ctx, DMB_ERR_ARG, "mode must be 0 or 1");
  if (mode != ctx->tc_epilogue) {
    clear_batch_graph(ctx);     // the captured step holds the other kernels
    invalidate_substeps(ctx);
  }
  ctx->tc_epilogue = mode;
  return DMB_OK;
}

dmb_status dmb_set_surrogate_scope(dmb_ctx *ctx, int32_t scope) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (scope != 0 && scope != 1) return fail(ctx, DMB_ERR_ARG, "scope must be 0 (the scan's indices) or 1 (n only)");
  ctx->mlp_scope = scope;
  return DMB_OK;
}

dmb_status dmb_set_cross_section(dmb_ctx *ctx, int32_t family, double v_c_kms) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (family != 0 && family != 1) return fail(ctx, DMB_ERR_ARG, "family must be 0 (power law) or 1 (screened law)");
  if (family == 1 && !(v_c_kms > 0.0 && isfinite(v_c_kms))) return fail(ctx, DMB_ERR_ARG, "v_c must be finite and > 0");
  if (family == 1 && ctx->rc.rate_mode == DMB_RATE_CLOSED)
    return fail(ctx, DMB_ERR_ARG, "the closed forms exist for the power law only: use the quadrature or the surrogate");
  const double vc = family == 1 ? v_c_kms : 0.0;
  if (family != ctx->xsec || vc != ctx->v_c) {
    invalidate_substeps(ctx);      // substep tables and captured graphs hold the old constants
    ctx->grid_ready = false;       // the gas coefficients of the sorted copy carry the normalisation
    ctx->pairs_ready = false;
  }
  ctx->xsec = family;
  ctx->v_c = vc;
  ctx->rc.xsec = family;
  ctx->rc.inv_vc2 = family == 1 ? 1.0 / (vc * vc) : 0.0;
  ctx->rc.n = family == 1 ? 0 : ctx->p.n;
  ctx->rc.alpha = alpha_of(ctx->rc.n);
  return DMB_OK;
}

dmb_status dmb_debug_rates_screened(dmb_ctx *ctx, int64_t k, const double *in, double *out) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (k < 0 || (k > 0 && (!in || !out))) return fail(ctx, DMB_ERR_ARG, "bad arguments");
  CK(launch_debug_rates_screened(ctx->p.fp64, alpha_of(0), k, in, out, ctx->stream), "debug rates (screened)");
  return DMB_OK;
}

dmb_status dmb_set_anisotropy(dmb_ctx *ctx, double beta) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!(beta >= -1.0 && beta <= 1.0)) return fail(ctx, DMB_ERR_ARG, "beta must lie in [-1, 1]");
  if (beta != ctx->mc_beta) {
    invalidate_substeps(ctx);      // substep tables and captured graphs hold the old constants
    ctx->grid_ready = false;       // the gas coefficients of the sorted copy carry sigma_bar
    ctx->pairs_ready = false;
  }
  ctx->mc_beta = beta;
  ctx->rc.sbar = 1.0 - beta / 3.0;
  return DMB_OK;
}

dmb_status dmb_set_graph(dmb_ctx *ctx, int on) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  ctx->use_graph = on != 0;
  if (!ctx->use_graph) clear_batch_graph(ctx);
  return DMB_OK;
}

dmb_status dmb_substep(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, uint64_t substep, double dt_min,
                       double *sums_out) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!ctx->bins_ready) return fail(ctx, DMB_ERR_STATE, "dmb_substep before dmb_set_bins");
  dmb_status st;
  if ((st = check_dm(ctx, dm)) != DMB_OK || (st = check_gas(ctx, gas)) != DMB_OK) return st;
  if (dm->n != ctx->dm.n || gas->n != ctx->gas.n) return fail(ctx, DMB_ERR_ARG, "particle counts differ from the grid");
  if (!(dt_min >= 0.0) || !isfinite(dt_min)) return fail(ctx, DMB_ERR_ARG, "dt_min must be finite and >= 0");
  if (ctx->rc.rate_mode == DMB_RATE_MLP) {
    if (!ctx->mlp_ready) return fail(ctx, DMB_ERR_STATE, "surrogate rate provider selected but no trained network");
    if (!surrogate_covers(ctx))
      return fail(ctx, DMB_ERR_DOMAIN, "the surrogate was not trained for this cross section (law or power-law index)");
  }
  const int lim = substep_lim(substep);
  if (ctx->use_graph) {
    st = substep_graph(ctx, dm, gas, lim, substep, dt_min);
  } else {
    st = ctx->p.fp64 ? substep_body<double>(ctx, dm, gas, lim, substep, dt_min, false)
                     : substep_body<float>(ctx, dm, gas, lim, substep, dt_min, false);
    ctx->graph_next_step = ~0ull;
  }
  if (st != DMB_OK) return st;
  if (sums_out) {
    CK(cudaMemcpyAsync(ctx->h_sums, ctx->sums.p, 16 * 8, cudaMemcpyDeviceToHost, ctx->stream), "sums readback");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    memcpy(sums_out, ctx->h_sums, 16 * 8);
  }
  return DMB_OK;
}

}  // extern "C"

// ---- autotuner of the launch shapes ----------------------------------------------------------
static dmb_status check_shapes(dmb_ctx *ctx, const int32_t *v) {
  if (v[0] < 4 || v[0] > 1024 || v[1] < 128 || v[1] > 65536 || v[2] < 1 || v[2] > 64 || v[3] < 1 || v[3] > 64 ||
      v[4] < 2 || v[4] > 4)
    return fail(ctx, DMB_ERR_ARG, "shapes out of range: unit [4, 1024], seg [128, 65536], blocks per SM [1, 64], "
                                  "surrogate warpgroups 2..4");
  return DMB_OK;
}

static void set_shapes(dmb_ctx *ctx, const int32_t *v) {
  ctx->shp.unit = v[0];
  ctx->shp.seg = v[1];
  ctx->shp.mf_bps = v[2];
  ctx->shp.mc_bps = v[3];
  ctx->shp.tc_wg = v[4];
  invalidate_substeps(ctx);   // substep tables and graphs were built with the old shapes
  ctx->pairs_ready = false;   // the search units and mean-field segments follow the shapes
}

static void get_shapes(const dmb_ctx *ctx, int32_t *v) {
  v[0] = ctx->shp.unit;
  v[1] = ctx->shp.seg;
  v[2] = ctx->shp.mf_bps;
  v[3] = ctx->shp.mc_bps;
  v[4] = ctx->shp.tc_wg;
}

// device time of one call of f (ms, events on the context stream); the call runs twice and the
// second (warm) run is the one timed
template <typename F>
static dmb_status time_call(dmb_ctx *ctx, cudaEvent_t e0, cudaEvent_t e1, F f, float *ms) {
  dmb_status st;
  if ((st = f()) != DMB_OK) return st;
  CK(cudaEventRecord(e0, ctx->stream), "event");
  if ((st = f()) != DMB_OK) return st;
  CK(cudaEventRecord(e1, ctx->stream), "event");
  CK(cudaEventSynchronize(e1), "event sync");
  CK(cudaEventElapsedTime(ms, e0, e1), "event time");
  return DMB_OK;
}

template <typename R>
static dmb_status autotune_impl(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, cudaEvent_t e0, cudaEvent_t e1,
                                double *report) {
  dmb_status st;
  float ms = 0.f;
  int k = 0;
  // 1. search work units (target leaves per unit): neighbours on the built grid
  if ((st = build_grid_checked(ctx, dm, gas)) != DMB_OK) return st;
  float best = 1e30f;
  int best_unit = ctx->shp.unit;
  for (int unit : {16, 32, 64, 128}) {
    ctx->shp.unit = unit;
    if ((st = time_call(ctx, e0, e1, [&]() { return neighbors_impl<R>(ctx); }, &ms)) != DMB_OK) return st;
    if (report) report[k++] = ms;
    if (ms < best) { best = ms; best_unit = unit; }
  }
  ctx->shp.unit = best_unit;
  if ((st = neighbors_impl<R>(ctx)) != DMB_OK) return st;
  // 2. mean field: segment length x blocks per SM (and the surrogate's warpgroups)
  const int64_t ng = gas->n, nd = dm->n;
  if (!ensure(ctx->mf_acc, ng * 24) || !ensure(ctx->mf_dudt, ng * 8) || !ensure(ctx->e_exp, ng * 8) ||
      !ensure(ctx->scratch_vel, nd * 24 + 8))
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for autotuner scratch");
  auto mf = [&]() {
    return meanfield_impl<R>(ctx, ptr<double>(ctx->mf_acc), ptr<double>(ctx->mf_dudt), ptr<double>(ctx->e_exp));
  };
  best = 1e30f;
  int best_seg = ctx->shp.seg, best_mf = ctx->shp.mf_bps;
  for (int seg : {512, 1024, 2048, 4096}) {
    ctx->shp.seg = seg;
    if ((st = build_segments(ctx, ctx->sg, ng)) != DMB_OK) return st;
    for (int bps : {8, 16, 32}) {
      ctx->shp.mf_bps = bps;
      if ((st = time_call(ctx, e0, e1, mf, &ms)) != DMB_OK) return st;
      if (report) report[k++] = ms;
      if (ms < best) { best = ms; best_seg = seg; best_mf = bps; }
    }
  }
  ctx->shp.seg = best_seg;
  ctx->shp.mf_bps = best_mf;
  if ((st = build_segments(ctx, ctx->sg, ng)) != DMB_OK) return st;
  if (ctx->rc.rate_mode == DMB_RATE_MLP && sizeof(R) == 4 && ctx->mlp_ready && ctx->mlp_engine == 0) {
    best = 1e30f;
    int best_wg = ctx->shp.tc_wg;
    for (int wg : {2, 3, 4}) {
      ctx->shp.tc_wg = wg;
      if ((st = time_call(ctx, e0, e1, mf, &ms)) != DMB_OK) return st;
      if (report) report[k++] = ms;
      if (ms < best) { best = ms; best_wg = wg; }
    }
    ctx->shp.tc_wg = best_wg;
  }
  // 3. Monte Carlo blocks per SM (the caller's velocities are read, the scratch written)
  best = 1e30f;
  int best_mc = ctx->shp.mc_bps;
  for (int bps : {4, 8, 16, 32}) {
    ctx->shp.mc_bps = bps;
    if ((st = time_call(ctx, e0, e1, [&]() {
           return mc_impl<R>(ctx, 0, 0.0, ptr<double>(ctx->scratch_vel), nullptr, nullptr, nullptr, nullptr);
         }, &ms)) != DMB_OK)
      return st;
    if (report) report[k++] = ms;
    if (ms < best) { best = ms; best_mc = bps; }
  }
  ctx->shp.mc_bps = best_mc;
  return check_status(ctx);
}

extern "C" {

dmb_status dmb_autotune(dmb_ctx *ctx, const dmb_dm *dm, const dmb_gas *gas, int32_t *shapes_out, double *report) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  dmb_status st;
  if ((st = check_dm(ctx, dm)) != DMB_OK || (st = check_gas(ctx, gas)) != DMB_OK) return st;
  if (ctx->nbox > 0) return fail(ctx, DMB_ERR_ARG, "autotune a single-box context");
  if (ctx->rc.rate_mode == DMB_RATE_MLP && !ctx->mlp_ready)
    return fail(ctx, DMB_ERR_STATE, "surrogate rate provider selected but no trained network");
  invalidate_substeps(ctx);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0), "event create");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(ctx, DMB_ERR_CUDA, "event create");
  }
  const bool timing = ctx->timing;
  ctx->timing = false;
  st = ctx->p.fp64 ? autotune_impl<double>(ctx, dm, gas, e0, e1, report)
                   : autotune_impl<float>(ctx, dm, gas, e0, e1, report);
  ctx->timing = timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DMB_OK) return st;
  if (shapes_out) get_shapes(ctx, shapes_out);
  return DMB_OK;
}

dmb_status dmb_set_shapes(dmb_ctx *ctx, const int32_t *shapes) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!shapes) return fail(ctx, DMB_ERR_ARG, "shapes is NULL");
  dmb_status st;
  if ((st = check_shapes(ctx, shapes)) != DMB_OK) return st;
  set_shapes(ctx, shapes);
  return DMB_OK;
}

dmb_status dmb_get_shapes(dmb_ctx *ctx, int32_t *shapes_out) {
  if (!ctx || !shapes_out) return fail(ctx, DMB_ERR_ARG, "NULL argument");
  get_shapes(ctx, shapes_out);
  return DMB_OK;
}

// ---- persisted launch shapes -----------------------------------------------------------------
// The file is one JSON object {"key": [unit, seg, mf_blocks, mc_blocks, warpgroups], ...}; keys are
// made of letters, digits and "._+-".  Read and written whole, entries of other keys kept.
static bool shapes_key_ok(const char *k) {
  if (!k || !*k) return false;
  for (const char *c = k; *c; ++c)
    if (!(isalnum((unsigned char)*c) || *c == '.' || *c == '_' || *c == '+' || *c == '-')) return false;
  return strlen(k) < 200;
}

static std::vector<std::pair<std::string, std::vector<long>>> shapes_read(const char *path) {
  std::vector<std::pair<std::string, std::vector<long>>> out;
  FILE *f = fopen(path, "rb");
  if (!f) return out;
  std::string txt;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof(buf), f)) > 0 && txt.size() < (1u << 20)) txt.append(buf, n);
  fclose(f);
  size_t i = 0;
  while ((i = txt.find('"', i)) != std::string::npos) {
    const size_t j = txt.find('"', i + 1);
    if (j == std::string::npos) break;
    std::string key = txt.substr(i + 1, j - i - 1);
    const size_t a = txt.find('[', j), b = txt.find(']', j);
    if (a == std::string::npos || b == std::string::npos || b < a) break;
    std::vector<long> v;
    const char *c = txt.c_str() + a + 1;
    while (c < txt.c_str() + b) {
      char *end = nullptr;
      const long x = strtol(c, &end, 10);
      if (end == c) { ++c; continue; }
      v.push_back(x);
      c = end;
    }
    out.emplace_back(key, v);
    i = b + 1;
  }
  return out;
}

dmb_status dmb_save_shapes(dmb_ctx *ctx, const char *path, const char *key) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!path || !shapes_key_ok(key)) return fail(ctx, DMB_ERR_ARG, "path is NULL or the key is not [A-Za-z0-9._+-]+");
  auto entries = shapes_read(path);
  int32_t v[5];
  get_shapes(ctx, v);
  std::vector<long> cur(v, v + 5);
  bool found = false;
  for (auto &e : entries)
    if (e.first == key) { e.second = cur; found = true; }
  if (!found) entries.emplace_back(key, cur);
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "wb");
  if (!f) return fail(ctx, DMB_ERR_ARG, "cannot write the shapes file");
  fprintf(f, "{\n");
  for (size_t k = 0; k < entries.size(); ++k) {
    fprintf(f, "  \"%s\": [", entries[k].first.c_str());
    for (size_t m = 0; m < entries[k].second.size(); ++m) fprintf(f, "%s%ld", m ? ", " : "", entries[k].second[m]);
    fprintf(f, "]%s\n", k + 1 < entries.size() ? "," : "");
  }
  fprintf(f, "}\n");
  const bool ok = fclose(f) == 0 && rename(tmp.c_str(), path) == 0;
  if (!ok) return fail(ctx, DMB_ERR_ARG, "cannot write the shapes file");
  return DMB_OK;
}

dmb_status dmb_load_shapes(dmb_ctx *ctx, const char *path, const char *key) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!path || !shapes_key_ok(key)) return fail(ctx, DMB_ERR_ARG, "path is NULL or the key is not [A-Za-z0-9._+-]+");
  for (auto &e : shapes_read(path)) {
    if (e.first != key) continue;
    if (e.second.size() != 5) return fail(ctx, DMB_ERR_ARG, "malformed shapes entry");
    int32_t v[5];
    for (int k = 0; k < 5; ++k) v[k] = (int32_t)e.second[k];
    dmb_status st;
    if ((st = check_shapes(ctx, v)) != DMB_OK) return st;
    set_shapes(ctx, v);
    return DMB_OK;
  }
  return fail(ctx, DMB_ERR_STATE, "no shapes stored under this key");
}

dmb_status dmb_set_timing(dmb_ctx *ctx, int on) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (on && !ctx->ev[0]) {
    for (int k = 0; k < 6; ++k) CK(cudaEventCreate(&ctx->ev[k]), "event create");
    for (int k = 0; k < 2; ++k) CK(cudaEventCreate(&ctx->sev[k]), "event create");
  }
  ctx->timing = on != 0;
  for (int k = 0; k < 8; ++k) ctx->stage_ms[k] = 0.0;
  ctx->timed_steps = 0;
  return DMB_OK;
}

dmb_status dmb_stage_times(dmb_ctx *ctx, double *ms_out, int64_t *steps_out) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (ms_out) for (int k = 0; k < 8; ++k) ms_out[k] = ctx->stage_ms[k];
  if (steps_out) *steps_out = ctx->timed_steps;
  for (int k = 0; k < 8; ++k) ctx->stage_ms[k] = 0.0;
  ctx->timed_steps = 0;
  return DMB_OK;
}

// ---- surrogate entry points ---------------------------------------------------------------
dmb_status dmb_train_surrogate(dmb_ctx *ctx, int64_t nsamples, int32_t epochs, uint64_t seed, double *report) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (nsamples < 4096 * 2 || nsamples > (1ll << 27) || epochs < 1 || epochs > 10000)
    return fail(ctx, DMB_ERR_ARG, "nsamples must be in [8192, 2^27] and epochs in [1, 10000]");
  dmb_status st;
  if ((st = ensure_mlp(ctx)) != DMB_OK) return st;
  cudaStream_t s = ctx->stream;
  const auto t0 = std::chrono::steady_clock::now();
  // training box and power-law indices: {-4, -2, 0, 2} and the context's n
  // the samples reach a quarter decade beyond the box in tau and m_chi (the box the network answers
  // for is unchanged), so that its corners are not the edge of what it has seen
  MlpDataSpec spec;
  const double margin = 0.25;
  spec.log_s_lo = ctx->mlp_box[0]; spec.log_s_hi = ctx->mlp_box[1];
  spec.log_tau_lo = ctx->mlp_box[2] - margin; spec.log_tau_hi = ctx->mlp_box[3] + margin;
  spec.log_m_lo = ctx->mlp_box[4] - margin; spec.log_m_hi = ctx->mlp_box[5] + margin;
  // the screened law has one normalisation (n = 0) and takes tau as varsigma^2 / v_c^2
  std::vector<int> ns = {-4, -2, 0, 2};
  if (std::find(ns.begin(), ns.end(), ctx->p.n) == ns.end()) ns.push_back(ctx->p.n);
  if (ctx->mlp_scope == 1) ns = {ctx->p.n};
  if (ctx->xsec == 1) ns = {0};
  spec.scr = ctx->xsec == 1 ? 1 : 0;
  // n = -4 (the 1F1 with the most curvature across the envelope's transition) is drawn three times
  // as often
  std::vector<int> draw = ns;
  if (std::find(ns.begin(), ns.end(), -4) != ns.end() && ns.size() > 1) draw.insert(draw.end(), {-4, -4});
  spec.n_count = (int)draw.size();
  for (int k = 0; k < spec.n_count; ++k) {
    spec.n_values[k] = draw[k];
    spec.alpha[k] = alpha_of(draw[k]);
    envelope(draw[k], spec.envA[k], spec.envB[k]);
  }
  const int B = 4096;
  const int64_t N = nsamples, Nval = N / 10, Ntr = N - Nval;
  DevBuf X, Y, idx, A1, A2, Z1, Z2, Z3, A3, dY, loss, dZ3, dZ2, dZ1, part2, part3, grad, Yv;
  const size_t BH = (size_t)B * MLP_H;
  bool ok = ensure(X, N * 16) && ensure(Y, N * 8) && ensure(idx, Ntr * 4) && ensure(A1, BH * 2) && ensure(A2, BH * 2) &&
            ensure(Z1, BH * 4) && ensure(Z2, BH * 4) && ensure(Z3, BH * 4) && ensure(A3, BH * 4) && ensure(dY, B * 8) &&
            ensure(loss, MLP_TRAIN_BLOCKS * 4) && ensure(dZ3, BH * 2) && ensure(dZ2, BH * 2) && ensure(dZ1, BH * 4) &&
            ensure(part2, (size_t)MLP_KSLICES * MLP_H * MLP_H * 4) && ensure(part3, (size_t)MLP_KSLICES * MLP_H * MLP_H * 4) &&
            ensure(grad, MLP_NPARAM * 4) && ensure(Yv, Nval * 8);
  auto cleanup = [&]() { for (DevBuf *b : {&X, &Y, &idx, &A1, &A2, &Z1, &Z2, &Z3, &A3, &dY, &loss, &dZ3, &dZ2, &dZ1, &part2, &part3, &grad, &Yv}) release(*b); };
  if (!ok) { cleanup(); return fail(ctx, DMB_ERR_OOM, "device allocation failed for surrogate training"); }
  cudaError_t e = mlp_make_data(spec, N, seed, ptr<float>(X), ptr<float>(Y), s);
  // initial weights: uniform(-sqrt(3/fan_in), sqrt(3/fan_in)), zero biases, small output layer
  std::vector<float> p0(MLP_NPARAM, 0.0f);
  std::mt19937_64 rng(seed ^ 0x9e3779b97f4a7c15ull);
  auto fill = [&](int off, int count, int fan_in, float scale) {
    std::uniform_real_distribution<float> U(-1.0f, 1.0f);
    const float b = scale * sqrtf(3.0f / (float)fan_in);
    for (int k = 0; k < count; ++k) p0[off + k] = b * U(rng);
  };
  fill(MLP_OFF_W1, MLP_H * MLP_IN, MLP_IN, 1.0f);
  fill(MLP_OFF_W2, MLP_H * MLP_H, MLP_H, 1.0f);
  fill(MLP_OFF_W3, MLP_H * MLP_H, MLP_H, 1.0f);
  fill(MLP_OFF_W4, MLP_OUT * MLP_H, MLP_H, 0.1f);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->mlp_p.p, p0.data(), MLP_NPARAM * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->mlp_m.p, 0, MLP_NPARAM * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->mlp_v.p, 0, MLP_NPARAM * 4, s);
  MlpDev d = mlp_dev(ctx);
  if (e == cudaSuccess) e = mlp_refresh(d, s);
  MlpWork w;
  w.A1 = ptr<__nv_bfloat16>(A1); w.A2 = ptr<__nv_bfloat16>(A2); w.dZ3 = ptr<__nv_bfloat16>(dZ3); w.dZ2 = ptr<__nv_bfloat16>(dZ2);
  w.Z1 = ptr<float>(Z1); w.Z2 = ptr<float>(Z2); w.Z3 = ptr<float>(Z3); w.A3 = ptr<float>(A3); w.dY = ptr<float>(dY);
  w.loss = ptr<float>(loss); w.dZ1 = ptr<float>(dZ1); w.part2 = ptr<float>(part2); w.part3 = ptr<float>(part3);
  w.grad = ptr<float>(grad);
  const int steps_per_epoch = (int)(Ntr / B);
  const int total = steps_per_epoch * epochs;
  std::vector<int> perm(Ntr);
  for (int64_t k = 0; k < Ntr; ++k) perm[k] = (int)k;
  int t_adam = 0;
  const float lr0 = 2e-3f, lr1 = 2e-5f;
  // The last quarter of the epochs weights the worst-fitted samples: every fourth of those epochs the
  // network's error on every training sample is measured, and each epoch then draws the worst eighth
  // four times over and a random half of the rest, so the worst-case error falls with the mean.
  const int hard_from = epochs >= 8 ? epochs - epochs / 4 : epochs;
  std::vector<float> yp, yh;
  std::vector<int> order;
  DevBuf Yp;
  if (hard_from < epochs && !ensure(Yp, (size_t)Ntr * 8)) {
    cleanup();
    return fail(ctx, DMB_ERR_OOM, "device allocation failed for surrogate training");
  }
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    if (ep >= hard_from) {
      if ((ep - hard_from) % 4 == 0) {
        yp.resize((size_t)Ntr * 2);
        yh.resize((size_t)Ntr * 2);
        e = mlp_infer(d, ptr<float>(X), Ntr, ptr<float>(Yp), s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(yp.data(), Yp.p, (size_t)Ntr * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(yh.data(), Y.p, (size_t)Ntr * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        std::vector<float> err(Ntr);
        for (int64_t k = 0; k < Ntr; ++k)
          err[k] = fmaxf(fabsf(yp[2 * k] - yh[2 * k]), fabsf(yp[2 * k + 1] - yh[2 * k + 1]));
        order.resize(Ntr);
        for (int64_t k = 0; k < Ntr; ++k) order[k] = (int)k;
        const int64_t nh = Ntr / 8;
        std::nth_element(order.begin(), order.begin() + nh, order.end(),
                         [&](int a, int b) { return err[a] > err[b]; });
      }
      // worst eighth x 4 + half of the rest = Ntr draws
      const int64_t nh = Ntr / 8;
      std::shuffle(order.begin() + nh, order.end(), rng);
      int64_t q = 0;
      for (int rep = 0; rep < 4; ++rep)
        for (int64_t k = 0; k < nh && q < Ntr; ++k) perm[q++] = order[k];
      for (int64_t k = nh; q < Ntr; ++k) perm[q++] = order[k];
      std::shuffle(perm.begin(), perm.end(), rng);
    } else {
      std::shuffle(perm.begin(), perm.end(), rng);
    }
    e = cudaMemcpyAsync(idx.p, perm.data(), Ntr * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // perm is reused next epoch
    for (int b = 0; b < steps_per_epoch && e == cudaSuccess; ++b) {
      ++t_adam;
      const float frac = (float)t_adam / (float)total;
      const float lr = lr1 + 0.5f * (lr0 - lr1) * (1.0f + cosf(3.14159265f * frac));
      e = mlp_train_batch(d, ptr<float>(X), ptr<float>(Y), ptr<int>(idx) + (size_t)b * B, B, w, lr, t_adam, s,
                          &ctx->launches);
    }
  }
  release(Yp);
  // last batch loss and the validation errors of FA, FB (relative), on the engine that evaluates
  // the pairs, over the held-out samples inside the box the network answers for
  std::vector<float> lossh(MLP_TRAIN_BLOCKS), yv(Nval * 2), yt(Nval * 2), xv(Nval * 4);
  if (e == cudaSuccess) {
    if (ctx->mlp_engine == 0) {
      TcArgs ta = {};
      ta.p = d.p;
      ta.w2 = d.w2;
      ta.w3 = d.w3;
      ta.n = Nval;
      ta.X = ptr<float>(X) + Ntr * 4;
      ta.Y = ptr<float>(Yv);
      ta.status = ptr<uint32_t>(ctx->status);
      e = mlp_tc_infer(ta, ctx->shp.tc_wg, s, &ctx->launches);
    } else {
      e = mlp_infer(d, ptr<float>(X) + Ntr * 4, Nval, ptr<float>(Yv), s);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(lossh.data(), loss.p, MLP_TRAIN_BLOCKS * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(yv.data(), Yv.p, Nval * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(yt.data(), ptr<float>(Y) + Ntr * 2, Nval * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(xv.data(), ptr<float>(X) + Ntr * 4, Nval * 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "surrogate training");
  double lsum = 0.0;
  for (float v : lossh) lsum += v;
  double mxA = 0, mxB = 0, meA = 0, meB = 0;
  int64_t nin = 0;
  for (int64_t k = 0; k < Nval; ++k) {
    const double lt = 2.0 * (double)xv[4 * k + 1], lm = (double)xv[4 * k + 2];
    if (lt < ctx->mlp_box[2] || lt > ctx->mlp_box[3] || lm < ctx->mlp_box[4] || lm > ctx->mlp_box[5]) continue;
    const double ea = fabs(expm1((double)yv[2 * k] - (double)yt[2 * k]));
    const double eb = fabs(expm1((double)yv[2 * k + 1] - (double)yt[2 * k + 1]));
    mxA = fmax(mxA, ea); mxB = fmax(mxB, eb); meA += ea; meB += eb;
    ++nin;
  }
  if (nin == 0) nin = 1;
  ctx->mlp_ready = true;
  ctx->mlp_n = ns;
  ctx->mlp_family = ctx->xsec;
  if (report) {
    report[0] = lsum / ((double)B * MLP_OUT);
    report[1] = mxA;
    report[2] = mxB;
    report[3] = meA / (double)nin;
    report[4] = meB / (double)nin;
    report[5] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    report[6] = (double)t_adam;
    report[7] = (double)N;
  }
  return DMB_OK;
}

dmb_status dmb_surrogate_params(dmb_ctx *ctx, float *host_out, int64_t *count) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (count) *count = MLP_NPARAM;
  if (!host_out) return DMB_OK;
  if (!ctx->mlp_ready) return fail(ctx, DMB_ERR_STATE, "no surrogate loaded");
  CK(cudaMemcpyAsync(host_out, ctx->mlp_p.p, MLP_NPARAM * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy");
  CK(cudaStreamSynchronize(ctx->stream), "synchronise");
  return DMB_OK;
}

dmb_status dmb_load_surrogate(dmb_ctx *ctx, const float *host_params, int64_t count) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!host_params || count != MLP_NPARAM) return fail(ctx, DMB_ERR_ARG, "expected the full parameter block");
  dmb_status st;
  if ((st = ensure_mlp(ctx)) != DMB_OK) return st;
  CK(cudaMemcpyAsync(ctx->mlp_p.p, host_params, MLP_NPARAM * 4, cudaMemcpyHostToDevice, ctx->stream), "copy");
  MlpDev d = mlp_dev(ctx);
  CK(mlp_refresh(d, ctx->stream), "refresh");
  CK(cudaStreamSynchronize(ctx->stream), "synchronise");
  ctx->mlp_ready = true;
  ctx->mlp_n = {-4, -2, 0, 2};
  if (std::find(ctx->mlp_n.begin(), ctx->mlp_n.end(), ctx->p.n) == ctx->mlp_n.end()) ctx->mlp_n.push_back(ctx->p.n);
  ctx->mlp_family = ctx->xsec;   // a loaded block is taken as a network of the current velocity law
  return DMB_OK;
}

dmb_status dmb_surrogate_infer(dmb_ctx *ctx, const float *X, int64_t n, float *Y) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!ctx->mlp_ready) return fail(ctx, DMB_ERR_STATE, "no surrogate loaded");
  CK(mlp_infer(mlp_dev(ctx), X, n, Y, ctx->stream), "surrogate inference");
  return DMB_OK;
}

dmb_status dmb_surrogate_grad(dmb_ctx *ctx, const float *X, const float *Y, int32_t B, float *grad, double *loss) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!ctx->mlp_ready) return fail(ctx, DMB_ERR_STATE, "no surrogate loaded");
  if (B < 1 || B > (1 << 20)) return fail(ctx, DMB_ERR_ARG, "batch size out of range");
  cudaStream_t s = ctx->stream;
  DevBuf idx, A1, A2, Z1, Z2, Z3, A3, dY, lossb, dZ3, dZ2, dZ1, part2, part3;
  const size_t BH = (size_t)B * MLP_H;
  bool ok = ensure(idx, (size_t)B * 4) && ensure(A1, BH * 2) && ensure(A2, BH * 2) && ensure(Z1, BH * 4) &&
            ensure(Z2, BH * 4) && ensure(Z3, BH * 4) && ensure(A3, BH * 4) && ensure(dY, (size_t)B * 8) &&
            ensure(lossb, MLP_TRAIN_BLOCKS * 4) && ensure(dZ3, BH * 2) && ensure(dZ2, BH * 2) && ensure(dZ1, BH * 4) &&
            ensure(part2, (size_t)MLP_KSLICES * MLP_H * MLP_H * 4) && ensure(part3, (size_t)MLP_KSLICES * MLP_H * MLP_H * 4);
  auto cleanup = [&]() { for (DevBuf *b : {&idx, &A1, &A2, &Z1, &Z2, &Z3, &A3, &dY, &lossb, &dZ3, &dZ2, &dZ1, &part2, &part3}) release(*b); };
  if (!ok) { cleanup(); return fail(ctx, DMB_ERR_OOM, "device allocation failed"); }
  std::vector<int> id(B);
  for (int k = 0; k < B; ++k) id[k] = k;
  MlpWork w;
  w.A1 = ptr<__nv_bfloat16>(A1); w.A2 = ptr<__nv_bfloat16>(A2); w.dZ3 = ptr<__nv_bfloat16>(dZ3); w.dZ2 = ptr<__nv_bfloat16>(dZ2);
  w.Z1 = ptr<float>(Z1); w.Z2 = ptr<float>(Z2); w.Z3 = ptr<float>(Z3); w.A3 = ptr<float>(A3); w.dY = ptr<float>(dY);
  w.loss = ptr<float>(lossb); w.dZ1 = ptr<float>(dZ1); w.part2 = ptr<float>(part2); w.part3 = ptr<float>(part3);
  w.grad = grad;
  MlpDev d = mlp_dev(ctx);
  std::vector<float> lh(MLP_TRAIN_BLOCKS);
  cudaError_t e = cudaMemcpyAsync(idx.p, id.data(), (size_t)B * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = mlp_grad(d, X, Y, ptr<int>(idx), B, w, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(lh.data(), lossb.p, MLP_TRAIN_BLOCKS * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "surrogate gradient");
  if (loss) {
    double t = 0.0;
    for (float v : lh) t += v;
    *loss = t / (double)B;   // mean over samples of the summed squared error of the two outputs
  }
  return DMB_OK;
}

dmb_status dmb_set_surrogate_engine(dmb_ctx *ctx, int32_t engine) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (engine != 0 && engine != 1) return fail(ctx, DMB_ERR_ARG, "engine must be 0 (tcgen05) or 1 (mma.sync)");
  ctx->mlp_engine = engine;
  clear_graphs(ctx);   // captured steps hold the other engine's launches
  clear_batch_graph(ctx);
  return DMB_OK;
}

dmb_status dmb_surrogate_infer_tc(dmb_ctx *ctx, const float *X, int64_t n, float *Y) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!ctx->mlp_ready) return fail(ctx, DMB_ERR_STATE, "no surrogate loaded");
  if (n < 0 || (n > 0 && (!X || !Y))) return fail(ctx, DMB_ERR_ARG, "bad arguments");
  MlpRun mr = mlp_run(ctx);
  TcArgs a = {};
  a.p = mr.p;
  a.w2 = mr.w2;
  a.w3 = mr.w3;
  a.n = n;
  a.X = X;
  a.Y = Y;
  a.status = ptr<uint32_t>(ctx->status);
  a.skip_commit = ctx->tc_skip_commit ? 1 : 0;
  ctx->tc_skip_commit = false;
  CK(mlp_tc_infer(a, ctx->shp.tc_wg, ctx->stream, &ctx->launches), "surrogate inference (tensor cores)");
  return check_status(ctx);
}

dmb_status dmb_debug_tc_timeout(dmb_ctx *ctx, int32_t on) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (on != 0 && on != 1) return fail(ctx, DMB_ERR_ARG, "on must be 0 or 1");
  ctx->tc_skip_commit = on == 1;
  return DMB_OK;
}

dmb_status dmb_surrogate_fallbacks(dmb_ctx *ctx, int64_t *out) {
  if (!ctx || !out) return fail(ctx, DMB_ERR_ARG, "NULL argument");
  *out = 0;
  if (!ctx->mlp_fallback.p) return DMB_OK;
  unsigned long long v = 0;
  CK(cudaMemcpyAsync(&v, ctx->mlp_fallback.p, 8, cudaMemcpyDeviceToHost, ctx->stream), "copy");
  CK(cudaStreamSynchronize(ctx->stream), "synchronise");
  *out = (int64_t)v;
  return DMB_OK;
}

dmb_status dmb_search_stats(dmb_ctx *ctx, uint64_t *out16) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  if (!out16) return fail(ctx, DMB_ERR_ARG, "out is NULL");
  CK(cudaMemcpyAsync(out16, ctx->search_stats.p, 16 * 8, cudaMemcpyDeviceToHost, ctx->stream), "stats readback");
  CK(cudaStreamSynchronize(ctx->stream), "synchronise");
  return DMB_OK;
}

dmb_status dmb_debug_overlap(dmb_ctx *ctx, int64_t k, const double *in, double *out) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  CK(launch_debug_overlap(ptr<float4>(ctx->gtab), ctx->p.fp64, k, in, out, ctx->stream), "debug overlap");
  return DMB_OK;
}

dmb_status dmb_debug_rates(dmb_ctx *ctx, int64_t k, const double *in, double *out) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  CK(launch_debug_rates(ctx->p.fp64, ctx->p.n, ctx->rc.rate_mode, ctx->rc.alpha, k, in, out, ctx->stream),
     "debug rates");
  return DMB_OK;
}

dmb_status dmb_debug_philox(dmb_ctx *ctx, int64_t k, const uint32_t *ctr, uint32_t *out) {
  if (!ctx) return fail(nullptr, DMB_ERR_ARG, "ctx is NULL");
  CK(launch_debug_philox(k, ctr, out, ctx->p.seed, ctx->stream), "debug philox");
  return DMB_OK;
}

}  // extern "C"
