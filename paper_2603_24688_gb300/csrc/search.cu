// Pair search on the 32-ary chunk trees, in two stages:
//   1. per query leaf, the target leaves whose boxes come within h_max + h_max (lane-parallel
//      tests of the 32 children of every visited node), listed in depth-first order;
//   2. those lists cut into work units of at most `unit` target leaves; one warp per unit
//      tests its 32 query particles against each target leaf (targets outside the query
//      leaf's reach are dropped by a ballot first) and counts or writes the pairs.
// Query rows come out in a fixed order (units, then leaves, then particles).  The same pass
// builds the target-major lists: per (tile, target) a ballot of the pair bits gives the
// target's new partners, counted (and later placed) with one atomic.  The order inside a
// target row then follows the tiles' completion; the Monte Carlo, which reads those rows, sums
// them exactly in fixed point and selects partners by gas id, so no result depends on it.
// The count pass keeps every tile's 32 x 32 pair mask (128 bytes per candidate leaf pair); the
// emit pass reads the masks and writes both lists without testing a distance again.  A float32
// emit pass can also form every pair's overlap g_ij and store it beside both lists (PairWeights),
// for pair sets that serve many interaction passes.
#include "pairs.cuh"
#include "physics.cuh"

#define SR_WARPS 4
#define SR_STACK 256

__device__ __forceinline__ float axis_gap(float qa, float qb, float na, float nb) {
  return fmaxf(0.0f, fmaxf(na - qb, qa - nb));
}

// squared distance between two boxes (minimum image when periodic, with the sides of up to two
// boxes: a leaf of batched boxes can straddle two of them)
__device__ __forceinline__ float box_gap2_one(const float qmn[3], const float qmx[3], const float4 &nmn,
                                              const float4 &nmx, int periodic, const BoxSide &bs) {
  float d2 = 0.f;
  const float na[3] = {nmn.x, nmn.y, nmn.z}, nb[3] = {nmx.x, nmx.y, nmx.z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float gap = axis_gap(qmn[k], qmx[k], na[k], nb[k]);
    if (periodic) {
      const float L = bs.Lhi[k];
      gap = fminf(gap, fminf(axis_gap(qmn[k] + L, qmx[k] + L, na[k], nb[k]), axis_gap(qmn[k] - L, qmx[k] - L, na[k], nb[k])));
    }
    d2 += gap * gap;
  }
  return d2;
}

struct LeafSides {
  BoxSide a, b;
  bool two;
};

template <int GEOM>
__device__ __forceinline__ LeafSides leaf_sides(const BoxSplit &bx, const int2 *leaf_box, int leaf) {
  LeafSides ls;
  if (GEOM == GEOM_BOXES) {
    const int2 r = leaf_box[leaf];
    ls.a = box_side<GEOM>(bx, r.x);
    ls.two = r.y != r.x;
    ls.b = ls.two ? box_side<GEOM>(bx, r.y) : ls.a;
  } else {
    ls.a = box_side<GEOM>(bx, 0);
    ls.b = ls.a;
    ls.two = false;
  }
  return ls;
}

template <int GEOM>
__device__ __forceinline__ float box_gap2(const float qmn[3], const float qmx[3], const float4 &nmn, const float4 &nmx,
                                          const LeafSides &ls) {
  float d2 = box_gap2_one(qmn, qmx, nmn, nmx, GEOM != GEOM_OPEN, ls.a);
  if (GEOM == GEOM_BOXES && ls.two) d2 = fminf(d2, box_gap2_one(qmn, qmx, nmn, nmx, 1, ls.b));
  return d2;
}

// Emit of the target-major lists for one tile: lane k owns target k (mycol = the query lanes
// paired with it), claims its positions with one atomic, and every query lane writes its entries.
// With tr.gidx each entry also gets its query-major position: the query lane's row continues at
// out0 (its position before this tile) with its pairs in ascending target order, myrow being the
// lane's targets in this tile.
__device__ __forceinline__ void emit_transposed(const TransposeOut &tr, int64_t base, unsigned lane, unsigned lt,
                                               unsigned m, uint32_t mycol, int64_t qi, int64_t out0 = 0,
                                               uint32_t myrow = 0u) {
  const int64_t tk = base + lane;
  int64_t p0 = 0, p1 = 0;
  if (mycol) {
    p0 = tr.ptr[tk] + atomicAdd(&tr.cursor[tk], (uint32_t)__popc(mycol));
    p1 = tr.ptr[tk + 1];
  }
  for (unsigned mm = m; mm; mm &= mm - 1) {
    const int k = __ffs(mm) - 1;
    const unsigned col = __shfl_sync(DMB_FULL, mycol, k);
    const int64_t s0 = __shfl_sync(DMB_FULL, p0, k), s1 = __shfl_sync(DMB_FULL, p1, k);
    if (col & (1u << lane)) {
      const int64_t pos = s0 + __popc(col & lt);
      if (pos < s1) {
        tr.rows[pos] = (uint32_t)qi;
        if (tr.gidx != nullptr) tr.gidx[pos] = (uint32_t)(out0 + __popc(myrow & ((1u << k) - 1u)));
      }
    }
  }
}

// ---- stage 1: candidate target leaves per query leaf -----------------------------------
template <typename R, bool EMIT, int GEOM>
__global__ void __launch_bounds__(SR_WARPS * 32)
k_leaf_pairs(SpeciesView<R> Q, SpeciesView<R> O, BoxSplit bx, const Frame *__restrict__ frame,
             uint32_t *__restrict__ item_cnt, const int64_t *__restrict__ item_ptr, uint32_t *__restrict__ items,
             uint32_t *status, unsigned long long *__restrict__ stats) {
  __shared__ int stack[SR_WARPS][SR_STACK];
  const int wib = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt = (1u << lane) - 1u;
  const float pad2 = 2.0f * frame->pad;
  const int nleaf = Q.cnt[0];
  unsigned long long st_nodes = 0;
  for (int a = blockIdx.x * SR_WARPS + wib; a < nleaf; a += gridDim.x * SR_WARPS) {
    const float4 qa = Q.bmin[Q.off[0] + a], qb = Q.bmax[Q.off[0] + a];
    uint32_t count = 0;
    const int64_t base = EMIT ? item_ptr[a] : 0;
    const int64_t lim = EMIT ? item_ptr[a + 1] - base : 0;
    if (qa.w >= 0.0f) {
      const float qmn[3] = {qa.x, qa.y, qa.z}, qmx[3] = {qb.x, qb.y, qb.z};
      const LeafSides ls = leaf_sides<GEOM>(bx, Q.leaf_box, a);
      const int top = O.levels - 1;
      if (top == 0) {
        // a single leaf: test it directly
        const float4 nmn = O.bmin[O.off[0]], nmx = O.bmax[O.off[0]];
        const float r = qa.w + nmn.w + pad2;
        if (nmn.w >= 0.0f && box_gap2<GEOM>(qmn, qmx, nmn, nmx, ls) < r * r) {
          if (EMIT && lane == 0 && lim > 0) items[base] = 0u;
          count = 1;
        }
      } else {
        int sp = 0;
        if (lane == 0) stack[wib][0] = (top << 27) | 0;
        sp = 1;
        __syncwarp();
        while (sp > 0) {
          const int e = stack[wib][sp - 1];
          --sp;
          __syncwarp();
          const int l = e >> 27, idx = e & ((1 << 27) - 1);
          ++st_nodes;
          const int c = idx * 32 + (int)lane;
          bool pass = false;
          if (c < O.cnt[l - 1]) {
            const float4 nmn = O.bmin[O.off[l - 1] + c], nmx = O.bmax[O.off[l - 1] + c];
            const float r = qa.w + nmn.w + pad2;
            pass = nmn.w >= 0.0f && box_gap2<GEOM>(qmn, qmx, nmn, nmx, ls) < r * r;
          }
          const unsigned m = __ballot_sync(DMB_FULL, pass);
          const int np = __popc(m);
          if (l - 1 == 0) {
            if (EMIT && pass && (int64_t)(count + __popc(m & lt)) < lim) items[base + count + __popc(m & lt)] = (uint32_t)c;
            count += np;
          } else if (np) {
            if (sp + np > SR_STACK) {
              if (lane == 0) atomicOr(status, DMB_BAD_OVERFLOW);
              break;
            }
            // push in reverse so the lowest child index is popped first
            if (pass) stack[wib][sp + np - 1 - __popc(m & lt)] = ((l - 1) << 27) | c;
            sp += np;
          }
          __syncwarp();
        }
      }
    }
    if (!EMIT && lane == 0) item_cnt[a] = count;
    if (EMIT && lane == 0 && (int64_t)count != item_ptr[a + 1] - item_ptr[a]) atomicOr(status, DMB_BAD_OVERFLOW);
  }
  if (stats != nullptr && lane == 0) atomicAdd(&stats[0], st_nodes);
}

// units per query leaf
__global__ void k_unit_counts(const int64_t *__restrict__ item_ptr, int nleaf, int unit, uint32_t *__restrict__ unit_cnt) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nleaf) return;
  const int64_t n = item_ptr[a + 1] - item_ptr[a];
  unit_cnt[a] = (uint32_t)((n + unit - 1) / unit);
}

__global__ void k_unit_map(const int64_t *__restrict__ item_ptr, const int64_t *__restrict__ unit_ptr, int nleaf,
                           int unit, uint32_t *__restrict__ unit_leaf, int64_t *__restrict__ unit_item0) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nleaf) return;
  const int64_t u0 = unit_ptr[a], u1 = unit_ptr[a + 1];
  for (int64_t u = u0; u < u1; ++u) {
    unit_leaf[u] = (uint32_t)a;
    unit_item0[u] = item_ptr[a] + (u - u0) * unit;
  }
}

// ---- stage 2: tiles of (query leaf) x (target leaf) -------------------------------------
// W: the emit pass also writes the pair weights (float32, with the tile masks)
template <typename R, bool EMIT, int GEOM, bool W>
__global__ void __launch_bounds__(SR_WARPS * 32, (W && GEOM != GEOM_BOXES) ? 8 : 0)
k_tile(SpeciesView<R> Q, SpeciesView<R> O, BoxSplit bx, const Frame *__restrict__ frame,
       const uint32_t *__restrict__ unit_leaf, const int64_t *__restrict__ unit_item0,
       const int64_t *__restrict__ item_ptr, const uint32_t *__restrict__ items, int64_t n_units, int unit,
       uint32_t *__restrict__ unit_cnt, const int64_t *__restrict__ row_ptr, uint32_t *__restrict__ rows,
       TransposeOut tr, uint32_t *__restrict__ tmask, uint32_t *status, unsigned long long *__restrict__ stats,
       const int64_t *__restrict__ n_units_dev, PairWeights pw) {
  typedef typename Vec<R>::v4 v4;
  __shared__ v4 sP[SR_WARPS][DMB_LEAF];
  __shared__ v4 sL[SR_WARPS][DMB_LEAF];
  __shared__ uint16_t sB[SR_WARPS][DMB_LEAF];
  const int wib = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31u;
  const float pad2 = 2.0f * frame->pad;
  const bool boxed = GEOM == GEOM_BOXES;
  const bool tr_on = EMIT ? tr.rows != nullptr : tr.cnt != nullptr;
  const bool want_col = tr_on || (!EMIT && tmask != nullptr);
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long st_tests = 0, st_leaves = 0;
  // n_units is a capacity when the unit count lives on the device (captured steps)
  const int64_t nu = n_units_dev != nullptr ? min(n_units, *n_units_dev) : n_units;
  for (int64_t u = (int64_t)blockIdx.x * SR_WARPS + wib; u < nu; u += (int64_t)gridDim.x * SR_WARPS) {
    const int a = (int)unit_leaf[u];
    const int64_t it0 = unit_item0[u];
    const int64_t it1 = min(it0 + (int64_t)unit, item_ptr[a + 1]);
    const int64_t qi = (int64_t)a * DMB_LEAF + lane;
    const bool valid = qi < Q.n;
    const float4 qa = Q.bmin[Q.off[0] + a], qb = Q.bmax[Q.off[0] + a];
    const float qmn[3] = {qa.x, qa.y, qa.z}, qmx[3] = {qb.x, qb.y, qb.z};
    v4 Pq = Vec<R>::make(0, 0, 0, 0), Lq = Vec<R>::make(0, 0, 0, 0);
    if (valid) { Pq = Q.P[qi]; Lq = Q.L[qi]; }
    // the query's negated hi and lo parts (two-wide distance test of the open geometry)
    const float2 nq_hxy = make_float2(-(float)Pq.x, -(float)Pq.y), nq_lxy = make_float2(-(float)Lq.x, -(float)Lq.y);
    const float nq_hz = -(float)Pq.z, nq_lz = -(float)Lq.z;
    const LeafSides ls = leaf_sides<GEOM>(bx, Q.leaf_box, a);
    const BoxSide side_q = (GEOM == GEOM_BOXES && valid) ? box_side<GEOM>(bx, Q.bid[qi]) : ls.a;
    const uint16_t box_q = (boxed && valid) ? Q.bid[qi] : (uint16_t)0;
    uint32_t cnt = 0;
    int64_t out = 0, out_end = 0;
    if (EMIT && valid) {
      out = row_ptr[qi] + unit_cnt[32 * u + lane];   // unit_cnt holds the exclusive offsets here
      out_end = row_ptr[qi + 1];
    }
    if constexpr (W) {
      // the query leaf's copies, row ends and boxes; per tile every target's pair mask and claimed
      // target-major range, every query lane's targets, the prefix of their counts and the
      // lane's row position
      __shared__ v4 sQP[SR_WARPS][DMB_LEAF];
      __shared__ v4 sQL[SR_WARPS][DMB_LEAF];
      __shared__ int64_t sEnd[SR_WARPS][DMB_LEAF], sOut[SR_WARPS][DMB_LEAF];
      __shared__ uint16_t sQB[SR_WARPS][DMB_LEAF];
      __shared__ uint32_t sCol[SR_WARPS][DMB_LEAF], sRow[SR_WARPS][DMB_LEAF], sOff[SR_WARPS][DMB_LEAF];
      __shared__ int64_t sP0[SR_WARPS][DMB_LEAF], sP1[SR_WARPS][DMB_LEAF];
      // as below, and each pair's weights.  The tile's pairs are spread evenly over the lanes
      // (pair h of the tile, in query-lane then target order, goes to lane h mod 32): the lane
      // finds the pair's query lane q from the prefix of the per-lane pair counts and its target
      // k as the r-th pair of that lane, forms the canonical displacement, distance and overlap
      // g_ij from the staged copies, and writes the query-major entry (row, M_target g_ij) at
      // lane q's position and the target-major entry (query, g_ij) at target k's claimed range.
      // Entries land where the plain emit pass puts them.
      __syncwarp();
      sQP[wib][lane] = Pq;
      sQL[wib][lane] = Lq;
      sEnd[wib][lane] = out_end;
      if (GEOM == GEOM_BOXES) sQB[wib][lane] = box_q;
      const int64_t qbase = (int64_t)a * DMB_LEAF;
      uint32_t col_next = it0 < it1 ? tmask[32 * it0 + lane] : 0u;
      uint32_t leaf_next = it0 < it1 ? items[it0] : 0u;
      v4 Pk_next = Vec<R>::make(0, 0, 0, 0), Lk_next = Vec<R>::make(0, 0, 0, 0);
      if (it0 < it1 && (int64_t)leaf_next * DMB_LEAF + lane < O.n) {
        Pk_next = O.P[(int64_t)leaf_next * DMB_LEAF + lane];
        Lk_next = O.L[(int64_t)leaf_next * DMB_LEAF + lane];
      }
      for (int64_t it = it0; it < it1; ++it) {
        const uint32_t mycol = col_next;
        const int64_t base = (int64_t)leaf_next * DMB_LEAF;
        __syncwarp();
        sP[wib][lane] = Pk_next;
        sL[wib][lane] = Lk_next;
        if (it + 1 < it1) {
          col_next = tmask[32 * (it + 1) + lane];
          leaf_next = items[it + 1];
          const int64_t nb = (int64_t)leaf_next * DMB_LEAF + lane;
          if (nb < O.n) {
            Pk_next = O.P[nb];
            Lk_next = O.L[nb];
          }
        }
        const unsigned m = __ballot_sync(DMB_FULL, mycol != 0u);
        if (!m) continue;
        int64_t p0 = 0, p1 = 0;                          // this lane's claim for target `lane`
        if (tr_on && mycol) {
          p0 = tr.ptr[base + lane] + atomicAdd(&tr.cursor[base + lane], (uint32_t)__popc(mycol));
          p1 = tr.ptr[base + lane + 1];
        }
        // this query lane's targets in the tile (bit k: paired with target k) and their count
        uint32_t myrow = 0u;
        for (unsigned mm = m; mm; mm &= mm - 1) {
          const int k = __ffs(mm) - 1;
          myrow |= ((__shfl_sync(DMB_FULL, mycol, k) >> lane) & 1u) << k;
        }
        const uint32_t cnt = (uint32_t)__popc(myrow);
        uint32_t incl = cnt;                              // inclusive prefix over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t v = __shfl_up_sync(DMB_FULL, incl, o);
          if ((int)lane >= o) incl += v;
        }
        const uint32_t npairs = __shfl_sync(DMB_FULL, incl, 31);
        sCol[wib][lane] = mycol;
        sP0[wib][lane] = p0;
        sP1[wib][lane] = p1;
        sRow[wib][lane] = myrow;
        sOff[wib][lane] = incl - cnt;
        sOut[wib][lane] = out;
        __syncwarp();
        for (uint32_t h = lane; h < npairs; h += 32) {
          int q = 0;                                      // the last lane whose pairs start at or before h
#pragma unroll
          for (int step = 16; step > 0; step >>= 1)
            if (sOff[wib][q + step] <= h) q += step;
          const uint32_t r = h - sOff[wib][q];
          uint32_t mm = sRow[wib][q];
          for (uint32_t i = 0; i < r; ++i) mm &= mm - 1;
          const int k = __ffs(mm) - 1;
          const v4 Pa = sQP[wib][q], La = sQL[wib][q], Pk = sP[wib][k], Lk = sL[wib][k];
          const BoxSide side = GEOM == GEOM_BOXES ? box_side<GEOM>(bx, sQB[wib][q]) : ls.a;
          R dx, dy, dz;
          pair_dx<R>(Pa, La, Pk, Lk, GEOM != GEOM_OPEN, side, dx, dy, dz);
          const float g = overlap_g<float>(pw.gtab, sqrt_pair((float)dist2_rn<R>(dx, dy, dz)), (float)Pa.w, (float)Pk.w);
          const int64_t oq = sOut[wib][q] + r;
          if (oq < sEnd[wib][q]) {
            rows[oq] = (uint32_t)(base + k);
            pw.q[oq] = (float)Lk.w * g;
          }
          if (tr_on) {
            const int64_t pos = sP0[wib][k] + __popc(sCol[wib][k] & ((1u << q) - 1u));
            if (pos < sP1[wib][k]) {
              tr.rows[pos] = (uint32_t)(qbase + q);
              if (pw.t != nullptr) pw.t[pos] = g;
              if (tr.gidx != nullptr) tr.gidx[pos] = (uint32_t)oq;
            }
          }
        }
        out += cnt;
      }
      continue;
    }
    if (EMIT && tmask != nullptr) {
      // the count pass left each tile's pair masks (lane k: the query lanes paired with target
      // k): the emit pass writes the pairs without testing distances again, loading the next
      // tile's mask and leaf while it writes this one's
      uint32_t col_next = it0 < it1 ? tmask[32 * it0 + lane] : 0u;
      uint32_t leaf_next = it0 < it1 ? items[it0] : 0u;
      for (int64_t it = it0; it < it1; ++it) {
        const uint32_t mycol = col_next;
        const int64_t base = (int64_t)leaf_next * DMB_LEAF;
        if (it + 1 < it1) {
          col_next = tmask[32 * (it + 1) + lane];
          leaf_next = items[it + 1];
        }
        const unsigned m = __ballot_sync(DMB_FULL, mycol != 0u);
        const int64_t out0 = out;
        uint32_t myrow = 0u;
        for (unsigned mm = m; mm; mm &= mm - 1) {
          const int k = __ffs(mm) - 1;
          if (__shfl_sync(DMB_FULL, mycol, k) & (1u << lane)) {
            if (out < out_end) rows[out] = (uint32_t)(base + k);
            ++out;
            myrow |= 1u << k;
          }
        }
        if (tr_on && m) emit_transposed(tr, base, lane, lt, m, mycol, qi, out0, myrow);
      }
      continue;
    }
    for (int64_t it = it0; it < it1; ++it) {
      const int64_t base = (int64_t)items[it] * DMB_LEAF;
      const int nk = (int)min((int64_t)DMB_LEAF, O.n - base);
      bool keep = false;
      __syncwarp();
      if ((int)lane < nk) {
        const v4 Pk = O.P[base + lane], Lk = O.L[base + lane];
        sP[wib][lane] = Pk;
        sL[wib][lane] = Lk;
        if (boxed) sB[wib][lane] = O.bid[base + lane];
        // float position (within a few float ulps of the span, covered by the pad)
        const float c[3] = {(float)Pk.x + (float)Lk.x, (float)Pk.y + (float)Lk.y, (float)Pk.z + (float)Lk.z};
        const float4 pmn = make_float4(c[0], c[1], c[2], 0.f), pmx = make_float4(c[0], c[1], c[2], 0.f);
        const float r = qa.w + (float)Pk.w + pad2;
        keep = box_gap2<GEOM>(qmn, qmx, pmn, pmx, ls) < r * r;
      }
      unsigned m = __ballot_sync(DMB_FULL, keep);
      __syncwarp();
      ++st_leaves;
      st_tests += (unsigned long long)__popc(m) * 32ull;
      uint32_t mycol = 0;                                // lane k: the query lanes paired with target k
      const int64_t out0 = out;
      uint32_t myrow = 0u;                               // this lane's targets in this tile
      for (unsigned mm = m; mm; mm &= mm - 1) {          // warp-uniform: m is a ballot
        const int k = __ffs(mm) - 1;
        const v4 Pk = sP[wib][k], Lk = sL[wib][k];
        bool hit;
        if constexpr (GEOM == GEOM_OPEN && sizeof(R) == 4) {
          // the canonical displacement and squared distance of pair_dx and dist2_rn with the x and
          // y components on two-wide float32 instructions (each lane of one rounds as the scalar
          // form does); the target minus the query is the exact negation of pair_dx's query
          // minus target, so the squares, and the predicate, are the same bits
          const float2 hxy = __fadd2_rn(make_float2((float)Pk.x, (float)Pk.y), nq_hxy);
          const float2 lxy = __fadd2_rn(make_float2((float)Lk.x, (float)Lk.y), nq_lxy);
          const float2 dxy = __fadd2_rn(hxy, lxy);
          const float dz = __fadd_rn(__fadd_rn((float)Pk.z, nq_hz), __fadd_rn((float)Lk.z, nq_lz));
          const float2 sq = __fmul2_rn(dxy, dxy);
          const float d2 = __fadd_rn(__fadd_rn(sq.x, sq.y), __fmul_rn(dz, dz));
          hit = valid && pair_test<float>(d2, (float)Pq.w, (float)Pk.w);
        } else {
          hit = valid && !(boxed && sB[wib][k] != box_q);   // pairs never join two boxes
          if (hit) {
            R dx, dy, dz;
            pair_dx<R>(Pq, Lq, Pk, Lk, GEOM != GEOM_OPEN, side_q, dx, dy, dz);
            hit = pair_test<R>(dist2_rn<R>(dx, dy, dz), Pq.w, Pk.w);
          }
        }
        if (hit) {
          if (EMIT) {
            if (out < out_end) rows[out] = (uint32_t)(base + k);
            ++out;
            myrow |= 1u << k;
          }
          ++cnt;
        }
        if (want_col) {
          const unsigned col = __ballot_sync(DMB_FULL, hit);
          if ((int)lane == k) mycol = col;
        }
      }
      if (!EMIT && tmask != nullptr) tmask[32 * it + lane] = mycol;
      if (tr_on && m) {
        // the other direction's lists: lane k owns target k, one atomic per (tile, target),
        // all targets of the tile at once
        if (!EMIT) {
          if (mycol) atomicAdd(&tr.cnt[base + lane], (uint32_t)__popc(mycol));
        } else {
          emit_transposed(tr, base, lane, lt, m, mycol, qi, out0, myrow);
        }
      }
    }
    if (!EMIT) unit_cnt[32 * u + lane] = valid ? cnt : 0u;
  }
  if (stats != nullptr && lane == 0) {
    atomicAdd(&stats[1], st_leaves);
    atomicAdd(&stats[2], st_tests);
  }
}

// per query leaf: exclusive offsets of each unit within every lane's row, and the row counts
__global__ void k_unit_prefix(const int64_t *__restrict__ unit_ptr, int nleaf, int64_t nq,
                              uint32_t *__restrict__ unit_cnt, uint32_t *__restrict__ counts) {
  const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  if (a >= nleaf) return;
  uint32_t run = 0;
  for (int64_t u = unit_ptr[a]; u < unit_ptr[a + 1]; ++u) {
    const uint32_t c = unit_cnt[32 * u + lane];
    unit_cnt[32 * u + lane] = run;
    run += c;
  }
  const int64_t qi = a * DMB_LEAF + lane;
  if (qi < nq) counts[qi] = run;
}

// ---- row segments: long rows cut into pieces of at most `seg` pairs -------------------
__global__ void k_seg_counts(const int64_t *__restrict__ row_ptr, int64_t n, int seg, uint32_t *__restrict__ cnt) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int64_t len = row_ptr[j + 1] - row_ptr[j];
  cnt[j] = (uint32_t)(len > 0 ? (len + seg - 1) / seg : 1);    // empty rows still get one segment
}

__global__ void k_seg_map(const int64_t *__restrict__ row_ptr, const int64_t *__restrict__ seg_ptr, int64_t n, int seg,
                          uint32_t *__restrict__ seg_row, int64_t *__restrict__ seg_begin) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int64_t u = seg_ptr[j]; u < seg_ptr[j + 1]; ++u) {
    seg_row[u] = (uint32_t)j;
    seg_begin[u] = row_ptr[j] + (u - seg_ptr[j]) * seg;
  }
}

cudaError_t launch_seg_counts(const int64_t *row_ptr, int64_t n, int seg, uint32_t *cnt, cudaStream_t s,
                              int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  k_seg_counts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(row_ptr, n, seg, cnt);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_seg_map(const int64_t *row_ptr, const int64_t *seg_ptr, int64_t n, int seg, uint32_t *seg_row,
                           int64_t *seg_begin, cudaStream_t s, int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  k_seg_map<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(row_ptr, seg_ptr, n, seg, seg_row, seg_begin);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

// ---- launchers ---------------------------------------------------------------------------
static int grid_for(int64_t warps) {
  int64_t b = (warps + SR_WARPS - 1) / SR_WARPS;
  if (b > 152 * 128) b = 152 * 128;
  return (int)(b > 0 ? b : 1);
}

template <typename R>
cudaError_t launch_leaf_pairs(SpeciesView<R> Q, SpeciesView<R> O, BoxSplit bx, const Frame *frame, bool emit,
                              uint32_t *item_cnt, const int64_t *item_ptr, uint32_t *items, uint32_t *status,
                              unsigned long long *stats, cudaStream_t s, int64_t *launches) {
  const int g = grid_for(Q.cnt[0]);
#define LP(E, G) k_leaf_pairs<R, E, G><<<g, SR_WARPS * 32, 0, s>>>(Q, O, bx, frame, item_cnt, item_ptr, items, status, stats)
  switch (geom_of(bx) * 2 + (emit ? 1 : 0)) {
    case 0: LP(false, GEOM_OPEN); break;
    case 1: LP(true, GEOM_OPEN); break;
    case 2: LP(false, GEOM_BOX); break;
    case 3: LP(true, GEOM_BOX); break;
    case 4: LP(false, GEOM_BOXES); break;
    default: LP(true, GEOM_BOXES); break;
  }
#undef LP
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_unit_counts(const int64_t *item_ptr, int nleaf, int unit, uint32_t *unit_cnt, cudaStream_t s,
                               int64_t *launches) {
  k_unit_counts<<<(nleaf + 255) / 256, 256, 0, s>>>(item_ptr, nleaf, unit, unit_cnt);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_unit_map(const int64_t *item_ptr, const int64_t *unit_ptr, int nleaf, int unit, uint32_t *unit_leaf,
                            int64_t *unit_item0, cudaStream_t s, int64_t *launches) {
  k_unit_map<<<(nleaf + 255) / 256, 256, 0, s>>>(item_ptr, unit_ptr, nleaf, unit, unit_leaf, unit_item0);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_tile(SpeciesView<R> Q, SpeciesView<R> O, BoxSplit bx, const Frame *frame, bool emit,
                        const uint32_t *unit_leaf, const int64_t *unit_item0, const int64_t *item_ptr,
                        const uint32_t *items, int64_t n_units, int unit, uint32_t *unit_cnt, const int64_t *row_ptr,
                        uint32_t *rows, TransposeOut tr, uint32_t *tmask, uint32_t *status, unsigned long long *stats,
                        cudaStream_t s, int64_t *launches, const int64_t *n_units_dev, PairWeights pw) {
  if (n_units <= 0) return cudaSuccess;
  const int g = grid_for(n_units);
#define TLW(G, W_)                                                                                                \
  k_tile<R, true, G, W_><<<g, SR_WARPS * 32, 0, s>>>(Q, O, bx, frame, unit_leaf, unit_item0, item_ptr, items, n_units, \
                                                     unit, unit_cnt, row_ptr, rows, tr, tmask, status, stats,         \
                                                     n_units_dev, pw)
  if constexpr (sizeof(R) == 4) {
    if (emit && tmask != nullptr && pw.q != nullptr) {
      switch (geom_of(bx)) {
        case GEOM_OPEN: TLW(GEOM_OPEN, true); break;
        case GEOM_BOX: TLW(GEOM_BOX, true); break;
        default: TLW(GEOM_BOXES, true); break;
      }
      if (launches) *launches += 1;
      return cudaGetLastError();
    }
  }
#undef TLW
#define TL(E, G)                                                                                                \
  k_tile<R, E, G, false><<<g, SR_WARPS * 32, 0, s>>>(Q, O, bx, frame, unit_leaf, unit_item0, item_ptr, items,     \
                                                     n_units, unit, unit_cnt, row_ptr, rows, tr, tmask, status,    \
                                                     stats, n_units_dev, PairWeights())
  switch (geom_of(bx) * 2 + (emit ? 1 : 0)) {
    case 0: TL(false, GEOM_OPEN); break;
    case 1: TL(true, GEOM_OPEN); break;
    case 2: TL(false, GEOM_BOX); break;
    case 3: TL(true, GEOM_BOX); break;
    case 4: TL(false, GEOM_BOXES); break;
    default: TL(true, GEOM_BOXES); break;
  }
#undef TL
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_unit_prefix(const int64_t *unit_ptr, int nleaf, int64_t nq, uint32_t *unit_cnt, uint32_t *counts,
                               cudaStream_t s, int64_t *launches) {
  const int64_t t = (int64_t)nleaf * 32;
  k_unit_prefix<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(unit_ptr, nleaf, nq, unit_cnt, counts);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

#define INST(R)                                                                                                     \
  template cudaError_t launch_leaf_pairs<R>(SpeciesView<R>, SpeciesView<R>, BoxSplit, const Frame *, bool,          \
                                            uint32_t *, const int64_t *, uint32_t *, uint32_t *,                    \
                                            unsigned long long *, cudaStream_t, int64_t *);                          \
  template cudaError_t launch_tile<R>(SpeciesView<R>, SpeciesView<R>, BoxSplit, const Frame *, bool,                \
                                      const uint32_t *, const int64_t *, const int64_t *, const uint32_t *, int64_t, \
                                      int, uint32_t *, const int64_t *, uint32_t *, TransposeOut, uint32_t *,         \
                                      uint32_t *,                                                                    \
                                      unsigned long long *,                                                          \
                                      cudaStream_t, int64_t *, const int64_t *, PairWeights);
INST(float)
INST(double)

// ---- capacity checks of a captured step ---------------------------------------------------
// One block: the device totals against the capacities the buffers were sized for.  On overflow it
// records the totals for the host, sets the gate and the status bit and clears the given offset
// arrays, so every later kernel of the step sees empty rows and touches nothing out of bounds.
__global__ void __launch_bounds__(1024) k_cap_check(CapCheck c) {
  __shared__ int over;
  if (threadIdx.x == 0) {
    int o = 0;
    for (int k = 0; k < 4; ++k)
      if (c.total[k] != nullptr) {
        const int64_t t = *c.total[k];
        c.need[c.slot[k]] = t;
        if (t > c.cap[k]) o = 1;
      }
    over = o;
    if (o) {
      *c.gate = 1u;
      atomicOr(c.status, DMB_BAD_OVERFLOW);
    }
  }
  __syncthreads();
  if (!over) return;
  for (int k = 0; k < 4; ++k)
    if (c.zero[k] != nullptr)
      for (int64_t i = threadIdx.x; i < c.zero_n[k]; i += blockDim.x) c.zero[k][i] = 0;
}

cudaError_t launch_cap_check(const CapCheck &c, cudaStream_t s, int64_t *launches) {
  k_cap_check<<<1, 1024, 0, s>>>(c);
  if (launches) *launches += 1;
  return cudaGetLastError();
}
