// DM Monte Carlo (Eqs. dm-update-vels, dm-update-prob, scatter_chi, prob_criterion): the
// categorical draw, the per-pair Bernoulli variant and their launcher; the overlap table and
// the debug evaluators.
#include "interact.cuh"

// W: g_ij comes from the pair weights a.g (float32 pair sets searched with weights) instead of
// the positions and the overlap table.
template <typename R, int GEOM, bool W>
__global__ void __launch_bounds__(MC_WARPS * 32, sizeof(R) == 4 ? 4 : 1)
k_mc(SpeciesView<R> D, SpeciesView<R> G, BoxSplit bx, const int64_t *__restrict__ row_ptr,
     const uint32_t *__restrict__ rows, const float4 *__restrict__ gtab, RunConst rc, McArgs a,
     R *__restrict__ pcache, McRec *__restrict__ rec) {
  typedef typename Vec<R>::v4 v4;
  const unsigned lane = threadIdx.x & 31u;
  const int wib = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * MC_WARPS;
  const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
  const R inv_v0 = (R)(1.0 / rc.v0);
  const R inv_vc2 = (R)rc.inv_vc2;
  const R beta = (R)a.beta;                          // dsigma/dOmega ~ 1 + beta cos theta
  const unsigned long long step = a.step_dev ? *a.step_dev : a.step;
  const int64_t nrows = a.list ? a.n_list : D.n;
  const R dt0 = (R)a.dt;
  // Warp w takes rows w, w + W, w + 2W, ... (W warps in the grid), 32 of them per visit: each
  // lane writes the record of its row if the row is empty (no gas partner: nothing can happen;
  // most DM particles outside the gas disk have none), and the whole warp then works through
  // the other rows one by one.
  const int64_t warp_id = (int64_t)blockIdx.x * MC_WARPS + wib;
  for (int64_t row0 = warp_id; row0 < nrows; row0 += 32 * nwarps) {
    const int64_t kl = row0 + (int64_t)lane * nwarps;
    int64_t il = 0;
    bool busy = false;
    if (kl < nrows) {
      il = a.list ? (int64_t)a.list[kl] : kl;
      busy = row_ptr[il + 1] > row_ptr[il];
      if (!busy) {
        McRec r;
        r.c_lo = 0ull; r.c_hi = 0ull; r.rmax = 0.0f; r.flags = 0u; r.partner = 0xffffffffu;
        r.dv[0] = r.dv[1] = r.dv[2] = 0.0;
        rec[il] = r;
      }
    }
    for (unsigned busy_rows = __ballot_sync(DMB_FULL, busy); busy_rows; busy_rows &= busy_rows - 1) {
      const int64_t i = __shfl_sync(DMB_FULL, il, __ffs(busy_rows) - 1);
      // dt_i = 2^bin dt: a power-of-two scaling, exact in the pair precision
      const R dt = a.bin ? dt0 * (R)(1ull << a.bin[D.perm[i]]) : dt0;
      const int64_t rs = row_ptr[i], re = row_ptr[i + 1];
      const v4 Pi = D.P[i], Li = D.L[i], Vi = D.V[i];
      const uint32_t id_i = D.id[i];
      const BoxSide side = box_side<GEOM>(bx, GEOM == GEOM_BOXES ? (int)D.bid[i] : 0);
      U128 sum = {0ull, 0ull};
      float rmax = 0.0f;
      // each pass loads the next pass's partner index ahead of its own gathers
      uint32_t j_next = rs + lane < re ? rows[rs + lane] : 0u;
      for (int64_t p = rs + lane; p < re; p += 32) {
        const uint32_t j = j_next;
        if (p + 32 < re) j_next = rows[p + 32];
        const v4 Vj = G.V[j], Kj = G.K[j];
        R rx, ry, rz, vr;
        R P;
        if constexpr (W) {   // g_ij from the search's emit pass
          P = pair_probability_g<R>((R)a.g[p], Vi, id_i, Vj, Kj, G.id[j], rc.n, inv_v0, inv_vc2, dt, step, k0, k1,
                                    rx, ry, rz, vr);
        } else {
          const v4 Pj = G.P[j], Lj = G.L[j];
          P = pair_probability<R>(Pi, Li, Vi, id_i, Pj, Lj, Vj, Kj, G.id[j], GEOM != GEOM_OPEN, side, gtab, rc.n,
                                  inv_v0, inv_vc2, dt, step, k0, k1, rx, ry, rz, vr);
        }
        pcache[p] = P;
        sum = u128_add(sum, to_fixed(P));
        const R e = Kj.w;                                   // mu_j / (m_chi + mu_j)
        // Eq. prob_criterion: 1 / min(0.1, 1e-4 / e^2) = max(10, 1e4 e^2), no division
        const R inv_cap = (R)1e4 * e * e > (R)10 ? (R)1e4 * e * e : (R)10;
        rmax = fmaxf(rmax, (float)(P * inv_cap));
      }
      const U128 C = warp_sum_u128(sum);
      rmax = warp_max(rmax);
      // selection uniform r_i = (k + 1/2) 2^-52, k the top 52 bits of (w0, w3): as a 64-bit fraction
      const uint4 wd = philox4x32_10(dm_counter(id_i, step), k0, k1);
      const unsigned long long k52 = ((unsigned long long)wd.x << 20) | (unsigned long long)(wd.w >> 12);
      const unsigned long long R64 = (k52 << 12) | (1ull << 11);
      const bool clamped = C.hi >= 1ull;                    // sum_j P_ij > 1: renormalise
      U128 T;
      if (clamped) T = u128_scale(R64, C); else { T.hi = 0ull; T.lo = R64; }
      const bool scat = u128_lt(T, C);
      bool band = near_rel(T, C, C);
      R dv0 = 0, dv1 = 0, dv2 = 0;
      uint32_t partner_id = 0xffffffffu;
      if (scat) {
        // binary search over the gas-id bits for the first partner (ascending id) whose
        // running sum exceeds T
        uint32_t prefix = 0;
        U128 base = {0ull, 0ull};
        for (int b = a.id_bits - 1; b >= 0; --b) {
          const uint32_t mid = prefix | (1u << b);
          U128 S = {0ull, 0ull};
          for (int64_t p = rs + lane; p < re; p += 32) {
            const uint32_t idj = G.id[rows[p]];
            if (idj >= prefix && idj < mid) S = u128_add(S, to_fixed(pcache[p]));
          }
          S = warp_sum_u128(S);
          const U128 top = u128_add(base, S);
          if (!u128_lt(T, top)) { base = top; prefix = mid; }
        }
        int64_t pstar = -1;
        for (int64_t p0 = rs; p0 < re; p0 += 32) {
          const int64_t p = p0 + lane;
          const bool hit = p < re && G.id[rows[p]] == prefix;
          const unsigned m = __ballot_sync(DMB_FULL, hit);
          if (m) { pstar = p0 + __ffs(m) - 1; break; }
        }
        if (pstar >= 0) {
          const uint32_t j = rows[pstar];
          const v4 Vj = G.V[j], Kj = G.K[j];
          R rx, ry, rz, vr;
          if constexpr (W) {
            (void)pair_probability_g<R>((R)a.g[pstar], Vi, id_i, Vj, Kj, G.id[j], rc.n, inv_v0, inv_vc2, dt, step,
                                        k0, k1, rx, ry, rz, vr);
          } else {
            const v4 Pj = G.P[j], Lj = G.L[j];
            (void)pair_probability<R>(Pi, Li, Vi, id_i, Pj, Lj, Vj, Kj, G.id[j], GEOM != GEOM_OPEN, side, gtab, rc.n,
                                      inv_v0, inv_vc2, dt, step, k0, k1, rx, ry, rz, vr);
          }
          const U128 hi = u128_add(base, to_fixed(pcache[pstar]));
          band = band || near_rel(T, base, hi) || near_rel(T, hi, hi);
          // isotropic new direction: cos(theta') = 2u - 1, phi' = 2 pi u'
          const R ct = (R)2 * uniform23<R>(wd.y) - (R)1;
          const R st = sqrt_t(fmax((R)0, (R)1 - ct * ct));
          R sp, cp;
          if (sizeof(R) == 4) { float s_, c_; sincospif(2.0f * (float)uniform23<float>(wd.z), &s_, &c_); sp = (R)s_; cp = (R)c_; }
          else { double s_, c_; sincospi(2.0 * uniform23<double>(wd.z), &s_, &c_); sp = (R)s_; cp = (R)c_; }
          const R f = Kj.w * vr;                             // mu_j/(m_chi + mu_j) v_rel
          const R inv = (R)1 / vr;
          if (beta == (R)0) {
            dv0 = f * (st * cp - rx * inv);
            dv1 = f * (st * sp - ry * inv);
            dv2 = f * (ct - rz * inv);
          } else {                                           // anisotropic: about the incoming direction
            const R ux = rx * inv, uy = ry * inv, uz = rz * inv;
            R nx, ny, nz;
            aniso_direction<R>(ct, sp, cp, beta, ux, uy, uz, nx, ny, nz);
            dv0 = f * (nx - ux);
            dv1 = f * (ny - uy);
            dv2 = f * (nz - uz);
          }
          partner_id = prefix;
        }
      }
      if (lane == 0) {
        McRec r;
        r.c_lo = C.lo;
        r.c_hi = C.hi;
        r.rmax = rmax;
        r.flags = (partner_id != 0xffffffffu ? 1u : 0u) | (clamped ? 2u : 0u) | (band ? 4u : 0u);
        r.partner = partner_id;
        r.dv[0] = (double)dv0;
        r.dv[1] = (double)dv1;
        r.dv[2] = (double)dv2;
        rec[i] = r;
      }
    }
  }
}

// ---- Monte Carlo, the per-pair Bernoulli variant ------------------------------------------
// Sec. 2.5 as GIZMO applies it: the pairs of DM particle i, in ascending gas id, each scatter
// when r_ij < P_ij, with P_ij from the particle's velocity at that point, so a scatter changes
// the probabilities of the pairs after it.  r_ij and the new direction come from the pair's
// Bernoulli stream (counter word 3 = step_hi | 2^30: words 0, 3 give r_ij with 52 bits, words
// 1, 2 the isotropic direction); v^B_ij is the pair's usual sample.  On the device: the first
// hit is the smallest gas id with r < P at the start velocity; after its kick the pairs of
// larger id are tested again with the new velocity, and so on (at most 64 scatters a step).
// The record is that of k_mc: C and rmax from the start velocity, partner = the first partner,
// dv = the sum of the kicks; flag 4 when some r_ij lay within 2^-20 P_ij of P_ij.
__device__ __forceinline__ uint4 bern_counter(uint32_t id_dm, uint32_t id_gas, unsigned long long step) {
  return make_uint4(id_dm, id_gas, (uint32_t)step, ((uint32_t)(step >> 32) & 0x3fffffffu) | 0x40000000u);
}
__device__ __forceinline__ double uniform52(uint32_t w_hi, uint32_t w_lo) {
  const unsigned long long k = ((unsigned long long)w_hi << 20) | (unsigned long long)(w_lo >> 12);
  return ((double)k + 0.5) * 0x1p-52;
}
__device__ __forceinline__ uint32_t warp_min_u32(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(DMB_FULL, v, o));
  return v;
}

template <typename R, int GEOM>
__global__ void __launch_bounds__(MC_WARPS * 32, sizeof(R) == 4 ? 2 : 1)
k_mc_bernoulli(SpeciesView<R> D, SpeciesView<R> G, BoxSplit bx, const int64_t *__restrict__ row_ptr,
               const uint32_t *__restrict__ rows, const float4 *__restrict__ gtab, RunConst rc, McArgs a,
               McRec *__restrict__ rec) {
  typedef typename Vec<R>::v4 v4;
  const unsigned lane = threadIdx.x & 31u;
  const int wib = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * MC_WARPS;
  const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
  const R inv_v0 = (R)(1.0 / rc.v0);
  const R inv_vc2 = (R)rc.inv_vc2;
  const R beta = (R)a.beta;                          // dsigma/dOmega ~ 1 + beta cos theta
  const unsigned long long step = a.step_dev ? *a.step_dev : a.step;
  const int64_t nrows = a.list ? a.n_list : D.n;
  const R dt0 = (R)a.dt;
  const uint32_t NONE = 0xffffffffu;
  const int64_t warp_id = (int64_t)blockIdx.x * MC_WARPS + wib;
  for (int64_t row0 = warp_id; row0 < nrows; row0 += 32 * nwarps) {
    const int64_t kl = row0 + (int64_t)lane * nwarps;
    int64_t il = 0;
    bool busy = false;
    if (kl < nrows) {
      il = a.list ? (int64_t)a.list[kl] : kl;
      busy = row_ptr[il + 1] > row_ptr[il];
      if (!busy) {
        McRec r;
        r.c_lo = 0ull; r.c_hi = 0ull; r.rmax = 0.0f; r.flags = 0u; r.partner = NONE;
        r.dv[0] = r.dv[1] = r.dv[2] = 0.0;
        rec[il] = r;
      }
    }
    for (unsigned busy_rows = __ballot_sync(DMB_FULL, busy); busy_rows; busy_rows &= busy_rows - 1) {
      const int64_t i = __shfl_sync(DMB_FULL, il, __ffs(busy_rows) - 1);
      const R dt = a.bin ? dt0 * (R)(1ull << a.bin[D.perm[i]]) : dt0;
      const int64_t rs = row_ptr[i], re = row_ptr[i + 1];
      const v4 Pi = D.P[i], Li = D.L[i];
      v4 Vc = D.V[i];                                   // the particle's velocity as it scatters
      const uint32_t id_i = D.id[i];
      const BoxSide side = box_side<GEOM>(bx, GEOM == GEOM_BOXES ? (int)D.bid[i] : 0);
      U128 sum = {0ull, 0ull};
      float rmax = 0.0f;
      bool band = false;
      uint32_t hit = NONE;
      for (int64_t p = rs + lane; p < re; p += 32) {
        const uint32_t j = rows[p];
        const v4 Pj = G.P[j], Lj = G.L[j], Vj = G.V[j], Kj = G.K[j];
        const uint32_t idj = G.id[j];
        R rx, ry, rz, vr;
        const R P = pair_probability<R>(Pi, Li, Vc, id_i, Pj, Lj, Vj, Kj, idj, GEOM != GEOM_OPEN, side, gtab, rc.n,
                                        inv_v0, inv_vc2, dt, step, k0, k1, rx, ry, rz, vr);
        sum = u128_add(sum, to_fixed(P));
        const R e = Kj.w;
        // Eq. prob_criterion: 1 / min(0.1, 1e-4 / e^2) = max(10, 1e4 e^2), no division
        const R inv_cap = (R)1e4 * e * e > (R)10 ? (R)1e4 * e * e : (R)10;
        rmax = fmaxf(rmax, (float)(P * inv_cap));
        const uint4 wb = philox4x32_10(bern_counter(id_i, idj, step), k0, k1);
        const double r = uniform52(wb.x, wb.w), Pd = (double)P;
        band = band || fabs(r - Pd) <= Pd * 0x1p-20;
        if (r < Pd && idj < hit) hit = idj;
      }
      const U128 C = warp_sum_u128(sum);
      rmax = warp_max(rmax);
      hit = warp_min_u32(hit);
      const uint32_t first = hit;
      R dv0 = 0, dv1 = 0, dv2 = 0;
      for (int nscat = 0; hit != NONE && nscat < 64; ++nscat) {
        // the pair of gas id `hit` (every lane evaluates it, so all hold the kick)
        int64_t pstar = -1;
        for (int64_t p0 = rs; p0 < re && pstar < 0; p0 += 32) {
          const int64_t p = p0 + lane;
          const unsigned m = __ballot_sync(DMB_FULL, p < re && G.id[rows[p]] == hit);
          if (m) pstar = p0 + __ffs(m) - 1;
        }
        if (pstar < 0) break;
        {
          const uint32_t j = rows[pstar];
          const v4 Pj = G.P[j], Lj = G.L[j], Vj = G.V[j], Kj = G.K[j];
          R rx, ry, rz, vr;
          (void)pair_probability<R>(Pi, Li, Vc, id_i, Pj, Lj, Vj, Kj, hit, GEOM != GEOM_OPEN, side, gtab, rc.n, inv_v0,
                                    inv_vc2, dt, step, k0, k1, rx, ry, rz, vr);
          const uint4 wb = philox4x32_10(bern_counter(id_i, hit, step), k0, k1);
          const R ct = (R)2 * uniform23<R>(wb.y) - (R)1;
          const R st = sqrt_t(fmax((R)0, (R)1 - ct * ct));
          R sp, cp;
          if (sizeof(R) == 4) { float s_, c_; sincospif(2.0f * (float)uniform23<float>(wb.z), &s_, &c_); sp = (R)s_; cp = (R)c_; }
          else { double s_, c_; sincospi(2.0 * uniform23<double>(wb.z), &s_, &c_); sp = (R)s_; cp = (R)c_; }
          const R f = Kj.w * vr;                             // mu_j/(m_chi + mu_j) v_rel
          const R inv = (R)1 / vr;
          R d0, d1, d2;
          if (beta == (R)0) {
            d0 = f * (st * cp - rx * inv);
            d1 = f * (st * sp - ry * inv);
            d2 = f * (ct - rz * inv);
          } else {                                           // anisotropic: about the incoming direction
            const R ux = rx * inv, uy = ry * inv, uz = rz * inv;
            R nx, ny, nz;
            aniso_direction<R>(ct, sp, cp, beta, ux, uy, uz, nx, ny, nz);
            d0 = f * (nx - ux);
            d1 = f * (ny - uy);
            d2 = f * (nz - uz);
          }
          Vc.x += d0; Vc.y += d1; Vc.z += d2;
          dv0 += d0; dv1 += d1; dv2 += d2;
        }
        // the next hit among the pairs of larger gas id, with the new velocity
        uint32_t next = NONE;
        for (int64_t p = rs + lane; p < re; p += 32) {
          const uint32_t j = rows[p];
          const uint32_t idj = G.id[j];
          if (idj <= hit) continue;
          const v4 Pj = G.P[j], Lj = G.L[j], Vj = G.V[j], Kj = G.K[j];
          R rx, ry, rz, vr;
          const R P = pair_probability<R>(Pi, Li, Vc, id_i, Pj, Lj, Vj, Kj, idj, GEOM != GEOM_OPEN, side, gtab, rc.n,
                                          inv_v0, inv_vc2, dt, step, k0, k1, rx, ry, rz, vr);
          const uint4 wb = philox4x32_10(bern_counter(id_i, idj, step), k0, k1);
          const double r = uniform52(wb.x, wb.w), Pd = (double)P;
          band = band || fabs(r - Pd) <= Pd * 0x1p-20;
          if (r < Pd && idj < next) next = idj;
        }
        hit = warp_min_u32(next);
      }
      band = __any_sync(DMB_FULL, band);
      if (lane == 0) {
        McRec r;
        r.c_lo = C.lo;
        r.c_hi = C.hi;
        r.rmax = rmax;
        r.flags = (first != NONE ? 1u : 0u) | (band ? 4u : 0u);
        r.partner = first;
        r.dv[0] = (double)dv0;
        r.dv[1] = (double)dv1;
        r.dv[2] = (double)dv2;
        rec[i] = r;
      }
    }
  }
}

template <typename R>
cudaError_t launch_mc(SpeciesView<R> D, SpeciesView<R> G, BoxSplit bx, const int64_t *row_ptr, const uint32_t *rows,
                      const float4 *gtab, RunConst rc, McArgs a, R *pcache, McRec *rec, int finish_blocks,
                      int blocks_per_sm, cudaStream_t s, int64_t *launches) {
  const int64_t nrows = a.list ? a.n_list : D.n;
  if (nrows <= 0) return cudaSuccess;
  int64_t blocks = (nrows + MC_WARPS - 1) / MC_WARPS;
  if (blocks > 152 * (int64_t)blocks_per_sm) blocks = 152 * (int64_t)blocks_per_sm;
  if (a.variant == 1) {
    switch (geom_of(bx)) {
      case GEOM_OPEN: k_mc_bernoulli<R, GEOM_OPEN><<<(unsigned)blocks, MC_WARPS * 32, 0, s>>>(D, G, bx, row_ptr, rows, gtab, rc, a, rec); break;
      case GEOM_BOX: k_mc_bernoulli<R, GEOM_BOX><<<(unsigned)blocks, MC_WARPS * 32, 0, s>>>(D, G, bx, row_ptr, rows, gtab, rc, a, rec); break;
      default: k_mc_bernoulli<R, GEOM_BOXES><<<(unsigned)blocks, MC_WARPS * 32, 0, s>>>(D, G, bx, row_ptr, rows, gtab, rc, a, rec); break;
    }
  } else {
#define MCL(G_, W_) k_mc<R, G_, W_><<<(unsigned)blocks, MC_WARPS * 32, 0, s>>>(D, G, bx, row_ptr, rows, gtab, rc, a, pcache, rec)
    bool stored = false;
    if constexpr (sizeof(R) == 4) {
      stored = a.g != nullptr;
      if (stored) {
        switch (geom_of(bx)) {
          case GEOM_OPEN: MCL(GEOM_OPEN, true); break;
          case GEOM_BOX: MCL(GEOM_BOX, true); break;
          default: MCL(GEOM_BOXES, true); break;
        }
      }
    }
    if (!stored) {
      switch (geom_of(bx)) {
        case GEOM_OPEN: MCL(GEOM_OPEN, false); break;
        case GEOM_BOX: MCL(GEOM_BOX, false); break;
        default: MCL(GEOM_BOXES, false); break;
      }
    }
#undef MCL
  }
  // the particle mass sits in L.w of the sorted copies
  const R *Lbase = reinterpret_cast<const R *>(D.L);
  k_mc_finish<<<finish_blocks, 256, 0, s>>>(D.n, D.perm, rec, sizeof(R) == 4 ? (const float *)(Lbase + 3) : nullptr,
                                            sizeof(R) == 8 ? (const double *)(Lbase + 3) : nullptr, 4, a);
  if (launches) *launches += 2;
  return cudaGetLastError();
}
template cudaError_t launch_mc<float>(SpeciesView<float>, SpeciesView<float>, BoxSplit, const int64_t *,
                                      const uint32_t *, const float4 *, RunConst, McArgs, float *, McRec *, int,
                                      int, cudaStream_t, int64_t *);
template cudaError_t launch_mc<double>(SpeciesView<double>, SpeciesView<double>, BoxSplit, const int64_t *,
                                       const uint32_t *, const float4 *, RunConst, McArgs, double *, McRec *, int,
                                       int, cudaStream_t, int64_t *);

// ---- overlap table and debug evaluators ------------------------------------------------
__global__ void k_gtable(float4 *__restrict__ T) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)DMB_GT_NQ * DMB_GT_CELLS) return;
  const int j = (int)(t / DMB_GT_CELLS), i = (int)(t % DMB_GT_CELLS);
  const double q = (double)j / (double)(DMB_GT_NQ - 1);
  const double dd = 2.0 / (double)(DMB_GT_ND - 1);
  float v[4];
  for (int k = 0; k < 4; ++k) {
    const int node = i - 1 + k;
    const double delta = fabs((double)node * dd);   // node -1 mirrors node 1 (g is even in d)
    v[k] = (float)overlap_G_exact(delta, q);
  }
  T[t] = make_float4(v[0], v[1], v[2], v[3]);
}

cudaError_t launch_gtable(float4 *T, cudaStream_t s, int64_t *launches) {
  const int64_t n = (int64_t)DMB_GT_NQ * DMB_GT_CELLS;
  k_gtable<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(T);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

__global__ void k_debug_overlap(const float4 *T, int fp64, int64_t k, const double *in, double *out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k) return;
  const double d = in[3 * t], hi = in[3 * t + 1], hj = in[3 * t + 2];
  if (fp64) out[t] = overlap_g<double>(T, d, hi, hj);
  else out[t] = (double)overlap_g<float>(T, (float)d, (float)hi, (float)hj);
}
cudaError_t launch_debug_overlap(const float4 *T, int fp64, int64_t k, const double *in, double *out, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_debug_overlap<<<(unsigned)((k + 127) / 128), 128, 0, s>>>(T, fp64, k, in, out);
  return cudaGetLastError();
}

__global__ void k_debug_rates(int fp64, int n, int mode, double alpha, int64_t k, const double *in, double *out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k) return;
  if (fp64) {
    double a, b;
    if (mode == DMB_RATE_QUAD) rates_quad<double>(in[t], n, alpha, a, b);
    else rates_FAB<double>(in[t], n, a, b);
    out[2 * t] = a;
    out[2 * t + 1] = b;
  } else {
    float a, b;
    if (mode == DMB_RATE_QUAD) rates_quad<float>((float)in[t], n, (float)alpha, a, b);
    else rates_FAB<float>((float)in[t], n, a, b);
    out[2 * t] = a;
    out[2 * t + 1] = b;
  }
}
cudaError_t launch_debug_rates(int fp64, int n, int mode, double alpha, int64_t k, const double *in, double *out,
                               cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_debug_rates<<<(unsigned)((k + 127) / 128), 128, 0, s>>>(fp64, n, mode, alpha, k, in, out);
  return cudaGetLastError();
}

__global__ void k_debug_rates_screened(int fp64, double alpha0, int64_t k, const double *in, double *out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k) return;
  const double x = in[2 * t], q = in[2 * t + 1];
  if (fp64) {
    double a, b;
    rates_quad<double>(x, 0, alpha0, a, b, q);
    out[2 * t] = a;
    out[2 * t + 1] = b;
  } else {
    float a, b;
    rates_quad<float>((float)x, 0, (float)alpha0, a, b, (float)q);
    out[2 * t] = a;
    out[2 * t + 1] = b;
  }
}
cudaError_t launch_debug_rates_screened(int fp64, double alpha0, int64_t k, const double *in, double *out,
                                        cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_debug_rates_screened<<<(unsigned)((k + 127) / 128), 128, 0, s>>>(fp64, alpha0, k, in, out);
  return cudaGetLastError();
}

__global__ void k_debug_philox(int64_t k, const uint32_t *ctr, uint32_t *out, unsigned long long seed) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k) return;
  const uint4 c = make_uint4(ctr[4 * t], ctr[4 * t + 1], ctr[4 * t + 2], ctr[4 * t + 3]);
  const uint4 w = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  out[4 * t] = w.x;
  out[4 * t + 1] = w.y;
  out[4 * t + 2] = w.z;
  out[4 * t + 3] = w.w;
}
cudaError_t launch_debug_philox(int64_t k, const uint32_t *ctr, uint32_t *out, unsigned long long seed,
                                cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_debug_philox<<<(unsigned)((k + 127) / 128), 128, 0, s>>>(k, ctr, out, seed);
  return cudaGetLastError();
}
