// The fused pair pass of a float32 step (mean field and Monte Carlo probabilities in one sweep)
// and the Monte Carlo selection that reads its probabilities.
#include "interact.cuh"

// ---- the fused pair pass of a float32 step: mean field and Monte Carlo probabilities -------
// One sweep over the gas-major pairs computes each pair's overlap g once and uses it twice: for
// the gas row's mean-field sums (as k_meanfield) and for P_ij of Eq. dm-update-prob (as k_mc,
// the same arithmetic through pair_probability_g), written to pg[p] at the pair's gas-major
// position.  The gas particle's copies and id are the row's, loaded once per segment.  The
// per-DM sums, the criterion ratio and the selection follow in k_mc_select, which reads the
// probabilities back through the DM-major rows' gas-major positions (gidx) and evaluates only the
// chosen partner's kick again.  One categorical draw, every DM particle with the step's dt.
template <int RM, int GEOM>
__global__ void __launch_bounds__(MF_WARPS * 32)
k_pairs_fused(SpeciesView<float> G, SpeciesView<float> D, BoxSplit bx, const int64_t *__restrict__ row_ptr,
              const uint32_t *__restrict__ rows, SegView sv, const float4 *__restrict__ gtab, RunConst rc,
              float *__restrict__ part, MlpRun mr, McArgs a, float *__restrict__ pg) {
  const unsigned lane = threadIdx.x & 31u;
  const int64_t nwarps = (int64_t)gridDim.x * MF_WARPS;
  const float inv_v0 = (float)(1.0 / rc.v0);
  const float inv_vc2 = (float)rc.inv_vc2;
  const float alpha = (float)rc.alpha;
  const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
  const unsigned long long step = a.step_dev ? *a.step_dev : a.step;
  const float dt = (float)a.dt;
  const int64_t n_seg = sv.n_seg >= 0 ? sv.n_seg : sv.seg_ptr[G.n];
  for (int64_t u = (int64_t)blockIdx.x * MF_WARPS + (threadIdx.x >> 5); u < n_seg; u += nwarps) {
    const int64_t j = sv.seg_row[u];
    const int64_t rs = sv.seg_begin[u], re = min(rs + (int64_t)sv.seg_len, row_ptr[j + 1]);
    float sx = 0, sy = 0, sz = 0, sw2 = 0, sb = 0, svw = 0;
    if (re > rs) {
      const float4 Pj = G.P[j], Lj = G.L[j], Vj = G.V[j], Kj = G.K[j];
      const uint32_t id_j = G.id[j];
      const BoxSide side = box_side<GEOM>(bx, GEOM == GEOM_BOXES ? (int)G.bid[j] : 0);
      const float sig = Vj.w;
      const bool hot = sig > 0.0f;
      const float inv2s2 = hot ? 0.5f / (sig * sig) : 0.0f;
      const float qv = sig * sig * inv_vc2;
      uint32_t i_next = rows[rs + lane < re ? rs + lane : rs];
      for (int64_t p0 = rs; p0 < re; p0 += 32) {
        const int64_t p = p0 + lane;
        const bool valid = p < re;
        const uint32_t i = i_next;
        if (p0 + 32 < re) i_next = rows[p + 32 < re ? p + 32 : rs];
        const float4 Pi = D.P[i], Li = D.L[i], Vi = D.V[i];
        const uint32_t id_i = D.id[i];
        float dx, dy, dz;
        pair_dx<float>(Pi, Li, Pj, Lj, GEOM != GEOM_OPEN, side, dx, dy, dz);
        const float d = sqrt_pair(dist2_rn<float>(dx, dy, dz));
        const float g = overlap_g<float>(gtab, d, Pi.w, Pj.w);
        const float wx = Vi.x - Vj.x, wy = Vi.y - Vj.y, wz = Vi.z - Vj.z;
        const float w2 = wx * wx + wy * wy + wz * wz;
        float FA, FB;
        if (hot) {
          if (RM == DMB_RATE_QUAD) {
            rates_quad<float>(w2 * inv2s2, rc.n, alpha, FA, FB, qv);
          } else if (RM == DMB_RATE_MLP) {
            const float2 fr = mr.rates[valid ? p : rs];
            FA = fr.x;
            FB = fr.y;
          } else {
            rates_FAB<float>(w2 * inv2s2, rc.n, FA, FB);
          }
        } else {
          const float wn = sqrt_t(w2);
          const float sn = sigma_ratio<float>(wn, rc.n, inv_v0, inv_vc2);
          FA = sn * wn;
          FB = sn * wn * w2;
        }
        if (!valid) continue;
        const float t = Li.w * g;
        const float tA = t * FA;
        sx += tA * wx;
        sy += tA * wy;
        sz += tA * wz;
        sw2 += tA * w2;
        sb += t * FB;
        svw += tA * (Vi.x * wx + Vi.y * wy + Vi.z * wz);
        float rx, ry, rz, vr;
        pg[p] = pair_probability_g<float>(g, Vi, id_i, Vj, Kj, id_j, rc.n, inv_v0, inv_vc2, dt, step, k0, k1, rx, ry,
                                          rz, vr);
      }
      sx = warp_sum<float>(sx);
      sy = warp_sum<float>(sy);
      sz = warp_sum<float>(sz);
      sw2 = warp_sum<float>(sw2);
      sb = warp_sum<float>(sb);
      svw = warp_sum<float>(svw);
    }
    if (lane < 6) {
      const float v = lane == 0 ? sx : lane == 1 ? sy : lane == 2 ? sz : lane == 3 ? sw2 : lane == 4 ? sb : svw;
      part[6 * u + lane] = v;
    }
  }
}

// The Monte Carlo of a float32 step after the fused pass: k_mc with each P_ij read from pg at the
// pair's gas-major position gidx[p] instead of being evaluated; the records are those of k_mc.
template <int GEOM>
__global__ void __launch_bounds__(MC_WARPS * 32, 4)
k_mc_select(SpeciesView<float> D, SpeciesView<float> G, BoxSplit bx, const int64_t *__restrict__ row_ptr,
            const uint32_t *__restrict__ rows, const uint32_t *__restrict__ gidx, const float *__restrict__ pg,
            const float4 *__restrict__ gtab, RunConst rc, McArgs a, McRec *__restrict__ rec) {
  const unsigned lane = threadIdx.x & 31u;
  const int wib = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * MC_WARPS;
  const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
  const float inv_v0 = (float)(1.0 / rc.v0);
  const float inv_vc2 = (float)rc.inv_vc2;
  const float beta = (float)a.beta;
  const unsigned long long step = a.step_dev ? *a.step_dev : a.step;
  const int64_t nrows = D.n;
  const float dt = (float)a.dt;
  const int64_t warp_id = (int64_t)blockIdx.x * MC_WARPS + wib;
  for (int64_t row0 = warp_id; row0 < nrows; row0 += 32 * nwarps) {
    const int64_t kl = row0 + (int64_t)lane * nwarps;
    bool busy = false;
    if (kl < nrows) {
      busy = row_ptr[kl + 1] > row_ptr[kl];
      if (!busy) {
        McRec r;
        r.c_lo = 0ull; r.c_hi = 0ull; r.rmax = 0.0f; r.flags = 0u; r.partner = 0xffffffffu;
        r.dv[0] = r.dv[1] = r.dv[2] = 0.0;
        rec[kl] = r;
      }
    }
    for (unsigned busy_rows = __ballot_sync(DMB_FULL, busy); busy_rows; busy_rows &= busy_rows - 1) {
      const int64_t i = __shfl_sync(DMB_FULL, kl, __ffs(busy_rows) - 1);
      const int64_t rs = row_ptr[i], re = row_ptr[i + 1];
      U128 sum = {0ull, 0ull};
      float rmax = 0.0f;
      for (int64_t p = rs + lane; p < re; p += 32) {
        const float P = pg[gidx[p]];
        sum = u128_add(sum, to_fixed(P));
        const float e = G.K[rows[p]].w;                     // mu_j / (m_chi + mu_j)
        const float inv_cap = 1e4f * e * e > 10.0f ? 1e4f * e * e : 10.0f;
        rmax = fmaxf(rmax, P * inv_cap);
      }
      const U128 C = warp_sum_u128(sum);
      rmax = warp_max(rmax);
      const uint32_t id_i = D.id[i];
      const uint4 wd = philox4x32_10(dm_counter(id_i, step), k0, k1);
      const unsigned long long k52 = ((unsigned long long)wd.x << 20) | (unsigned long long)(wd.w >> 12);
      const unsigned long long R64 = (k52 << 12) | (1ull << 11);
      const bool clamped = C.hi >= 1ull;
      U128 T;
      if (clamped) T = u128_scale(R64, C); else { T.hi = 0ull; T.lo = R64; }
      const bool scat = u128_lt(T, C);
      bool band = near_rel(T, C, C);
      float dv0 = 0, dv1 = 0, dv2 = 0;
      uint32_t partner_id = 0xffffffffu;
      if (scat) {
        uint32_t prefix = 0;
        U128 base = {0ull, 0ull};
        for (int b = a.id_bits - 1; b >= 0; --b) {
          const uint32_t mid = prefix | (1u << b);
          U128 S = {0ull, 0ull};
          for (int64_t p = rs + lane; p < re; p += 32) {
            const uint32_t idj = G.id[rows[p]];
            if (idj >= prefix && idj < mid) S = u128_add(S, to_fixed(pg[gidx[p]]));
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
          const float4 Pi = D.P[i], Li = D.L[i], Vi = D.V[i];
          const BoxSide side = box_side<GEOM>(bx, GEOM == GEOM_BOXES ? (int)D.bid[i] : 0);
          const float4 Pj = G.P[j], Lj = G.L[j], Vj = G.V[j], Kj = G.K[j];
          float rx, ry, rz, vr;
          (void)pair_probability<float>(Pi, Li, Vi, id_i, Pj, Lj, Vj, Kj, G.id[j], GEOM != GEOM_OPEN, side, gtab, rc.n,
                                        inv_v0, inv_vc2, dt, step, k0, k1, rx, ry, rz, vr);
          const U128 hi = u128_add(base, to_fixed(pg[gidx[pstar]]));
          band = band || near_rel(T, base, hi) || near_rel(T, hi, hi);
          const float ct = 2.0f * uniform23<float>(wd.y) - 1.0f;
          const float st = sqrt_t(fmaxf(0.0f, 1.0f - ct * ct));
          float sp, cp;
          sincospif(2.0f * uniform23<float>(wd.z), &sp, &cp);
          const float f = Kj.w * vr;
          const float inv = 1.0f / vr;
          if (beta == 0.0f) {
            dv0 = f * (st * cp - rx * inv);
            dv1 = f * (st * sp - ry * inv);
            dv2 = f * (ct - rz * inv);
          } else {
            const float ux = rx * inv, uy = ry * inv, uz = rz * inv;
            float nx, ny, nz;
            aniso_direction<float>(ct, sp, cp, beta, ux, uy, uz, nx, ny, nz);
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

cudaError_t launch_pairs_fused(SpeciesView<float> G, SpeciesView<float> D, BoxSplit bx, const int64_t *row_ptr,
                               const uint32_t *rows, SegView sv, int64_t n_seg_max, const float4 *gtab, RunConst rc,
                               MfOut out, float *part, MlpRun mr, McArgs a, float *pg, int blocks_per_sm,
                               cudaStream_t s, int64_t *launches) {
  if (G.n <= 0) return cudaSuccess;
  int64_t blocks = (n_seg_max + MF_WARPS - 1) / MF_WARPS;
  if (blocks > 152 * (int64_t)blocks_per_sm) blocks = 152 * (int64_t)blocks_per_sm;
  if (blocks < 1) blocks = 1;
#define PF(RM, G_) \
  k_pairs_fused<RM, G_><<<(unsigned)blocks, MF_WARPS * 32, 0, s>>>(G, D, bx, row_ptr, rows, sv, gtab, rc, part, mr, a, pg)
#define PF_GEOM(RM)                                       \
  switch (geom_of(bx)) {                                  \
    case GEOM_OPEN: PF(RM, GEOM_OPEN); break;             \
    case GEOM_BOX: PF(RM, GEOM_BOX); break;               \
    default: PF(RM, GEOM_BOXES); break;                   \
  }
  if (rc.rate_mode == DMB_RATE_QUAD) {
    PF_GEOM(DMB_RATE_QUAD)
  } else if (rc.rate_mode == DMB_RATE_MLP) {
    PF_GEOM(DMB_RATE_MLP)
  } else {
    PF_GEOM(DMB_RATE_CLOSED)
  }
#undef PF_GEOM
#undef PF
  k_meanfield_finish<float><<<(unsigned)((G.n + 255) / 256), 256, 0, s>>>(G, sv, part, out);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_mc_select(SpeciesView<float> D, SpeciesView<float> G, BoxSplit bx, const int64_t *row_ptr,
                             const uint32_t *rows, const uint32_t *gidx, const float *pg, const float4 *gtab,
                             RunConst rc, McArgs a, McRec *rec, int finish_blocks, int blocks_per_sm, cudaStream_t s,
                             int64_t *launches) {
  if (D.n <= 0) return cudaSuccess;
  int64_t blocks = (D.n + MC_WARPS - 1) / MC_WARPS;
  if (blocks > 152 * (int64_t)blocks_per_sm) blocks = 152 * (int64_t)blocks_per_sm;
  switch (geom_of(bx)) {
    case GEOM_OPEN: k_mc_select<GEOM_OPEN><<<(unsigned)blocks, MC_WARPS * 32, 0, s>>>(D, G, bx, row_ptr, rows, gidx, pg, gtab, rc, a, rec); break;
    case GEOM_BOX: k_mc_select<GEOM_BOX><<<(unsigned)blocks, MC_WARPS * 32, 0, s>>>(D, G, bx, row_ptr, rows, gidx, pg, gtab, rc, a, rec); break;
    default: k_mc_select<GEOM_BOXES><<<(unsigned)blocks, MC_WARPS * 32, 0, s>>>(D, G, bx, row_ptr, rows, gidx, pg, gtab, rc, a, rec); break;
  }
  const float *Lbase = reinterpret_cast<const float *>(D.L);
  k_mc_finish<<<finish_blocks, 256, 0, s>>>(D.n, D.perm, rec, Lbase + 3, nullptr, 4, a);
  if (launches) *launches += 2;
  return cudaGetLastError();
}
