// Pair physics: gas mean field (Eqs. gas-dVdt, gas-dTdt) and DM Monte Carlo
// (Eqs. dm-update-vels, dm-update-prob, scatter_chi, prob_criterion).
#include "mlp.cuh"
#include "pairs.cuh"
#include "physics.cuh"

#define MF_WARPS 8
#define MC_WARPS 8

// ---- mean field: one warp per gas particle, lanes stride over its DM partners ---------
// Per-lane partial sums and the reduction across the warp stay in the pair precision R;
// the float64 results (and the perm scatter to caller order) are formed by
// k_meanfield_finish with one thread per gas particle, where float64 instructions cover
// 32 particles each (GB300 runs float64 at 1/64 of the float32 rate).
template <typename R, int RM>
__global__ void __launch_bounds__(MF_WARPS * 32)
k_meanfield(SpeciesView<R> G, SpeciesView<R> D, BoxSplit bx, const int64_t *__restrict__ row_ptr,
            const uint32_t *__restrict__ rows, SegView sv, const float4 *__restrict__ gtab, RunConst rc,
            R *__restrict__ part, MlpRun mr) {
  typedef typename Vec<R>::v4 v4;
  extern __shared__ __align__(16) unsigned char mf_smem[];
  if (RM == DMB_RATE_MLP) {   // the network's weights, once per block
    MlpSmem &M = *reinterpret_cast<MlpSmem *>(mf_smem);
    for (int t = threadIdx.x; t < MLP_H * MLP_H / 8; t += blockDim.x) {
      reinterpret_cast<uint4 *>(M.W2)[t] = reinterpret_cast<const uint4 *>(mr.w2)[t];
      reinterpret_cast<uint4 *>(M.W3)[t] = reinterpret_cast<const uint4 *>(mr.w3)[t];
    }
    for (int t = threadIdx.x; t < MLP_H * MLP_IN; t += blockDim.x) M.W1[t] = mr.p[MLP_OFF_W1 + t];
    for (int t = threadIdx.x; t < MLP_H; t += blockDim.x) {
      M.b1[t] = mr.p[MLP_OFF_B1 + t];
      M.b2[t] = mr.p[MLP_OFF_B2 + t];
      M.b3[t] = mr.p[MLP_OFF_B3 + t];
    }
    for (int t = threadIdx.x; t < MLP_OUT * MLP_H; t += blockDim.x) M.W4[t] = mr.p[MLP_OFF_W4 + t];
    if (threadIdx.x < MLP_OUT) M.b4[threadIdx.x] = mr.p[MLP_OFF_B4 + threadIdx.x];
    __syncthreads();
  }
  unsigned fallback = 0;
  const unsigned lane = threadIdx.x & 31u;
  const int64_t nwarps = (int64_t)gridDim.x * MF_WARPS;
  const R inv_v0 = (R)(1.0 / rc.v0);
  const R alpha = (R)rc.alpha;
  const int64_t n_seg = sv.seg_ptr[G.n];
  for (int64_t u = (int64_t)blockIdx.x * MF_WARPS + (threadIdx.x >> 5); u < n_seg; u += nwarps) {
    const int64_t j = sv.seg_row[u];
    const int64_t rs = sv.seg_begin[u], re = min(rs + (int64_t)MF_SEG, row_ptr[j + 1]);
    R sx = 0, sy = 0, sz = 0, sw2 = 0, sb = 0, svw = 0;
    if (re > rs) {
      const v4 Pj = G.P[j], Lj = G.L[j], Vj = G.V[j];
      const R sig = Vj.w;
      const bool hot = sig > (R)0;
      const R inv2s2 = hot ? (R)0.5 / (sig * sig) : (R)0;
      // warp-uniform trip count (the surrogate's tensor-core layers need all 32 lanes)
      for (int64_t p0 = rs; p0 < re; p0 += 32) {
        const int64_t p = p0 + lane;
        const bool valid = p < re;
        const uint32_t i = rows[valid ? p : rs];
        const v4 Pi = D.P[i], Li = D.L[i], Vi = D.V[i];
        R dx, dy, dz;
        pair_dx<R>(Pi, Li, Pj, Lj, bx, dx, dy, dz);
        const R d = sqrt_t(dist2_rn<R>(dx, dy, dz));
        const R g = overlap_g<R>(gtab, d, Pi.w, Pj.w);
        const R wx = Vi.x - Vj.x, wy = Vi.y - Vj.y, wz = Vi.z - Vj.z;
        const R w2 = wx * wx + wy * wy + wz * wz;
        R FA, FB;
        if (hot) {
          if (RM == DMB_RATE_QUAD) {
            rates_quad<R>(w2 * inv2s2, rc.n, alpha, FA, FB);
          } else if (RM == DMB_RATE_MLP) {
            const MlpSmem &M = *reinterpret_cast<const MlpSmem *>(mf_smem);
            const float sgm = (float)sig, sv_ = sqrtf((float)w2) / sgm;
            float xin[MLP_IN];
            const bool in_dom = mlp_inputs(mr.dom, sv_, sgm, xin);
            float yme[MLP_OUT] = {0.f, 0.f};
            const unsigned gq = lane >> 2;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              float xl[MLP_IN], xh[MLP_IN], yl[MLP_OUT], yh[MLP_OUT];
#pragma unroll
              for (int m = 0; m < MLP_IN; ++m) {
                xl[m] = __shfl_sync(DMB_FULL, xin[m], 16 * half + gq);
                xh[m] = __shfl_sync(DMB_FULL, xin[m], 16 * half + gq + 8);
              }
              mlp_forward16(M, xl, xh, yl, yh);
              // row r of this half sits in lanes 4 (r mod 8) .. as y_lo (r < 8) or y_hi (r >= 8)
              const int r = (int)lane - 16 * half;
              const int src = 4 * (r & 7);
#pragma unroll
              for (int o = 0; o < MLP_OUT; ++o) {
                const float a = __shfl_sync(DMB_FULL, yl[o], src & 31), b = __shfl_sync(DMB_FULL, yh[o], src & 31);
                if (r >= 0 && r < 16) yme[o] = r < 8 ? a : b;
              }
            }
            float fa, fb;
            mlp_outputs(mr.dom, sv_, yme, fa, fb);
            FA = (R)fa;
            FB = (R)fb;
            if (valid && !in_dom) {   // outside the training box: the quadrature, counted
              rates_quad<R>(w2 * inv2s2, rc.n, alpha, FA, FB);
              ++fallback;
            }
          } else {
            rates_FAB<R>(w2 * inv2s2, rc.n, FA, FB);
          }
        } else {
          const R wn = sqrt_t(w2);
          const R sn = ipow<R>(wn * inv_v0, rc.n);
          FA = sn * wn;
          FB = sn * wn * w2;
        }
        if (!valid) continue;
        const R t = Li.w * g;          // M_i g_ij
        const R tA = t * FA;
        sx += tA * wx;
        sy += tA * wy;
        sz += tA * wz;
        sw2 += tA * w2;
        sb += t * FB;
        svw += tA * (Vi.x * wx + Vi.y * wy + Vi.z * wz);
      }
      sx = warp_sum<R>(sx);
      sy = warp_sum<R>(sy);
      sz = warp_sum<R>(sz);
      sw2 = warp_sum<R>(sw2);
      sb = warp_sum<R>(sb);
      svw = warp_sum<R>(svw);
    }
    if (lane < 6) {
      const R v = lane == 0 ? sx : lane == 1 ? sy : lane == 2 ? sz : lane == 3 ? sw2 : lane == 4 ? sb : svw;
      part[6 * u + lane] = v;
    }
  }
  if (RM == DMB_RATE_MLP && mr.fallback_count) {
    fallback = warp_sum<unsigned>(fallback);
    if (lane == 0 && fallback) atomicAdd(mr.fallback_count, (unsigned long long)fallback);
  }
}

// acc_j = cA sum(t FA w), du_j/dt = cA sum(t FA w^2) - cB sum(t FB), and the App. C expected
// DM energy change of the pairs, M_j (cB sum(t FB) - cA sum(t FA v_i.w)), without dt
template <typename R>
__global__ void k_meanfield_finish(SpeciesView<R> G, const int64_t *__restrict__ seg_ptr, const R *__restrict__ part,
                                   MfOut out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= G.n) return;
  const typename Vec<R>::v4 K = G.K[j];
  const double cA = (double)K.x, cB = (double)K.y;
  double q[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t u = seg_ptr[j]; u < seg_ptr[j + 1]; ++u)   // segments in order: deterministic
    for (int k = 0; k < 6; ++k) q[k] += (double)part[6 * u + k];
  const uint32_t c = G.perm[j];
  out.acc[3 * (int64_t)c + 0] = cA * q[0];
  out.acc[3 * (int64_t)c + 1] = cA * q[1];
  out.acc[3 * (int64_t)c + 2] = cA * q[2];
  out.dudt[c] = cA * q[3] - cB * q[4];
  if (out.e_exp) out.e_exp[j] = (double)G.L[j].w * (cB * q[4] - cA * q[5]);
}

template <typename R>
cudaError_t launch_meanfield(SpeciesView<R> G, SpeciesView<R> D, BoxSplit bx, const int64_t *row_ptr,
                             const uint32_t *rows, SegView sv, int64_t n_seg_max, const float4 *gtab, RunConst rc,
                             MfOut out, R *part, MlpRun mr, cudaStream_t s, int64_t *launches) {
  if (G.n <= 0) return cudaSuccess;
  int64_t blocks = (n_seg_max + MF_WARPS - 1) / MF_WARPS;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (rc.rate_mode == DMB_RATE_QUAD) {
    k_meanfield<R, DMB_RATE_QUAD><<<(unsigned)blocks, MF_WARPS * 32, 0, s>>>(G, D, bx, row_ptr, rows, sv, gtab, rc,
                                                                              part, mr);
  } else if (rc.rate_mode == DMB_RATE_MLP) {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k_meanfield<R, DMB_RATE_MLP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(MlpSmem));
      if (e != cudaSuccess) return e;
      attr = true;
    }
    k_meanfield<R, DMB_RATE_MLP><<<(unsigned)blocks, MF_WARPS * 32, sizeof(MlpSmem), s>>>(G, D, bx, row_ptr, rows, sv,
                                                                                           gtab, rc, part, mr);
  } else {
    k_meanfield<R, DMB_RATE_CLOSED><<<(unsigned)blocks, MF_WARPS * 32, 0, s>>>(G, D, bx, row_ptr, rows, sv, gtab, rc,
                                                                                part, mr);
  }
  k_meanfield_finish<R><<<(unsigned)((G.n + 255) / 256), 256, 0, s>>>(G, sv.seg_ptr, part, out);
  if (launches) *launches += 2;
  return cudaGetLastError();
}
template cudaError_t launch_meanfield<float>(SpeciesView<float>, SpeciesView<float>, BoxSplit, const int64_t *,
                                             const uint32_t *, SegView, int64_t, const float4 *, RunConst, MfOut,
                                             float *, MlpRun, cudaStream_t, int64_t *);
template cudaError_t launch_meanfield<double>(SpeciesView<double>, SpeciesView<double>, BoxSplit, const int64_t *,
                                              const uint32_t *, SegView, int64_t, const float4 *, RunConst, MfOut,
                                              double *, MlpRun, cudaStream_t, int64_t *);

// ---- Monte Carlo: one warp per DM particle ---------------------------------------------
// The sampled partner velocity v^B_ij = V_j + varsigma_j z (z from the pair's Philox block)
// and P_ij = (M_j/mu_j) g_ij sigma(v_rel) v_rel dt.
template <typename R>
__device__ __forceinline__ R pair_probability(const typename Vec<R>::v4 &Pi, const typename Vec<R>::v4 &Li,
                                              const typename Vec<R>::v4 &Vi, uint32_t id_i,
                                              const typename Vec<R>::v4 &Pj, const typename Vec<R>::v4 &Lj,
                                              const typename Vec<R>::v4 &Vj, const typename Vec<R>::v4 &Kj,
                                              uint32_t id_j, const BoxSplit &bx, const float4 *gtab, int n,
                                              R inv_v0, R dt, unsigned long long step, uint32_t k0, uint32_t k1,
                                              R &rx, R &ry, R &rz, R &vrel) {
  R dx, dy, dz;
  pair_dx<R>(Pi, Li, Pj, Lj, bx, dx, dy, dz);
  const R d = sqrt_t(dist2_rn<R>(dx, dy, dz));
  const R g = overlap_g<R>(gtab, d, Pi.w, Pj.w);
  const uint4 w = philox4x32_10(pair_counter(id_i, id_j, step), k0, k1);
  R z0, z1, z2;
  box_muller3<R>(w, z0, z1, z2);
  const R sig = Vj.w;
  rx = Vi.x - (Vj.x + sig * z0);
  ry = Vi.y - (Vj.y + sig * z1);
  rz = Vi.z - (Vj.z + sig * z2);
  vrel = sqrt_t(rx * rx + ry * ry + rz * rz);
  return Kj.z * dt * g * ipow<R>(vrel * inv_v0, n) * vrel;
}

// U128 comparison helpers for the decision band: |a - b| <= c 2^-20 (about 1e-6 c)
__device__ __forceinline__ U128 u128_absdiff(U128 a, U128 b) {
  U128 r;
  if (u128_lt(a, b)) { U128 t = a; a = b; b = t; }
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull);
  return r;
}
__device__ __forceinline__ U128 u128_shr20(U128 a) {
  U128 r;
  r.lo = (a.lo >> 20) | (a.hi << 44);
  r.hi = a.hi >> 20;
  return r;
}
__device__ __forceinline__ bool near_rel(U128 a, U128 b, U128 c) { return !u128_lt(u128_shr20(c), u128_absdiff(a, b)); }

template <typename R>
__global__ void __launch_bounds__(MC_WARPS * 32)
k_mc(SpeciesView<R> D, SpeciesView<R> G, BoxSplit bx, const int64_t *__restrict__ row_ptr,
     const uint32_t *__restrict__ rows, const float4 *__restrict__ gtab, RunConst rc, McArgs a,
     R *__restrict__ pcache, McRec *__restrict__ rec) {
  typedef typename Vec<R>::v4 v4;
  const unsigned lane = threadIdx.x & 31u;
  const int wib = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * MC_WARPS;
  const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
  const R inv_v0 = (R)(1.0 / rc.v0);
  const R dt = (R)a.dt;
  for (int64_t i = (int64_t)blockIdx.x * MC_WARPS + wib; i < D.n; i += nwarps) {
    const int64_t rs = row_ptr[i], re = row_ptr[i + 1];
    if (re == rs) {                       // no gas partner: nothing can happen
      if (lane == 0) {
        McRec r;
        r.c_lo = 0ull; r.c_hi = 0ull; r.rmax = 0.0f; r.flags = 0u; r.partner = 0xffffffffu;
        r.dv[0] = r.dv[1] = r.dv[2] = 0.0;
        rec[i] = r;
      }
      continue;
    }
    const v4 Pi = D.P[i], Li = D.L[i], Vi = D.V[i];
    const uint32_t id_i = D.id[i];
    U128 sum = {0ull, 0ull};
    float rmax = 0.0f;
    for (int64_t p = rs + lane; p < re; p += 32) {
      const uint32_t j = rows[p];
      const v4 Pj = G.P[j], Lj = G.L[j], Vj = G.V[j], Kj = G.K[j];
      R rx, ry, rz, vr;
      const R P = pair_probability<R>(Pi, Li, Vi, id_i, Pj, Lj, Vj, Kj, G.id[j], bx, gtab, rc.n, inv_v0, dt, a.step,
                                      k0, k1, rx, ry, rz, vr);
      pcache[p] = P;
      sum = u128_add(sum, to_fixed(P));
      const R e = Kj.w;                                   // mu_j / (m_chi + mu_j)
      const R cap = (R)1e-4 / (e * e) < (R)0.1 ? (R)1e-4 / (e * e) : (R)0.1;   // Eq. prob_criterion
      rmax = fmaxf(rmax, (float)(P / cap));
    }
    const U128 C = warp_sum_u128(sum);
    rmax = warp_max(rmax);
    // selection uniform r_i = (k + 1/2) 2^-52, k the top 52 bits of (w0, w3): as a 64-bit fraction
    const uint4 wd = philox4x32_10(dm_counter(id_i, a.step), k0, k1);
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
        const v4 Pj = G.P[j], Lj = G.L[j], Vj = G.V[j], Kj = G.K[j];
        R rx, ry, rz, vr;
        (void)pair_probability<R>(Pi, Li, Vi, id_i, Pj, Lj, Vj, Kj, G.id[j], bx, gtab, rc.n, inv_v0, dt, a.step, k0,
                                  k1, rx, ry, rz, vr);
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
        dv0 = f * (st * cp - rx * inv);
        dv1 = f * (st * sp - ry * inv);
        dv2 = f * (ct - rz * inv);
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

// float64 side of the Monte Carlo, one thread per DM particle: new velocities in caller
// order and deterministic block partials of the step sums
__global__ void __launch_bounds__(256)
k_mc_finish(int64_t n, const uint32_t *__restrict__ perm, const McRec *__restrict__ rec,
            const float *__restrict__ mass_f, const double *__restrict__ mass_d, int mass_stride, McArgs a) {
  __shared__ double red[8][256];
  __shared__ float redm[256];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  float mx = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const McRec r = rec[i];
    const uint32_t c = perm[i];
    const double M = mass_f ? (double)mass_f[(int64_t)mass_stride * i] : mass_d[(int64_t)mass_stride * i];
    const double v0 = a.vel_in[3 * (int64_t)c], v1 = a.vel_in[3 * (int64_t)c + 1], v2 = a.vel_in[3 * (int64_t)c + 2];
    double n0 = v0, n1 = v1, n2 = v2;
    if (r.flags & 1u) {
      n0 = v0 + r.dv[0];
      n1 = v1 + r.dv[1];
      n2 = v2 + r.dv[2];
      acc[0] += M * (n0 - v0);
      acc[1] += M * (n1 - v1);
      acc[2] += M * (n2 - v2);
      acc[3] += 0.5 * M * ((n0 * n0 + n1 * n1 + n2 * n2) - (v0 * v0 + v1 * v1 + v2 * v2));
      acc[4] += 1.0;
    }
    a.vel_out[3 * (int64_t)c] = n0;
    a.vel_out[3 * (int64_t)c + 1] = n1;
    a.vel_out[3 * (int64_t)c + 2] = n2;
    const double Cd = (r.c_hi | r.c_lo) ? (double)r.c_hi + ldexp((double)r.c_lo, -64) : 0.0;
    if (a.scattered) a.scattered[c] = (uint8_t)(r.flags & 1u);
    if (a.partner) a.partner[c] = r.partner;
    if (a.p_ratio) a.p_ratio[c] = r.rmax;
    if (a.p_total) a.p_total[c] = Cd;
    if (r.flags & 2u) acc[5] += 1.0;
    if (r.flags & 4u) acc[6] += 1.0;
    acc[7] += Cd;
    mx = fmaxf(mx, r.rmax);
  }
  const int t = threadIdx.x;
  for (int k = 0; k < 8; ++k) red[k][t] = acc[k];
  redm[t] = mx;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) {
      for (int k = 0; k < 8; ++k) red[k][t] += red[k][t + o];
      redm[t] = fmaxf(redm[t], redm[t + o]);
    }
    __syncthreads();
  }
  if (t < 8) a.block_sums[8 * (int64_t)blockIdx.x + t] = red[t][0];
  if (t == 0) a.block_max[blockIdx.x] = (double)redm[0];
}

template <typename R>
cudaError_t launch_mc(SpeciesView<R> D, SpeciesView<R> G, BoxSplit bx, const int64_t *row_ptr, const uint32_t *rows,
                      const float4 *gtab, RunConst rc, McArgs a, R *pcache, McRec *rec, int finish_blocks,
                      cudaStream_t s, int64_t *launches) {
  int64_t blocks = (D.n + MC_WARPS - 1) / MC_WARPS;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_mc<R><<<(unsigned)blocks, MC_WARPS * 32, 0, s>>>(D, G, bx, row_ptr, rows, gtab, rc, a, pcache, rec);
  // the particle mass sits in L.w of the sorted copies
  const R *Lbase = reinterpret_cast<const R *>(D.L);
  k_mc_finish<<<finish_blocks, 256, 0, s>>>(D.n, D.perm, rec, sizeof(R) == 4 ? (const float *)(Lbase + 3) : nullptr,
                                            sizeof(R) == 8 ? (const double *)(Lbase + 3) : nullptr, 4, a);
  if (launches) *launches += 2;
  return cudaGetLastError();
}
template cudaError_t launch_mc<float>(SpeciesView<float>, SpeciesView<float>, BoxSplit, const int64_t *,
                                      const uint32_t *, const float4 *, RunConst, McArgs, float *, McRec *, int,
                                      cudaStream_t, int64_t *);
template cudaError_t launch_mc<double>(SpeciesView<double>, SpeciesView<double>, BoxSplit, const int64_t *,
                                       const uint32_t *, const float4 *, RunConst, McArgs, double *, McRec *, int,
                                       cudaStream_t, int64_t *);

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
