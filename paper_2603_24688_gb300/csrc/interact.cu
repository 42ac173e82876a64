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
template <typename R, int RM, int GEOM>
__global__ void __launch_bounds__(MF_WARPS * 32)
k_meanfield(SpeciesView<R> G, SpeciesView<R> D, BoxSplit bx, const int64_t *__restrict__ row_ptr,
            const uint32_t *__restrict__ rows, SegView sv, const float4 *__restrict__ gtab, RunConst rc,
            R *__restrict__ part, MlpRun mr) {
  typedef typename Vec<R>::v4 v4;
  unsigned fallback = 0;
  const unsigned lane = threadIdx.x & 31u;
  const int64_t nwarps = (int64_t)gridDim.x * MF_WARPS;
  const R inv_v0 = (R)(1.0 / rc.v0);
  const R inv_vc2 = (R)rc.inv_vc2;
  const R alpha = (R)rc.alpha;
  const int64_t n_seg = sv.n_seg >= 0 ? sv.n_seg : sv.seg_ptr[G.n];
  for (int64_t u = (int64_t)blockIdx.x * MF_WARPS + (threadIdx.x >> 5); u < n_seg; u += nwarps) {
    const int64_t j = sv.seg_row[u];
    const int64_t rs = sv.seg_begin[u], re = min(rs + (int64_t)sv.seg_len, row_ptr[j + 1]);
    R sx = 0, sy = 0, sz = 0, sw2 = 0, sb = 0, svw = 0;
    if (re > rs) {
      const v4 Pj = G.P[j], Lj = G.L[j], Vj = G.V[j];
      const BoxSide side = box_side<GEOM>(bx, GEOM == GEOM_BOXES ? (int)G.bid[j] : 0);
      const R sig = Vj.w;
      const bool hot = sig > (R)0;
      const R inv2s2 = hot ? (R)0.5 / (sig * sig) : (R)0;
      const R qv = sig * sig * inv_vc2;                 // varsigma^2 / v_c^2 (screened law)
      // warp-uniform trip count (the surrogate's tensor-core layers need all 32 lanes)
      // each pass loads the next pass's partner index ahead of its own gathers
      uint32_t i_next = rows[rs + lane < re ? rs + lane : rs];
      for (int64_t p0 = rs; p0 < re; p0 += 32) {
        const int64_t p = p0 + lane;
        const bool valid = p < re;
        const uint32_t i = i_next;
        if (p0 + 32 < re) i_next = rows[p + 32 < re ? p + 32 : rs];
        const v4 Pi = D.P[i], Li = D.L[i], Vi = D.V[i];
        R dx, dy, dz;
        pair_dx<R>(Pi, Li, Pj, Lj, GEOM != GEOM_OPEN, side, dx, dy, dz);
        const R d = sqrt_pair(dist2_rn<R>(dx, dy, dz));
        const R g = overlap_g<R>(gtab, d, Pi.w, Pj.w);
        const R wx = Vi.x - Vj.x, wy = Vi.y - Vj.y, wz = Vi.z - Vj.z;
        const R w2 = wx * wx + wy * wy + wz * wz;
        R FA, FB;
        if (hot) {
          if (RM == DMB_RATE_QUAD) {
            rates_quad<R>(w2 * inv2s2, rc.n, alpha, FA, FB, qv);
          } else if (RM == DMB_RATE_MLP) {
            const float2 fr = mr.rates[valid ? p : rs];    // from k_mlp_pair_rates
            FA = (R)fr.x;
            FB = (R)fr.y;
          } else {
            rates_FAB<R>(w2 * inv2s2, rc.n, FA, FB);
          }
        } else {
          const R wn = sqrt_t(w2);
          const R sn = sigma_ratio<R>(wn, rc.n, inv_v0, inv_vc2);
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
  (void)fallback;
}

// ---- surrogate rates of every gas-major pair (before the mean field) ---------------------
#define MLP_ACT_OFFSET ((sizeof(MlpSmemPad) + 127) / 128 * 128)
static_assert(MLP_ACT_OFFSET % 16 == 0, "activation buffers must be 16-byte aligned for ldmatrix");
static_assert((MLP_LDW * sizeof(__nv_bfloat16)) % 16 == 0, "padded rows must keep 16-byte alignment");
// One warp per mean-field segment; 32 pairs per iteration: the inputs of pair p0 + r in lane r,
// layer 1 lane by lane into the warp's activation buffer, the two 128 x 128 layers on the tensor
// cores (mlp_layer32), the output layer on the CUDA cores.  Pairs outside the training box get
// the quadrature instead, counted.
__global__ void __launch_bounds__(MF_WARPS * 32)
k_mlp_pair_rates(SpeciesView<float> G, SpeciesView<float> D, const int64_t *__restrict__ row_ptr,
                 const uint32_t *__restrict__ rows, SegView sv, RunConst rc, MlpRun mr, float2 *__restrict__ rates) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MlpSmemPad &M = *reinterpret_cast<MlpSmemPad *>(smraw);
  // ldmatrix needs 16-byte aligned rows: the activation buffers start on a 128-byte boundary
  __nv_bfloat16 *actbuf = reinterpret_cast<__nv_bfloat16 *>(smraw + MLP_ACT_OFFSET);
  for (int t = threadIdx.x; t < MLP_H * MLP_H / 2; t += blockDim.x) {
    const int o = (2 * t) / MLP_H, i = (2 * t) % MLP_H;
    *reinterpret_cast<uint32_t *>(&M.W2[o * MLP_LDW + i]) = *reinterpret_cast<const uint32_t *>(&mr.w2[2 * t]);
    *reinterpret_cast<uint32_t *>(&M.W3[o * MLP_LDW + i]) = *reinterpret_cast<const uint32_t *>(&mr.w3[2 * t]);
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
  const unsigned lane = threadIdx.x & 31u;
  __nv_bfloat16 *act = actbuf + (threadIdx.x >> 5) * 32 * MLP_LDW;
  const int64_t nwarps = (int64_t)gridDim.x * MF_WARPS;
  const int64_t n_seg = sv.n_seg >= 0 ? sv.n_seg : sv.seg_ptr[G.n];
  const float alpha = (float)rc.alpha;
  unsigned fallback = 0;
  for (int64_t u = (int64_t)blockIdx.x * MF_WARPS + (threadIdx.x >> 5); u < n_seg; u += nwarps) {
    const int64_t j = sv.seg_row[u];
    const int64_t rs = sv.seg_begin[u], re = min(rs + (int64_t)sv.seg_len, row_ptr[j + 1]);
    if (re <= rs) continue;
    const float4 Vj = G.V[j];
    const float sig = Vj.w;
    if (!(sig > 0.0f)) continue;                        // cold gas: the mean field uses the exact limit
    for (int64_t p0 = rs; p0 < re; p0 += 32) {
      const int64_t p = p0 + lane;
      const bool valid = p < re;
      const float4 Vi = D.V[rows[valid ? p : rs]];
      const float wx = Vi.x - Vj.x, wy = Vi.y - Vj.y, wz = Vi.z - Vj.z;
      const float w2 = wx * wx + wy * wy + wz * wz;
      const float sig2 = sig * sig, s2 = __fdividef(w2, sig2);
      float xin[MLP_IN];
      const bool in_dom = mlp_inputs(mr.dom, s2, sig2, xin);
      // layer 1 for this lane's row
      __nv_bfloat16 *arow = act + lane * MLP_LDW;
#pragma unroll 4
      for (int c = 0; c < MLP_H; c += 2) {
        float z0 = M.b1[c], z1 = M.b1[c + 1];
#pragma unroll
        for (int m = 0; m < MLP_IN; ++m) { z0 += M.W1[c * MLP_IN + m] * xin[m]; z1 += M.W1[(c + 1) * MLP_IN + m] * xin[m]; }
        *reinterpret_cast<uint32_t *>(arow + c) = pack_bf16(mlp_act(z0), mlp_act(z1));
      }
      __syncwarp();
      float y[2][2][MLP_OUT] = {{{0.f, 0.f}, {0.f, 0.f}}, {{0.f, 0.f}, {0.f, 0.f}}};
      mlp_layer32(M.W2, M.b2, act, false, M.W4, y);
      mlp_layer32(M.W3, M.b3, act, true, M.W4, y);
      // output layer: reduce the partial dot products over the 4 lanes of each quad
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int o = 0; o < MLP_OUT; ++o) {
            float v = y[m][h][o];
            v += __shfl_xor_sync(DMB_FULL, v, 1);
            v += __shfl_xor_sync(DMB_FULL, v, 2);
            y[m][h][o] = v + M.b4[o];
          }
      // row r = lane: held by quad (r mod 16) mod 8 as m = r / 16, half = (r mod 16) / 8
      const int r = (int)lane, m = r >> 4, hf = (r >> 3) & 1, src = 4 * (r & 7);
      float yr[MLP_OUT];
#pragma unroll
      for (int o = 0; o < MLP_OUT; ++o) {
        const float c00 = __shfl_sync(DMB_FULL, y[0][0][o], src), c01 = __shfl_sync(DMB_FULL, y[0][1][o], src);
        const float c10 = __shfl_sync(DMB_FULL, y[1][0][o], src), c11 = __shfl_sync(DMB_FULL, y[1][1][o], src);
        yr[o] = m == 0 ? (hf == 0 ? c00 : c01) : (hf == 0 ? c10 : c11);
      }
      if (valid) {
        float FA, FB;
        if (in_dom) {
          mlp_outputs(mr.dom, s2, sig2, yr, FA, FB);
        } else {
          rates_quad<float>(0.5f * s2, rc.n, alpha, FA, FB, sig2 * (float)rc.inv_vc2);
          ++fallback;
        }
        rates[p] = make_float2(FA, FB);
      }
    }
  }
  fallback = warp_sum<unsigned>(fallback);
  if (lane == 0 && fallback && mr.fallback_count) atomicAdd(mr.fallback_count, (unsigned long long)fallback);
}

static const size_t kMlpRatesSmem = MLP_ACT_OFFSET + (size_t)MF_WARPS * 32 * MLP_LDW * sizeof(__nv_bfloat16);

cudaError_t prepare_mlp_pair_rates() {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_pair_rates, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMlpRatesSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return cudaSuccess;
}

cudaError_t launch_mlp_pair_rates(SpeciesView<float> G, SpeciesView<float> D, const int64_t *row_ptr,
                                  const uint32_t *rows, SegView sv, int64_t n_seg_max, RunConst rc, MlpRun mr,
                                  float2 *rates, cudaStream_t s, int64_t *launches) {
  const size_t smem = kMlpRatesSmem;
  cudaError_t e = prepare_mlp_pair_rates();
  if (e != cudaSuccess) return e;
  int64_t blocks = (n_seg_max + MF_WARPS - 1) / MF_WARPS;
  if (blocks > 152 * 2) blocks = 152 * 2;
  if (blocks < 1) blocks = 1;
  k_mlp_pair_rates<<<(unsigned)blocks, MF_WARPS * 32, smem, s>>>(G, D, row_ptr, rows, sv, rc, mr, rates);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

// acc_j = cA sum(t FA w), du_j/dt = cA sum(t FA w^2) - cB sum(t FB), and the App. C expected
// DM energy change of the pairs, M_j (cB sum(t FB) - cA sum(t FA v_i.w)), without dt
template <typename R>
__global__ void k_meanfield_finish(SpeciesView<R> G, SegView sv, const R *__restrict__ part, MfOut out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (sv.list ? sv.n_rows : G.n)) return;
  const int64_t j = sv.list ? (int64_t)sv.list[k] : k;
  const typename Vec<R>::v4 K = G.K[j];
  const double cA = (double)K.x, cB = (double)K.y;
  double q[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t u = sv.seg_ptr[k]; u < sv.seg_ptr[k + 1]; ++u)   // segments in order: deterministic
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
                             MfOut out, R *part, MlpRun mr, int blocks_per_sm, cudaStream_t s, int64_t *launches) {
  if (G.n <= 0) return cudaSuccess;
  int64_t blocks = (n_seg_max + MF_WARPS - 1) / MF_WARPS;
  if (blocks > 152 * (int64_t)blocks_per_sm) blocks = 152 * (int64_t)blocks_per_sm;
  if (blocks < 1) blocks = 1;
#define MF(RM, G_) k_meanfield<R, RM, G_><<<(unsigned)blocks, MF_WARPS * 32, 0, s>>>(G, D, bx, row_ptr, rows, sv, gtab, rc, part, mr)
#define MF_GEOM(RM)                                       \
  switch (geom_of(bx)) {                                  \
    case GEOM_OPEN: MF(RM, GEOM_OPEN); break;             \
    case GEOM_BOX: MF(RM, GEOM_BOX); break;               \
    default: MF(RM, GEOM_BOXES); break;                   \
  }
  if (rc.rate_mode == DMB_RATE_QUAD) {
    MF_GEOM(DMB_RATE_QUAD)
  } else if (rc.rate_mode == DMB_RATE_MLP) {
    MF_GEOM(DMB_RATE_MLP)
  } else {
    MF_GEOM(DMB_RATE_CLOSED)
  }
#undef MF_GEOM
#undef MF
  const int64_t nfin = sv.list ? sv.n_rows : G.n;
  if (nfin > 0) k_meanfield_finish<R><<<(unsigned)((nfin + 255) / 256), 256, 0, s>>>(G, sv, part, out);
  if (launches) *launches += 2;
  return cudaGetLastError();
}
template cudaError_t launch_meanfield<float>(SpeciesView<float>, SpeciesView<float>, BoxSplit, const int64_t *,
                                             const uint32_t *, SegView, int64_t, const float4 *, RunConst, MfOut,
                                             float *, MlpRun, int, cudaStream_t, int64_t *);
template cudaError_t launch_meanfield<double>(SpeciesView<double>, SpeciesView<double>, BoxSplit, const int64_t *,
                                              const uint32_t *, SegView, int64_t, const float4 *, RunConst, MfOut,
                                              double *, MlpRun, int, cudaStream_t, int64_t *);

// ---- Monte Carlo: one warp per DM particle ---------------------------------------------
// The sampled partner velocity v^B_ij = V_j + varsigma_j z (z from the pair's Philox block)
// and P_ij = (M_j/mu_j) g_ij sigma(v_rel) v_rel dt.
// P_ij given the pair's overlap g (the fused pair pass computes g once for both the mean field
// and the Monte Carlo; pair_probability below computes it first)
template <typename R>
__device__ __forceinline__ R pair_probability_g(R g, const typename Vec<R>::v4 &Vi, uint32_t id_i,
                                                const typename Vec<R>::v4 &Vj, const typename Vec<R>::v4 &Kj,
                                                uint32_t id_j, int n, R inv_v0, R inv_vc2, R dt,
                                                unsigned long long step, uint32_t k0, uint32_t k1, R &rx, R &ry,
                                                R &rz, R &vrel) {
  const uint4 w = philox4x32_10(pair_counter(id_i, id_j, step), k0, k1);
  R z0, z1, z2;
  box_muller3<R>(w, z0, z1, z2);
  const R sig = Vj.w;
  rx = Vi.x - (Vj.x + sig * z0);
  ry = Vi.y - (Vj.y + sig * z1);
  rz = Vi.z - (Vj.z + sig * z2);
  vrel = sqrt_pair(rx * rx + ry * ry + rz * rz);
  return Kj.z * dt * g * sigma_ratio<R>(vrel, n, inv_v0, inv_vc2) * vrel;
}

template <typename R>
__device__ __forceinline__ R pair_probability(const typename Vec<R>::v4 &Pi, const typename Vec<R>::v4 &Li,
                                              const typename Vec<R>::v4 &Vi, uint32_t id_i,
                                              const typename Vec<R>::v4 &Pj, const typename Vec<R>::v4 &Lj,
                                              const typename Vec<R>::v4 &Vj, const typename Vec<R>::v4 &Kj,
                                              uint32_t id_j, int periodic, const BoxSide &side, const float4 *gtab,
                                              int n, R inv_v0, R inv_vc2, R dt, unsigned long long step,
                                              uint32_t k0, uint32_t k1, R &rx, R &ry, R &rz, R &vrel) {
  R dx, dy, dz;
  pair_dx<R>(Pi, Li, Pj, Lj, periodic, side, dx, dy, dz);
  const R d = sqrt_pair(dist2_rn<R>(dx, dy, dz));
  const R g = overlap_g<R>(gtab, d, Pi.w, Pj.w);
  return pair_probability_g<R>(g, Vi, id_i, Vj, Kj, id_j, n, inv_v0, inv_vc2, dt, step, k0, k1, rx, ry, rz, vrel);
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

template <typename R, int GEOM>
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
        const v4 Pj = G.P[j], Lj = G.L[j], Vj = G.V[j], Kj = G.K[j];
        R rx, ry, rz, vr;
        const R P = pair_probability<R>(Pi, Li, Vi, id_i, Pj, Lj, Vj, Kj, G.id[j], GEOM != GEOM_OPEN, side, gtab, rc.n, inv_v0,
                                        inv_vc2, dt, step, k0, k1, rx, ry, rz, vr);
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
          const v4 Pj = G.P[j], Lj = G.L[j], Vj = G.V[j], Kj = G.K[j];
          R rx, ry, rz, vr;
          (void)pair_probability<R>(Pi, Li, Vi, id_i, Pj, Lj, Vj, Kj, G.id[j], GEOM != GEOM_OPEN, side, gtab, rc.n, inv_v0, inv_vc2, dt,
                                    step, k0, k1, rx, ry, rz, vr);
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

// float64 side of the Monte Carlo, one thread per DM particle: new velocities in caller
// order and deterministic block partials of the step sums
__global__ void __launch_bounds__(256)
k_mc_finish(int64_t n, const uint32_t *__restrict__ perm, const McRec *__restrict__ rec,
            const float *__restrict__ mass_f, const double *__restrict__ mass_d, int mass_stride, McArgs a) {
  __shared__ double red[8][256];
  __shared__ float redm[256];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  float mx = 0.0f;
  const int64_t nrows = a.list ? a.n_list : n;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nrows; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = a.list ? (int64_t)a.list[k] : k;
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
    if (a.v_sorted != nullptr) {   // keep the sorted copy current for the next substep
      if (a.v_sorted_fp64) reinterpret_cast<double4_32a *>(a.v_sorted)[i] = Vec<double>::make(n0, n1, n2, 0.0);
      else reinterpret_cast<float4 *>(a.v_sorted)[i] = make_float4((float)n0, (float)n1, (float)n2, 0.0f);
    }
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
    switch (geom_of(bx)) {
      case GEOM_OPEN: k_mc<R, GEOM_OPEN><<<(unsigned)blocks, MC_WARPS * 32, 0, s>>>(D, G, bx, row_ptr, rows, gtab, rc, a, pcache, rec); break;
      case GEOM_BOX: k_mc<R, GEOM_BOX><<<(unsigned)blocks, MC_WARPS * 32, 0, s>>>(D, G, bx, row_ptr, rows, gtab, rc, a, pcache, rec); break;
      default: k_mc<R, GEOM_BOXES><<<(unsigned)blocks, MC_WARPS * 32, 0, s>>>(D, G, bx, row_ptr, rows, gtab, rc, a, pcache, rec); break;
    }
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
