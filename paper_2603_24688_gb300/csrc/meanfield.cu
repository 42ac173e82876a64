// Gas mean field (Eqs. gas-dVdt, gas-dTdt): the per-segment kernel, the warp-level surrogate
// rates, and the launcher with its float64 finish.
#include "interact.cuh"

// ---- mean field: one warp per gas particle, lanes stride over its DM partners ---------
// Per-lane partial sums and the reduction across the warp stay in the pair precision R;
// the float64 results (and the perm scatter to caller order) are formed by
// k_meanfield_finish with one thread per gas particle, where float64 instructions cover
// 32 particles each (GB300 runs float64 at 1/64 of the float32 rate).
// W: M_i g_ij comes from the pair weights wq (float32 pair sets searched with weights) instead of
// the positions and the overlap table.
template <typename R, int RM, int GEOM, bool W>
__global__ void __launch_bounds__(MF_WARPS * 32)
k_meanfield(SpeciesView<R> G, SpeciesView<R> D, BoxSplit bx, const int64_t *__restrict__ row_ptr,
            const uint32_t *__restrict__ rows, SegView sv, const float4 *__restrict__ gtab, RunConst rc,
            R *__restrict__ part, MlpRun mr, const float *__restrict__ wq) {
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
        const v4 Vi = D.V[i];
        R t;                           // M_i g_ij
        if constexpr (W) {
          t = valid ? (R)wq[p] : (R)0;   // formed by the search's emit pass
        } else {
          const v4 Pi = D.P[i], Li = D.L[i];
          R dx, dy, dz;
          pair_dx<R>(Pi, Li, Pj, Lj, GEOM != GEOM_OPEN, side, dx, dy, dz);
          const R d = sqrt_pair(dist2_rn<R>(dx, dy, dz));
          t = Li.w * overlap_g<R>(gtab, d, Pi.w, Pj.w);
        }
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

template <typename R>
cudaError_t launch_meanfield(SpeciesView<R> G, SpeciesView<R> D, BoxSplit bx, const int64_t *row_ptr,
                             const uint32_t *rows, SegView sv, int64_t n_seg_max, const float4 *gtab, RunConst rc,
                             MfOut out, R *part, MlpRun mr, int blocks_per_sm, cudaStream_t s, int64_t *launches,
                             const float *wq) {
  if (G.n <= 0) return cudaSuccess;
  int64_t blocks = (n_seg_max + MF_WARPS - 1) / MF_WARPS;
  if (blocks > 152 * (int64_t)blocks_per_sm) blocks = 152 * (int64_t)blocks_per_sm;
  if (blocks < 1) blocks = 1;
#define MF(RM, G_)                                                                                              \
  do {                                                                                                          \
    if constexpr (sizeof(R) == 4) {                                                                             \
      if (wq != nullptr) {                                                                                      \
        k_meanfield<R, RM, G_, true><<<(unsigned)blocks, MF_WARPS * 32, 0, s>>>(G, D, bx, row_ptr, rows, sv,  \
                                                                                 gtab, rc, part, mr, wq);      \
        break;                                                                                                  \
      }                                                                                                         \
    }                                                                                                           \
    k_meanfield<R, RM, G_, false><<<(unsigned)blocks, MF_WARPS * 32, 0, s>>>(G, D, bx, row_ptr, rows, sv, gtab, \
                                                                              rc, part, mr, nullptr);           \
  } while (0)
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
                                             float *, MlpRun, int, cudaStream_t, int64_t *, const float *);
template cudaError_t launch_meanfield<double>(SpeciesView<double>, SpeciesView<double>, BoxSplit, const int64_t *,
                                              const uint32_t *, SegView, int64_t, const float4 *, RunConst, MfOut,
                                              double *, MlpRun, int, cudaStream_t, int64_t *, const float *);
