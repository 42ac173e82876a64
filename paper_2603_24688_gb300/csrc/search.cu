// Warp-cooperative pair search over the chunk tree (count and emit passes).
#include "pairs.cuh"
#include "physics.cuh"

#define SR_WARPS 4
#define SR_STACK 64

__device__ __forceinline__ float axis_gap(float qa, float qb, float na, float nb) {
  return fmaxf(0.0f, fmaxf(na - qb, qa - nb));
}

template <typename R, bool EMIT>
__global__ void __launch_bounds__(SR_WARPS * 32)
k_pair_search(SpeciesView<R> Q, SpeciesView<R> O, BoxSplit bx, const Frame *__restrict__ frame,
              uint32_t *__restrict__ counts, const int64_t *__restrict__ row_ptr, uint32_t *__restrict__ rows,
              uint32_t *status) {
  typedef typename Vec<R>::v4 v4;
  __shared__ v4 sP[SR_WARPS][DMB_LEAF];
  __shared__ v4 sL[SR_WARPS][DMB_LEAF];
  const int wib = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31u;
  const int64_t nchunk = (Q.n + 31) / 32;
  const float pad = frame->pad;
  for (int64_t chunk = (int64_t)blockIdx.x * SR_WARPS + wib; chunk < nchunk; chunk += (int64_t)gridDim.x * SR_WARPS) {
    const int64_t qi = chunk * 32 + lane;
    const bool valid = qi < Q.n;
    v4 Pq = Vec<R>::make(0, 0, 0, 0), Lq = Vec<R>::make(0, 0, 0, 0);
    float c[3] = {0.f, 0.f, 0.f};
    float hq = 0.f;
    if (valid) {
      Pq = Q.P[qi];
      Lq = Q.L[qi];
      c[0] = (float)((double)Pq.x + (double)Lq.x);
      c[1] = (float)((double)Pq.y + (double)Lq.y);
      c[2] = (float)((double)Pq.z + (double)Lq.z);
      hq = (float)Pq.w;
    }
    float qmn[3], qmx[3], hqm = valid ? hq : 0.f;
    for (int k = 0; k < 3; ++k) { qmn[k] = valid ? c[k] : INFINITY; qmx[k] = valid ? c[k] : -INFINITY; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      for (int k = 0; k < 3; ++k) {
        qmn[k] = fminf(qmn[k], __shfl_xor_sync(DMB_FULL, qmn[k], o));
        qmx[k] = fmaxf(qmx[k], __shfl_xor_sync(DMB_FULL, qmx[k], o));
      }
      hqm = fmaxf(hqm, __shfl_xor_sync(DMB_FULL, hqm, o));
    }
    hqm *= (1.0f + 1e-6f);
    uint32_t cnt = 0;
    int64_t out_base = 0, out_end = 0;
    if (EMIT && valid) { out_base = row_ptr[qi]; out_end = row_ptr[qi + 1]; }
    int stack[SR_STACK];
    int sp = 0;
    stack[sp++] = 1;
    while (sp > 0) {
      const int node = stack[--sp];
      const float4 nmn = O.bmin[node], nmx = O.bmax[node];
      if (!(nmn.w >= 0.0f)) continue;                    // empty node
      float d2 = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float na = k == 0 ? nmn.x : (k == 1 ? nmn.y : nmn.z);
        const float nb = k == 0 ? nmx.x : (k == 1 ? nmx.y : nmx.z);
        float gap = axis_gap(qmn[k], qmx[k], na, nb);
        if (bx.periodic) {
          const float L = bx.Lhi[k];
          gap = fminf(gap, fminf(axis_gap(qmn[k] + L, qmx[k] + L, na, nb), axis_gap(qmn[k] - L, qmx[k] - L, na, nb)));
        }
        d2 += gap * gap;
      }
      const float r = hqm + nmn.w + 2.0f * pad;
      if (d2 >= r * r) continue;
      if (node >= O.p2) {
        const int64_t base = (int64_t)(node - O.p2) * DMB_LEAF;
        if (base >= O.n) continue;
        const int nk = (int)min((int64_t)DMB_LEAF, O.n - base);
        __syncwarp();
        if ((int)lane < nk) { sP[wib][lane] = O.P[base + lane]; sL[wib][lane] = O.L[base + lane]; }
        __syncwarp();
        if (valid) {
          for (int k = 0; k < nk; ++k) {
            const v4 Pk = sP[wib][k], Lk = sL[wib][k];
            R dx, dy, dz;
            pair_dx<R>(Pq, Lq, Pk, Lk, bx, dx, dy, dz);
            if (pair_test<R>(dist2_rn<R>(dx, dy, dz), Pq.w, Pk.w)) {
              if (EMIT) {
                const int64_t at = out_base + cnt;
                if (at < out_end) rows[at] = (uint32_t)(base + k);
              }
              ++cnt;
            }
          }
        }
      } else {
        if (sp + 2 > SR_STACK) { atomicOr(status, DMB_BAD_OVERFLOW); break; }
        stack[sp++] = 2 * node + 1;
        stack[sp++] = 2 * node;
      }
    }
    if (valid) {
      if (!EMIT) counts[qi] = cnt;
      else if ((int64_t)cnt != out_end - out_base) atomicOr(status, DMB_BAD_OVERFLOW);
    }
  }
}

template <typename R>
cudaError_t launch_pair_search(SpeciesView<R> Q, SpeciesView<R> O, BoxSplit bx, const Frame *frame, bool emit,
                               uint32_t *counts, const int64_t *row_ptr, uint32_t *rows, uint32_t *status,
                               cudaStream_t s, int64_t *launches) {
  if (Q.n <= 0) return cudaSuccess;
  const int64_t nchunk = (Q.n + 31) / 32;
  int64_t blocks = (nchunk + SR_WARPS - 1) / SR_WARPS;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (emit)
    k_pair_search<R, true><<<(unsigned)blocks, SR_WARPS * 32, 0, s>>>(Q, O, bx, frame, counts, row_ptr, rows, status);
  else
    k_pair_search<R, false><<<(unsigned)blocks, SR_WARPS * 32, 0, s>>>(Q, O, bx, frame, counts, row_ptr, rows, status);
  if (launches) *launches += 1;
  return cudaGetLastError();
}
template cudaError_t launch_pair_search<float>(SpeciesView<float>, SpeciesView<float>, BoxSplit, const Frame *, bool,
                                               uint32_t *, const int64_t *, uint32_t *, uint32_t *, cudaStream_t,
                                               int64_t *);
template cudaError_t launch_pair_search<double>(SpeciesView<double>, SpeciesView<double>, BoxSplit, const Frame *,
                                                bool, uint32_t *, const int64_t *, uint32_t *, uint32_t *,
                                                cudaStream_t, int64_t *);
