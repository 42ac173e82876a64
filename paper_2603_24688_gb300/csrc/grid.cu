// Frame, Morton keys, gather into sorted float copies, and the chunk tree.
#include <math.h>

#include "grid.cuh"

// ---- frame ---------------------------------------------------------------------------
#define FR_THREADS 256

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

// per block: min/max of x, y, z over both species and max h per species
__global__ void k_frame_partial(const double *__restrict__ dpos, const double *__restrict__ dh, int64_t nd,
                                const double *__restrict__ gpos, const double *__restrict__ gh, int64_t ng,
                                double *__restrict__ part) {
  __shared__ double red[8][FR_THREADS];
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  double hd = 0.0, hg = 0.0;
  const int64_t tot = nd + ng;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const double *p = i < nd ? dpos + 3 * i : gpos + 3 * (i - nd);
    for (int c = 0; c < 3; ++c) {
      const double v = p[c];
      if (finite_d(v)) { mn[c] = fmin(mn[c], v); mx[c] = fmax(mx[c], v); }
    }
    if (i < nd) hd = fmax(hd, dh[i]); else hg = fmax(hg, gh[i - nd]);
  }
  const int t = threadIdx.x;
  for (int c = 0; c < 3; ++c) { red[c][t] = mn[c]; red[3 + c][t] = mx[c]; }
  red[6][t] = hd;
  red[7][t] = hg;
  __syncthreads();
  for (int o = FR_THREADS / 2; o > 0; o >>= 1) {
    if (t < o) {
      for (int c = 0; c < 3; ++c) {
        red[c][t] = fmin(red[c][t], red[c][t + o]);
        red[3 + c][t] = fmax(red[3 + c][t], red[3 + c][t + o]);
      }
      red[6][t] = fmax(red[6][t], red[6][t + o]);
      red[7][t] = fmax(red[7][t], red[7][t + o]);
    }
    __syncthreads();
  }
  if (t < 8) part[blockIdx.x * 8 + t] = red[t][0];
}

__global__ void __launch_bounds__(256)
k_frame_final(const double *__restrict__ part, int nb, int periodic, double L0, double L1, double L2, int bits,
              Frame *frame, uint32_t *status) {
  __shared__ double red[8][256];
  const int t = threadIdx.x;
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  double hd = 0.0, hg = 0.0;
  for (int b = t; b < nb; b += 256) {
    for (int c = 0; c < 3; ++c) { mn[c] = fmin(mn[c], part[b * 8 + c]); mx[c] = fmax(mx[c], part[b * 8 + 3 + c]); }
    hd = fmax(hd, part[b * 8 + 6]);
    hg = fmax(hg, part[b * 8 + 7]);
  }
  for (int c = 0; c < 3; ++c) { red[c][t] = mn[c]; red[3 + c][t] = mx[c]; }
  red[6][t] = hd;
  red[7][t] = hg;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) {
      for (int c = 0; c < 3; ++c) {
        red[c][t] = fmin(red[c][t], red[c][t + o]);
        red[3 + c][t] = fmax(red[3 + c][t], red[3 + c][t + o]);
      }
      red[6][t] = fmax(red[6][t], red[6][t + o]);
      red[7][t] = fmax(red[7][t], red[7][t + o]);
    }
    __syncthreads();
  }
  if (t != 0) return;
  for (int c = 0; c < 3; ++c) { mn[c] = red[c][0]; mx[c] = red[3 + c][0]; }
  hd = red[6][0];
  hg = red[7][0];
  Frame f;
  double span;
  if (periodic) {
    for (int c = 0; c < 3; ++c) f.origin[c] = 0.0;
    span = fmax(L0, fmax(L1, L2));
    if (hd + hg >= 0.5 * fmin(L0, fmin(L1, L2))) atomicOr(status, DMB_BAD_PERIODIC);
  } else {
    span = 0.0;
    for (int c = 0; c < 3; ++c) {
      if (!(mx[c] >= mn[c])) { mn[c] = 0.0; mx[c] = 0.0; }
      f.origin[c] = mn[c];
      span = fmax(span, mx[c] - mn[c]);
    }
    span = span > 0.0 ? span * (1.0 + 1e-9) : 1.0;
  }
  f.span = span;
  // smallest power of two delta with span <= 2^23 delta
  int e;
  frexp(span, &e);                 // span < 2^e
  f.delta = ldexp(1.0, e - 23);
  f.inv_delta = ldexp(1.0, 23 - e);
  f.bits = bits;
  f.key_scale = ldexp(1.0, bits) / span;
  f.pad = (float)(4.0 * ldexp(1.0, e) * 1.1920928955078125e-07);   // a few float ulps of the span
  f.hmax_dm = hd;
  f.hmax_gas = hg;
  *frame = f;
}

cudaError_t launch_frame(const double *dm_pos, const double *dm_h, int64_t ndm, const double *gas_pos,
                         const double *gas_h, int64_t ngas, int periodic, const double box[3], double *part,
                         int64_t part_elems, Frame *frame, uint32_t *status, cudaStream_t s, int64_t *launches) {
  int nb = (int)fmin((double)(part_elems / 8), 1024.0);
  const int64_t need = (ndm + ngas + FR_THREADS - 1) / FR_THREADS;
  if (need < nb) nb = (int)(need > 0 ? need : 1);
  const int64_t ntot = ndm + ngas;
  const int bits_per_axis = (int)fmin(21.0, fmax(10.0, ceil(log2((double)(ntot > 1 ? ntot : 2)) / 3.0) + 7.0));
  k_frame_partial<<<nb, FR_THREADS, 0, s>>>(dm_pos, dm_h, ndm, gas_pos, gas_h, ngas, part);
  k_frame_final<<<1, 256, 0, s>>>(part, nb, periodic, box[0], box[1], box[2], bits_per_axis, frame, status);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

// ---- Morton keys ---------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint64_t v) {  // 21 bits -> every third bit
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

__device__ __forceinline__ double wrap_coord(double x, double L) {
  double w = x - L * floor(x / L);
  if (w >= L) w -= L;
  if (w < 0.0) w = 0.0;
  return w;
}

// Single box: 3 x bits Morton key of the position in the frame.  Batched boxes: the box index in
// the bits above, then the Morton key of the position inside the box (so boxes stay contiguous).
__global__ void k_morton(const double *__restrict__ pos, int64_t n, int periodic, double L0, double L1, double L2,
                         const Frame *__restrict__ frame, BatchArgs ba, uint64_t *__restrict__ keys,
                         uint32_t *__restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Frame f = *frame;
  double Ls[3] = {L0, L1, L2};
  uint64_t boxkey = 0;
  if (ba.box_of != nullptr) {
    const uint32_t b = ba.box_of[i];
    for (int c = 0; c < 3; ++c) Ls[c] = ba.bp[b].L[c];
    boxkey = (uint64_t)b << (3 * f.bits);
  }
  const uint64_t top = (1ull << f.bits) - 1ull;
  uint64_t q[3];
  for (int c = 0; c < 3; ++c) {
    double x = pos[3 * i + c];
    if (periodic) x = wrap_coord(x, Ls[c]);
    double u = (ba.box_of != nullptr ? x : x - f.origin[c]) * f.key_scale;
    if (!(u >= 0.0)) u = 0.0;                      // also catches NaN (flagged in gather)
    uint64_t k = u >= (double)top ? top : (uint64_t)u;
    q[c] = k;
  }
  keys[i] = boxkey | spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
  vals[i] = (uint32_t)i;
}

cudaError_t launch_morton(const double *pos, int64_t n, int periodic, const double box[3], const Frame *frame,
                          BatchArgs ba, uint64_t *keys, uint32_t *vals, cudaStream_t s, int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  k_morton<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, n, periodic, box[0], box[1], box[2], frame, ba, keys, vals);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

// ---- gather into the sorted split representation ----------------------------------
template <typename R>
__global__ void k_gather(const double *__restrict__ pos, const double *__restrict__ vel,
                         const double *__restrict__ mass, const double *__restrict__ h, const double *__restrict__ T,
                         const double *__restrict__ mu, const uint32_t *__restrict__ id, int64_t n,
                         const uint32_t *__restrict__ perm, int periodic, double L0, double L1, double L2,
                         const Frame *__restrict__ frame, RunConst rc, BatchArgs ba,
                         typename Vec<R>::v4 *__restrict__ P, typename Vec<R>::v4 *__restrict__ Lo,
                         typename Vec<R>::v4 *__restrict__ V, typename Vec<R>::v4 *__restrict__ K,
                         uint32_t *__restrict__ sid, uint16_t *__restrict__ bid, uint32_t *status) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t i = perm[s];
  const double delta = frame->delta, inv_delta = frame->inv_delta;
  double Ls[3] = {L0, L1, L2};
  double xoff = 0.0;
  bool bad = false;
  if (ba.box_of != nullptr) {
    // batched boxes: this box's sides, constants and slot in the virtual space
    const uint32_t b = ba.box_of[i];
    const BoxParamDev bp = ba.bp[b];
    for (int c = 0; c < 3; ++c) Ls[c] = bp.L[c];
    xoff = bp.offset_x;
    rc.S = bp.S;
    rc.m_chi = bp.m_chi;
    bid[s] = (uint16_t)b;
    const double hh = h[i];
    if (!(hh < 0.25 * fmin(Ls[0], fmin(Ls[1], Ls[2])))) atomicOr(status, DMB_BAD_PERIODIC);
  }
  R hi[3], lo[3];
  for (int c = 0; c < 3; ++c) {
    double x = pos[3 * (int64_t)i + c];
    bad |= !isfinite(x);
    if (periodic) x = wrap_coord(x, Ls[c]);
    if (c == 0) x += xoff;
    const double rel = x - frame->origin[c];
    const double hq = floor(rel * inv_delta) * delta;   // k * delta, |k| < 2^24
    hi[c] = (R)hq;
    lo[c] = (R)(rel - hq);
  }
  const double hh = h[i], mm = mass[i];
  bad |= !(hh > 0.0) || !isfinite(hh) || !(mm > 0.0) || !isfinite(mm);
  double v[3];
  for (int c = 0; c < 3; ++c) { v[c] = vel[3 * (int64_t)i + c]; bad |= !isfinite(v[c]); }
  P[s] = Vec<R>::make(hi[0], hi[1], hi[2], (R)hh);
  Lo[s] = Vec<R>::make(lo[0], lo[1], lo[2], (R)mm);
  double sig = 0.0;
  if (T != nullptr) {
    const double t = T[i], m = mu[i];
    bad |= !(t >= 0.0) || !isfinite(t) || !(m > 0.0) || !isfinite(m);
    const double s2 = rc.kT_over_mp * t / m;         // varsigma^2 [(km/s)^2]
    sig = sqrt(fmax(s2, 0.0));
    double cA, cB, kP0, e;
    gas_coeffs(rc, sig, mm, m, cA, cB, kP0, e);
    K[s] = Vec<R>::make((R)cA, (R)cB, (R)kP0, (R)e);
  }
  V[s] = Vec<R>::make((R)v[0], (R)v[1], (R)v[2], (R)sig);
  sid[s] = id[i];
  if (bad) atomicOr(status, DMB_BAD_VALUE);
}

template <typename R>
cudaError_t launch_gather(const double *pos, const double *vel, const double *mass, const double *h,
                          const double *T, const double *mu, const uint32_t *id, int64_t n, const uint32_t *perm,
                          int periodic, const double box[3], const Frame *frame, RunConst rc, BatchArgs ba,
                          typename Vec<R>::v4 *P, typename Vec<R>::v4 *L, typename Vec<R>::v4 *V,
                          typename Vec<R>::v4 *K, uint32_t *sid, uint16_t *bid, uint32_t *status, cudaStream_t s,
                          int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  k_gather<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, vel, mass, h, T, mu, id, n, perm, periodic, box[0],
                                                          box[1], box[2], frame, rc, ba, P, L, V, K, sid, bid,
                                                          status);
  if (launches) *launches += 1;
  return cudaGetLastError();
}
template cudaError_t launch_gather<float>(const double *, const double *, const double *, const double *,
                                          const double *, const double *, const uint32_t *, int64_t,
                                          const uint32_t *, int, const double *, const Frame *, RunConst, BatchArgs,
                                          float4 *, float4 *, float4 *, float4 *, uint32_t *, uint16_t *, uint32_t *,
                                          cudaStream_t, int64_t *);
template cudaError_t launch_gather<double>(const double *, const double *, const double *, const double *,
                                           const double *, const double *, const uint32_t *, int64_t,
                                           const uint32_t *, int, const double *, const Frame *, RunConst, BatchArgs,
                                           double4_32a *, double4_32a *, double4_32a *, double4_32a *, uint32_t *,
                                           uint16_t *, uint32_t *, cudaStream_t, int64_t *);

// ---- chunk tree ------------------------------------------------------------------------
// Leaves hold DMB_LEAF consecutive sorted particles; every inner node groups 32 consecutive
// nodes of the level below.  Boxes are float with a conservative pad; bmin.w = h_max.
int tree_layout(int64_t n, int *levels, int off[DMB_MAX_LEVELS], int cnt[DMB_MAX_LEVELS]) {
  int64_t c = (n + DMB_LEAF - 1) / DMB_LEAF;
  if (c < 1) c = 1;
  int l = 0, total = 0;
  while (true) {
    off[l] = total;
    cnt[l] = (int)c;
    total += (int)c;
    ++l;
    if (c == 1 || l == DMB_MAX_LEVELS) break;
    c = (c + 31) / 32;
  }
  *levels = l;
  return total;
}

template <typename R>
__global__ void k_tree_leaves(const typename Vec<R>::v4 *__restrict__ P, const typename Vec<R>::v4 *__restrict__ L,
                              int64_t n, int nleaf, const Frame *__restrict__ frame, float4 *__restrict__ bmin,
                              float4 *__restrict__ bmax, const uint16_t *__restrict__ bid, int2 *__restrict__ leaf_box) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  if (warp >= nleaf) return;
  const int64_t i = warp * DMB_LEAF + lane;
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  float hm = -INFINITY;
  if (i < n) {
    const typename Vec<R>::v4 p = P[i], l = L[i];
    const float c[3] = {(float)((double)p.x + (double)l.x), (float)((double)p.y + (double)l.y),
                        (float)((double)p.z + (double)l.z)};
    for (int k = 0; k < 3; ++k) { mn[k] = c[k]; mx[k] = c[k]; }
    hm = (float)p.w;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    for (int k = 0; k < 3; ++k) {
      mn[k] = fminf(mn[k], __shfl_xor_sync(DMB_FULL, mn[k], o));
      mx[k] = fmaxf(mx[k], __shfl_xor_sync(DMB_FULL, mx[k], o));
    }
    hm = fmaxf(hm, __shfl_xor_sync(DMB_FULL, hm, o));
  }
  if (bid != nullptr) {
    int b0 = i < n ? (int)bid[i] : 0x7fffffff, b1 = i < n ? (int)bid[i] : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      b0 = min(b0, __shfl_xor_sync(DMB_FULL, b0, o));
      b1 = max(b1, __shfl_xor_sync(DMB_FULL, b1, o));
    }
    if (lane == 0) leaf_box[warp] = make_int2(b1 >= 0 ? b0 : 0, b1 >= 0 ? b1 : 0);
  }
  if (lane == 0) {
    const float pad = frame->pad;
    if (hm > -INFINITY) {
      bmin[warp] = make_float4(mn[0] - pad, mn[1] - pad, mn[2] - pad, hm * (1.0f + 1e-6f));
      bmax[warp] = make_float4(mx[0] + pad, mx[1] + pad, mx[2] + pad, 0.0f);
    } else {
      bmin[warp] = make_float4(INFINITY, INFINITY, INFINITY, -INFINITY);
      bmax[warp] = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.0f);
    }
  }
}

// one warp per parent: union of its (up to) 32 children
__global__ void k_tree_level(float4 *__restrict__ bmin, float4 *__restrict__ bmax, int child_off, int child_cnt,
                             int par_off, int par_cnt) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  if (warp >= par_cnt) return;
  const int64_t c = warp * 32 + lane;
  float4 a = make_float4(INFINITY, INFINITY, INFINITY, -INFINITY), b = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.0f);
  if (c < child_cnt) { a = bmin[child_off + c]; b = bmax[child_off + c]; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a.x = fminf(a.x, __shfl_xor_sync(DMB_FULL, a.x, o));
    a.y = fminf(a.y, __shfl_xor_sync(DMB_FULL, a.y, o));
    a.z = fminf(a.z, __shfl_xor_sync(DMB_FULL, a.z, o));
    a.w = fmaxf(a.w, __shfl_xor_sync(DMB_FULL, a.w, o));
    b.x = fmaxf(b.x, __shfl_xor_sync(DMB_FULL, b.x, o));
    b.y = fmaxf(b.y, __shfl_xor_sync(DMB_FULL, b.y, o));
    b.z = fmaxf(b.z, __shfl_xor_sync(DMB_FULL, b.z, o));
  }
  if (lane == 0) {
    bmin[par_off + warp] = a;
    bmax[par_off + warp] = make_float4(b.x, b.y, b.z, 0.0f);
  }
}

template <typename R>
cudaError_t launch_tree(const typename Vec<R>::v4 *P, const typename Vec<R>::v4 *L, int64_t n, const Frame *frame,
                        float4 *bmin, float4 *bmax, int levels, const int *off, const int *cnt, const uint16_t *bid,
                        int2 *leaf_box, cudaStream_t s, int64_t *launches) {
  const int64_t t0 = (int64_t)cnt[0] * 32;
  k_tree_leaves<R><<<(unsigned)((t0 + 255) / 256), 256, 0, s>>>(P, L, n, cnt[0], frame, bmin + off[0], bmax + off[0],
                                                                 bid, leaf_box);
  if (launches) *launches += 1;
  for (int l = 1; l < levels; ++l) {
    const int64_t t = (int64_t)cnt[l] * 32;
    k_tree_level<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(bmin, bmax, off[l - 1], cnt[l - 1], off[l], cnt[l]);
    if (launches) *launches += 1;
  }
  return cudaGetLastError();
}
template cudaError_t launch_tree<float>(const float4 *, const float4 *, int64_t, const Frame *, float4 *, float4 *,
                                        int, const int *, const int *, const uint16_t *, int2 *, cudaStream_t,
                                        int64_t *);
template cudaError_t launch_tree<double>(const double4_32a *, const double4_32a *, int64_t, const Frame *, float4 *,
                                         float4 *, int, const int *, const int *, const uint16_t *, int2 *,
                                         cudaStream_t, int64_t *);
