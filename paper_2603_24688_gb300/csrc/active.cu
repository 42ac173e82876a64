// Active sets of hierarchical substeps (bin ordering, per-prefix tables) and the kick of the
// active gas.
#include "active.cuh"
#include "step.cuh"

__global__ void k_bin_keys(const uint8_t *__restrict__ bin, const uint32_t *__restrict__ perm, int64_t n,
                           uint64_t *__restrict__ keys, uint32_t *__restrict__ vals, uint32_t *status) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t b = bin[perm[s]];
  if (b >= DMB_NBINS) atomicOr(status, DMB_BAD_VALUE);
  keys[s] = b < DMB_NBINS ? b : DMB_NBINS - 1;
  vals[s] = (uint32_t)s;
}

cudaError_t launch_bin_keys(const uint8_t *bin, const uint32_t *perm, int64_t n, uint64_t *keys, uint32_t *vals,
                            uint32_t *status, cudaStream_t s, int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  k_bin_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(bin, perm, n, keys, vals, status);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

// thread s in [0, n]: the bins b in (key[s-1], key[s]] start at s (key[-1] = -1, key[n] = 64)
__global__ void k_bin_bounds(const uint64_t *__restrict__ keys, int64_t n, int64_t *__restrict__ start) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s > n) return;
  const int kprev = s > 0 ? (int)keys[s - 1] : -1;
  const int kcur = s < n ? (int)keys[s] : DMB_NBINS;
  for (int b = kprev + 1; b <= kcur; ++b) start[b] = s;
}

cudaError_t launch_bin_bounds(const uint64_t *keys, int64_t n, int64_t *start, cudaStream_t s, int64_t *launches) {
  k_bin_bounds<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(keys, n, start);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

__global__ void k_list_counts(const uint32_t *__restrict__ list, int64_t n, const int64_t *__restrict__ row_ptr,
                              int seg, uint32_t *__restrict__ len, uint32_t *__restrict__ segs) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t j = list[k];
  const int64_t l = row_ptr[j + 1] - row_ptr[j];
  len[k] = (uint32_t)l;
  if (seg > 0) segs[k] = (uint32_t)((l + seg - 1) / seg);
}

cudaError_t launch_list_counts(const uint32_t *list, int64_t n, const int64_t *row_ptr, int seg, uint32_t *len,
                               uint32_t *segs, cudaStream_t s, int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  k_list_counts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(list, n, row_ptr, seg, len, segs);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

__global__ void k_list_seg_map(const uint32_t *__restrict__ list, int64_t n, const int64_t *__restrict__ row_ptr,
                               const int64_t *__restrict__ seg_ptr, int seg, uint32_t *__restrict__ seg_row,
                               int64_t *__restrict__ seg_begin) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t j = list[k];
  for (int64_t u = seg_ptr[k]; u < seg_ptr[k + 1]; ++u) {
    seg_row[u] = j;
    seg_begin[u] = row_ptr[j] + (u - seg_ptr[k]) * seg;
  }
}

cudaError_t launch_list_seg_map(const uint32_t *list, int64_t n, const int64_t *row_ptr, const int64_t *seg_ptr,
                                int seg, uint32_t *seg_row, int64_t *seg_begin, cudaStream_t s, int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  k_list_seg_map<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(list, n, row_ptr, seg_ptr, seg, seg_row, seg_begin);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

__global__ void k_pick(const int64_t *__restrict__ arr, const int64_t *__restrict__ start, int64_t *__restrict__ out) {
  const int b = threadIdx.x;
  if (b <= DMB_NBINS) out[b] = arr[start[b]];
}

cudaError_t launch_pick(const int64_t *arr, const int64_t *start, int64_t *out, cudaStream_t s, int64_t *launches) {
  k_pick<<<1, 96, 0, s>>>(arr, start, out);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

__global__ void k_step_set(unsigned long long *step, unsigned long long value, int advance) {
  if (threadIdx.x == 0) *step = advance ? *step + 1ull : value;
}

cudaError_t launch_step_set(unsigned long long *step, unsigned long long value, cudaStream_t s, int64_t *launches) {
  k_step_set<<<1, 32, 0, s>>>(step, value, 0);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_step_advance(unsigned long long *step, cudaStream_t s, int64_t *launches) {
  k_step_set<<<1, 32, 0, s>>>(step, 0ull, 1);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

template <typename R>
__global__ void __launch_bounds__(KICK_THREADS)
k_kick_gas_list(double *__restrict__ vel, double *__restrict__ T, const double *__restrict__ mu,
                const double *__restrict__ mass, const double *__restrict__ acc, const double *__restrict__ dudt,
                const double *__restrict__ e_exp, const uint32_t *__restrict__ list, int64_t n_list,
                const uint32_t *__restrict__ perm, const uint8_t *__restrict__ bin, double dt_min, RunConst rc,
                typename Vec<R>::v4 *__restrict__ Vs, typename Vec<R>::v4 *__restrict__ Ks, double *__restrict__ out) {
  __shared__ double red[KICK_NSUM][KICK_THREADS];
  double s[KICK_NSUM] = {0, 0, 0, 0, 0, 0};
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_list; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t j = list[k];
    const int64_t c = perm[j];
    const double dt = ldexp(dt_min, (int)bin[c]);
    const double M = mass[c];
    double V[3], Vn[3];
    for (int q = 0; q < 3; ++q) {
      V[q] = vel[3 * c + q];
      Vn[q] = V[q] + acc[3 * c + q] * dt;
      vel[3 * c + q] = Vn[q];
      s[q] += M * acc[3 * c + q] * dt;
    }
    const double m = mu[c];
    const double u0 = 1.5 * rc.kT_over_mp * T[c] / m;       // u = (3/2) k_B T / mu
    double u1 = u0 + dudt[c] * dt;
    if (u1 < 0.0) { u1 = 0.0; s[4] += 1.0; }
    const double Tn = u1 * m / (1.5 * rc.kT_over_mp);
    T[c] = Tn;
    s[3] += M * (0.5 * ((Vn[0] * Vn[0] + Vn[1] * Vn[1] + Vn[2] * Vn[2]) - (V[0] * V[0] + V[1] * V[1] + V[2] * V[2])) +
                 (u1 - u0));
    if (e_exp) s[5] += e_exp[j] * dt;
    // refreshed sorted copies, as the gather forms them
    const double sig = sqrt(fmax(rc.kT_over_mp * Tn / m, 0.0));
    double cA, cB, kP0, e;
    gas_coeffs(rc, sig, M, m, cA, cB, kP0, e);
    Vs[j] = Vec<R>::make((R)Vn[0], (R)Vn[1], (R)Vn[2], (R)sig);
    Ks[j] = Vec<R>::make((R)cA, (R)cB, (R)kP0, (R)e);
  }
  for (int q = 0; q < KICK_NSUM; ++q) red[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int o = KICK_THREADS / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int q = 0; q < KICK_NSUM; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < KICK_NSUM) out[KICK_NSUM * (int64_t)blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

template <typename R>
cudaError_t launch_kick_gas_list(double *vel, double *T, const double *mu, const double *mass, const double *acc,
                                 const double *dudt, const double *e_exp, const uint32_t *list, int64_t n_list,
                                 const uint32_t *perm, const uint8_t *bin, double dt_min, RunConst rc,
                                 typename Vec<R>::v4 *Vs, typename Vec<R>::v4 *Ks, double *block_sums, int blocks,
                                 cudaStream_t s, int64_t *launches) {
  k_kick_gas_list<R><<<blocks, KICK_THREADS, 0, s>>>(vel, T, mu, mass, acc, dudt, e_exp, list, n_list, perm, bin,
                                                     dt_min, rc, Vs, Ks, block_sums);
  if (launches) *launches += 1;
  return cudaGetLastError();
}
template cudaError_t launch_kick_gas_list<float>(double *, double *, const double *, const double *, const double *,
                                                 const double *, const double *, const uint32_t *, int64_t,
                                                 const uint32_t *, const uint8_t *, double, RunConst, float4 *,
                                                 float4 *, double *, int, cudaStream_t, int64_t *);
template cudaError_t launch_kick_gas_list<double>(double *, double *, const double *, const double *, const double *,
                                                  const double *, const double *, const uint32_t *, int64_t,
                                                  const uint32_t *, const uint8_t *, double, RunConst, double4_32a *,
                                                  double4_32a *, double *, int, cudaStream_t, int64_t *);

// A particle whose criterion ratio x = max_j P_ij / cap_j exceeds 1 (or is not finite) moves to
// the largest bin b' <= b with x 2^(b' - b) <= 1 (P_ij is proportional to dt): with x = m 2^e,
// m in [1/2, 1), k = ceil(log2 x) is e, or e - 1 when m = 1/2.  One with x < 1/4 moves up one
// bin when the next substep is a multiple of 2^(b+1) and b < max_bin.  Decisions are integer
// functions of the float ratio, so they are exact.
__global__ void k_rebin(const float *__restrict__ ratio, uint8_t *__restrict__ bin, int64_t n, int max_bin,
                        unsigned long long substep, const uint8_t *__restrict__ active,
                        unsigned long long *__restrict__ changed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool moved = false;
  if (i < n && (active == nullptr || active[i] != 0)) {
    const float x = ratio[i];
    const int b = bin[i];
    int nb = b;
    if (!isfinite(x)) {
      nb = 0;
    } else if (x > 1.0f) {
      int e;
      const float m = frexpf(x, &e);
      const int k = m == 0.5f ? e - 1 : e;
      nb = b - k < 0 ? 0 : b - k;
    } else if (x < 0.25f && b < max_bin && (substep & ((2ull << b) - 1ull)) == 0ull) {
      nb = b + 1;
    }
    if (nb != b) {
      bin[i] = (uint8_t)nb;
      moved = true;
    }
  }
  const unsigned m = __ballot_sync(DMB_FULL, moved);
  if ((threadIdx.x & 31u) == 0u && m != 0u) atomicAdd(changed, (unsigned long long)__popc(m));
}

cudaError_t launch_rebin(const float *ratio, uint8_t *bin, int64_t n, int max_bin, unsigned long long substep,
                         const uint8_t *active, unsigned long long *changed, cudaStream_t s, int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  k_rebin<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ratio, bin, n, max_bin, substep, active, changed);
  if (launches) *launches += 1;
  return cudaGetLastError();
}
