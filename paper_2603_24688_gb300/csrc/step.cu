// Gas kicks (V_j += a_j dt, u_j += du_j/dt dt clamped at 0) and deterministic float64 sums.
#include "step.cuh"

__global__ void __launch_bounds__(KICK_THREADS)
k_kick_gas(double *__restrict__ vel, double *__restrict__ T, const double *__restrict__ mu,
           const double *__restrict__ mass, const double *__restrict__ acc, const double *__restrict__ dudt,
           const double *__restrict__ e_exp, int64_t n, double dt, double kT_over_mp, double *__restrict__ out,
           const uint32_t *__restrict__ gate) {
  __shared__ double red[KICK_NSUM][KICK_THREADS];
  double s[KICK_NSUM] = {0, 0, 0, 0, 0, 0};
  // a captured step whose lists overflowed kicks nothing (the host repeats the step)
  const int64_t nk = (gate != nullptr && *gate != 0u) ? 0 : n;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nk; c += (int64_t)gridDim.x * blockDim.x) {
    const double M = mass[c];
    double V[3], Vn[3];
    for (int k = 0; k < 3; ++k) {
      V[k] = vel[3 * c + k];
      Vn[k] = V[k] + acc[3 * c + k] * dt;
      vel[3 * c + k] = Vn[k];
      s[k] += M * acc[3 * c + k] * dt;
    }
    const double m = mu[c];
    const double u0 = 1.5 * kT_over_mp * T[c] / m;       // u = (3/2) k_B T / mu
    double u1 = u0 + dudt[c] * dt;
    if (u1 < 0.0) { u1 = 0.0; s[4] += 1.0; }
    T[c] = u1 * m / (1.5 * kT_over_mp);
    s[3] += M * (0.5 * ((Vn[0] * Vn[0] + Vn[1] * Vn[1] + Vn[2] * Vn[2]) - (V[0] * V[0] + V[1] * V[1] + V[2] * V[2])) +
                 (u1 - u0));
    if (e_exp) s[5] += e_exp[c] * dt;   // e_exp is in sorted order; the total does not depend on it
  }
  for (int k = 0; k < KICK_NSUM; ++k) red[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int o = KICK_THREADS / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int k = 0; k < KICK_NSUM; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < KICK_NSUM) out[KICK_NSUM * (int64_t)blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

cudaError_t launch_kick_gas(double *vel, double *T, const double *mu, const double *mass, const double *acc,
                            const double *dudt, const double *e_exp, int64_t n, double dt, double kT_over_mp,
                            double *block_sums, int blocks, cudaStream_t s, int64_t *launches,
                            const uint32_t *gate) {
  k_kick_gas<<<blocks, KICK_THREADS, 0, s>>>(vel, T, mu, mass, acc, dudt, e_exp, n, dt, kT_over_mp, block_sums, gate);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

// one block: every thread sums a fixed strided subset of the partials, then a fixed tree
__global__ void __launch_bounds__(256)
k_final_sums(const double *__restrict__ mcb, const double *__restrict__ mcm, int mc_nb,
             const double *__restrict__ kb, int k_nb, double dt, double n_pairs, double *sums,
             const int64_t *__restrict__ n_pairs_dev) {
  __shared__ double red[8 + KICK_NSUM + 1][256];
  const int t = threadIdx.x;
  double m[8] = {0, 0, 0, 0, 0, 0, 0, 0}, k[KICK_NSUM] = {0, 0, 0, 0, 0, 0}, mx = 0.0;
  for (int b = t; b < mc_nb; b += 256) {
    for (int c = 0; c < 8; ++c) m[c] += mcb[8 * b + c];
    mx = fmax(mx, mcm[b]);
  }
  for (int b = t; b < k_nb; b += 256)
    for (int c = 0; c < KICK_NSUM; ++c) k[c] += kb[KICK_NSUM * b + c];
  for (int c = 0; c < 8; ++c) red[c][t] = m[c];
  for (int c = 0; c < KICK_NSUM; ++c) red[8 + c][t] = k[c];
  red[8 + KICK_NSUM][t] = mx;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) {
      for (int c = 0; c < 8 + KICK_NSUM; ++c) red[c][t] += red[c][t + o];
      red[8 + KICK_NSUM][t] = fmax(red[8 + KICK_NSUM][t], red[8 + KICK_NSUM][t + o]);
    }
    __syncthreads();
  }
  if (t == 0) {
    const double *M = &red[0][0];
    sums[0] = red[0][0];
    sums[1] = red[1][0];
    sums[2] = red[2][0];
    sums[3] = red[8][0];
    sums[4] = red[9][0];
    sums[5] = red[10][0];
    sums[6] = red[3][0];
    sums[7] = red[11][0];
    sums[8] = red[13][0];
    sums[9] = red[4][0];
    sums[10] = red[5][0];
    sums[11] = red[12][0];
    sums[12] = n_pairs_dev != nullptr ? (double)*n_pairs_dev : n_pairs;
    sums[13] = red[7][0];
    sums[14] = red[8 + KICK_NSUM][0];
    sums[15] = red[6][0];
    (void)M;
  }
}

cudaError_t launch_final_sums(const double *mc_blocks, const double *mc_max, int mc_nb, const double *kick_blocks,
                              int kick_nb, double dt, double n_pairs, double *sums, cudaStream_t s,
                              int64_t *launches, const int64_t *n_pairs_dev) {
  k_final_sums<<<1, 256, 0, s>>>(mc_blocks, mc_max, mc_nb, kick_blocks, kick_nb, dt, n_pairs, sums, n_pairs_dev);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

// pairs as (DM caller index, gas caller index), gas-major
__global__ void k_pairs_out(const int64_t *__restrict__ row_ptr, const uint32_t *__restrict__ rows,
                            const uint32_t *__restrict__ gperm, const uint32_t *__restrict__ dperm, int64_t ng,
                            int64_t cap, uint32_t *__restrict__ out) {
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  if (j >= ng) return;
  const int64_t rs = row_ptr[j], re = row_ptr[j + 1];
  const uint32_t gj = gperm[j];
  for (int64_t p = rs + lane; p < re && p < cap; p += 32) {
    out[2 * p] = dperm[rows[p]];
    out[2 * p + 1] = gj;
  }
}

cudaError_t launch_pairs_out(const int64_t *row_ptr, const uint32_t *rows, const uint32_t *gas_perm,
                             const uint32_t *dm_perm, int64_t ng, int64_t capacity, uint32_t *out, cudaStream_t s,
                             int64_t *launches) {
  if (ng <= 0 || capacity <= 0) return cudaSuccess;
  k_pairs_out<<<(unsigned)((ng * 32 + 255) / 256), 256, 0, s>>>(row_ptr, rows, gas_perm, dm_perm, ng, capacity, out);
  if (launches) *launches += 1;
  return cudaGetLastError();
}
