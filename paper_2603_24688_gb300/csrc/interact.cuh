// Shared parts of the pair-physics kernels (mean field, Monte Carlo, fused pass): the pair
// probability of Eq. dm-update-prob, the decision-band helpers and the two float64 finishes.
#pragma once
#include "mlp.cuh"
#include "pairs.cuh"
#include "physics.cuh"

#define MF_WARPS 8
#define MC_WARPS 8

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

// float64 side of the Monte Carlo, one thread per DM particle: new velocities in caller
// order and deterministic block partials of the step sums
static __global__ void __launch_bounds__(256)
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
