// Training and inference of the rate surrogate on the GPU: data from the device quadrature,
// forward / backward / weight-gradient kernels (bf16 tensor cores for the 128 x 128 layers),
// Adam, and a batched inference kernel.
#include <math.h>

#include <algorithm>
#include <random>
#include <vector>

#include "mlp.cuh"
#include "mlp_host.cuh"
#include "physics.cuh"

#define MLP_WARPS 4

// ---- parameter images ------------------------------------------------------------------------
// Device copies used by the kernels: float32 master parameters, bf16 W2/W3 (row-major
// [out][in]) and their transposes (row-major [in][out]) for the backward pass.
__global__ void k_mlp_refresh(const float *__restrict__ p, __nv_bfloat16 *__restrict__ w2, __nv_bfloat16 *__restrict__ w3,
                              __nv_bfloat16 *__restrict__ w2t, __nv_bfloat16 *__restrict__ w3t) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= MLP_H * MLP_H) return;
  const int o = t / MLP_H, i = t % MLP_H;
  w2[t] = __float2bfloat16_rn(p[MLP_OFF_W2 + t]);
  w3[t] = __float2bfloat16_rn(p[MLP_OFF_W3 + t]);
  w2t[i * MLP_H + o] = __float2bfloat16_rn(p[MLP_OFF_W2 + t]);
  w3t[i * MLP_H + o] = __float2bfloat16_rn(p[MLP_OFF_W3 + t]);
}

// copy the network into shared memory (W2/W3 from the given bf16 arrays: forward or transposed)
__device__ void mlp_load_smem(MlpSmem &M, const float *__restrict__ p, const __nv_bfloat16 *__restrict__ w2,
                              const __nv_bfloat16 *__restrict__ w3) {
  for (int t = threadIdx.x; t < MLP_H * MLP_H / 8; t += blockDim.x) {
    reinterpret_cast<uint4 *>(M.W2)[t] = reinterpret_cast<const uint4 *>(w2)[t];
    reinterpret_cast<uint4 *>(M.W3)[t] = reinterpret_cast<const uint4 *>(w3)[t];
  }
  for (int t = threadIdx.x; t < MLP_H * MLP_IN; t += blockDim.x) M.W1[t] = p[MLP_OFF_W1 + t];
  for (int t = threadIdx.x; t < MLP_H; t += blockDim.x) {
    M.b1[t] = p[MLP_OFF_B1 + t];
    M.b2[t] = p[MLP_OFF_B2 + t];
    M.b3[t] = p[MLP_OFF_B3 + t];
  }
  for (int t = threadIdx.x; t < MLP_OUT * MLP_H; t += blockDim.x) M.W4[t] = p[MLP_OFF_W4 + t];
  if (threadIdx.x < MLP_OUT) M.b4[threadIdx.x] = p[MLP_OFF_B4 + threadIdx.x];
  __syncthreads();
}

// ---- training data: samples of the normalised integrals from the float64 quadrature -----------
__global__ void k_mlp_data(int64_t N, unsigned long long seed, MlpDataSpec spec, float *__restrict__ X,
                           float *__restrict__ Y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint4 w = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0x5eedu, 0x4d4c5000u), (uint32_t)seed,
                                (uint32_t)(seed >> 32));
  const double u0 = uniform23<double>(w.x), u1 = uniform23<double>(w.y), u2 = uniform23<double>(w.z);
  const int k = (int)(w.w % (uint32_t)spec.n_count);
  const double ls = spec.log_s_lo + (spec.log_s_hi - spec.log_s_lo) * u0;
  const double lt = spec.log_tau_lo + (spec.log_tau_hi - spec.log_tau_lo) * u1;
  const double lm = spec.log_m_lo + (spec.log_m_hi - spec.log_m_lo) * u2;
  const int n = spec.n_values[k];
  const double s = pow(10.0, ls), x = 0.5 * s * s;
  const double q = spec.scr ? pow(10.0, lt) : 0.0;      // screened law: tau = varsigma^2 / v_c^2
  double FA, FB;
  rates_quad<double>(x, n, spec.alpha[k], FA, FB, q);
  const double ls2 = spec.scr ? 2.0 * log1p(q * (2.0 * x + 3.0)) : 0.0;
  X[4 * i + 0] = (float)(0.5 * ls);
  X[4 * i + 1] = (float)(0.5 * lt);
  X[4 * i + 2] = (float)lm;
  X[4 * i + 3] = (float)(0.25 * n);
  const double *eA = spec.envA[k], *eB = spec.envB[k];
  Y[2 * i + 0] = (float)(log(FA) - eA[3] * log1p(x * (eA[0] + x * (eA[1] + x * eA[2]))) + ls2);
  Y[2 * i + 1] = (float)(log(FB) - eB[3] * log1p(x * (eB[0] + x * (eB[1] + x * eB[2]))) + ls2);
}

// ---- training forward: 16-row tiles per warp, intermediates stored for the backward pass ----
struct MlpTrainBufs {
  const float *X, *Y;            // [N][4], [N][2]
  const int *idx;                // [B] sample indices of the batch
  int B;
  __nv_bfloat16 *A1, *A2;        // [B][H] activations fed to the tensor cores
  float *Z1, *Z2, *Z3, *A3;      // [B][H]
  float *dY;                     // [B][2]
  float *loss;                   // [blocks] partial sums of the squared error
  __nv_bfloat16 *dZ3, *dZ2;      // [B][H]
  float *dZ1;                    // [B][H]
};

__global__ void __launch_bounds__(MLP_WARPS * 32)
k_mlp_forward_train(const float *__restrict__ p, const __nv_bfloat16 *__restrict__ w2,
                    const __nv_bfloat16 *__restrict__ w3, MlpTrainBufs tb) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MlpSmem &M = *reinterpret_cast<MlpSmem *>(smraw);
  __shared__ float red[MLP_WARPS];
  mlp_load_smem(M, p, w2, w3);
  const unsigned lane = threadIdx.x & 31u, g = lane >> 2, tig = lane & 3u;
  const int warp = threadIdx.x >> 5;
  float lsum = 0.0f;
  const int tiles = (tb.B + 15) / 16;
  for (int tile = blockIdx.x * MLP_WARPS + warp; tile < tiles; tile += gridDim.x * MLP_WARPS) {
    const int r0 = tile * 16 + g, r1 = r0 + 8;
    const bool v0 = r0 < tb.B, v1 = r1 < tb.B;
    const int s0 = v0 ? tb.idx[r0] : 0, s1 = v1 ? tb.idx[r1] : 0;
    float xl[MLP_IN], xh[MLP_IN];
    for (int m = 0; m < MLP_IN; ++m) { xl[m] = tb.X[4 * s0 + m]; xh[m] = tb.X[4 * s1 + m]; }
    float acc[16][4];
    uint32_t af[8][4];
    for (int nt = 0; nt < 16; ++nt)
      for (int e = 0; e < 2; ++e) {
        const int col = nt * 8 + tig * 2 + e;
        float zl = M.b1[col], zh = M.b1[col];
        for (int m = 0; m < MLP_IN; ++m) { zl += M.W1[col * MLP_IN + m] * xl[m]; zh += M.W1[col * MLP_IN + m] * xh[m]; }
        acc[nt][e] = zl;
        acc[nt][2 + e] = zh;
      }
    // store z1, then activate and pack (bias already added: pass a zero bias)
    for (int nt = 0; nt < 16; ++nt)
      for (int e = 0; e < 2; ++e) {
        const int col = nt * 8 + tig * 2 + e;
        if (v0) tb.Z1[r0 * MLP_H + col] = acc[nt][e];
        if (v1) tb.Z1[r1 * MLP_H + col] = acc[nt][2 + e];
      }
    for (int nt = 0; nt < 16; ++nt)
      for (int e = 0; e < 4; ++e) acc[nt][e] = mlp_act(acc[nt][e]);
    for (int kt = 0; kt < 8; ++kt) {
      af[kt][0] = pack_bf16(acc[2 * kt][0], acc[2 * kt][1]);
      af[kt][1] = pack_bf16(acc[2 * kt][2], acc[2 * kt][3]);
      af[kt][2] = pack_bf16(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
      af[kt][3] = pack_bf16(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
    }
    for (int kt = 0; kt < 8; ++kt) {   // A1 (bf16, exactly what the tensor cores see)
      const int c0 = kt * 16 + tig * 2;
      if (v0) { *reinterpret_cast<uint32_t *>(&tb.A1[r0 * MLP_H + c0]) = af[kt][0]; *reinterpret_cast<uint32_t *>(&tb.A1[r0 * MLP_H + c0 + 8]) = af[kt][2]; }
      if (v1) { *reinterpret_cast<uint32_t *>(&tb.A1[r1 * MLP_H + c0]) = af[kt][1]; *reinterpret_cast<uint32_t *>(&tb.A1[r1 * MLP_H + c0 + 8]) = af[kt][3]; }
    }
    // layer 2
    mlp_layer_mma(M.W2, af, acc);
    for (int nt = 0; nt < 16; ++nt)
      for (int e = 0; e < 2; ++e) {
        const int col = nt * 8 + tig * 2 + e;
        acc[nt][e] += M.b2[col];
        acc[nt][2 + e] += M.b2[col];
        if (v0) tb.Z2[r0 * MLP_H + col] = acc[nt][e];
        if (v1) tb.Z2[r1 * MLP_H + col] = acc[nt][2 + e];
      }
    for (int nt = 0; nt < 16; ++nt)
      for (int e = 0; e < 4; ++e) acc[nt][e] = mlp_act(acc[nt][e]);
    for (int kt = 0; kt < 8; ++kt) {
      af[kt][0] = pack_bf16(acc[2 * kt][0], acc[2 * kt][1]);
      af[kt][1] = pack_bf16(acc[2 * kt][2], acc[2 * kt][3]);
      af[kt][2] = pack_bf16(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
      af[kt][3] = pack_bf16(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
      const int c0 = kt * 16 + tig * 2;
      if (v0) { *reinterpret_cast<uint32_t *>(&tb.A2[r0 * MLP_H + c0]) = af[kt][0]; *reinterpret_cast<uint32_t *>(&tb.A2[r0 * MLP_H + c0 + 8]) = af[kt][2]; }
      if (v1) { *reinterpret_cast<uint32_t *>(&tb.A2[r1 * MLP_H + c0]) = af[kt][1]; *reinterpret_cast<uint32_t *>(&tb.A2[r1 * MLP_H + c0 + 8]) = af[kt][3]; }
    }
    // layer 3 and the output layer
    mlp_layer_mma(M.W3, af, acc);
    float pl[MLP_OUT] = {0.f, 0.f}, ph[MLP_OUT] = {0.f, 0.f};
    for (int nt = 0; nt < 16; ++nt)
      for (int e = 0; e < 2; ++e) {
        const int col = nt * 8 + tig * 2 + e;
        const float zl = acc[nt][e] + M.b3[col], zh = acc[nt][2 + e] + M.b3[col];
        const float al = mlp_act(zl), ah = mlp_act(zh);
        if (v0) { tb.Z3[r0 * MLP_H + col] = zl; tb.A3[r0 * MLP_H + col] = al; }
        if (v1) { tb.Z3[r1 * MLP_H + col] = zh; tb.A3[r1 * MLP_H + col] = ah; }
        for (int o = 0; o < MLP_OUT; ++o) { pl[o] += M.W4[o * MLP_H + col] * al; ph[o] += M.W4[o * MLP_H + col] * ah; }
      }
    for (int o = 0; o < MLP_OUT; ++o) {
      pl[o] += __shfl_xor_sync(DMB_FULL, pl[o], 1);
      pl[o] += __shfl_xor_sync(DMB_FULL, pl[o], 2);
      ph[o] += __shfl_xor_sync(DMB_FULL, ph[o], 1);
      ph[o] += __shfl_xor_sync(DMB_FULL, ph[o], 2);
    }
    if (tig == 0) {
      const float invB = 1.0f / (float)tb.B;
      for (int o = 0; o < MLP_OUT; ++o) {
        if (v0) { const float d = pl[o] + M.b4[o] - tb.Y[2 * s0 + o]; tb.dY[2 * r0 + o] = 2.0f * d * invB; lsum += d * d; }
        if (v1) { const float d = ph[o] + M.b4[o] - tb.Y[2 * s1 + o]; tb.dY[2 * r1 + o] = 2.0f * d * invB; lsum += d * d; }
      }
    }
  }
  lsum = warp_sum<float>(lsum);
  if (lane == 0) red[warp] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int k = 0; k < MLP_WARPS; ++k) s += red[k];
    tb.loss[blockIdx.x] = s;
  }
}

// ---- backward through the activations: dZ3, dZ2 (bf16) and dZ1 ------------------------------
__global__ void __launch_bounds__(MLP_WARPS * 32)
k_mlp_backward(const float *__restrict__ p, const __nv_bfloat16 *__restrict__ w2t,
               const __nv_bfloat16 *__restrict__ w3t, MlpTrainBufs tb) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MlpSmem &M = *reinterpret_cast<MlpSmem *>(smraw);   // W2/W3 slots hold the transposes
  mlp_load_smem(M, p, w2t, w3t);
  const unsigned lane = threadIdx.x & 31u, g = lane >> 2, tig = lane & 3u;
  const int warp = threadIdx.x >> 5;
  const int tiles = (tb.B + 15) / 16;
  for (int tile = blockIdx.x * MLP_WARPS + warp; tile < tiles; tile += gridDim.x * MLP_WARPS) {
    const int r0 = tile * 16 + g, r1 = r0 + 8;
    const bool v0 = r0 < tb.B, v1 = r1 < tb.B;
    float dyl[MLP_OUT], dyh[MLP_OUT];
    for (int o = 0; o < MLP_OUT; ++o) { dyl[o] = v0 ? tb.dY[2 * r0 + o] : 0.f; dyh[o] = v1 ? tb.dY[2 * r1 + o] : 0.f; }
    float acc[16][4];
    uint32_t af[8][4];
    // dz3 = (W4^T dy) * act'(z3)
    for (int nt = 0; nt < 16; ++nt)
      for (int e = 0; e < 2; ++e) {
        const int col = nt * 8 + tig * 2 + e;
        float dl = 0.f, dh = 0.f;
        for (int o = 0; o < MLP_OUT; ++o) { dl += M.W4[o * MLP_H + col] * dyl[o]; dh += M.W4[o * MLP_H + col] * dyh[o]; }
        acc[nt][e] = v0 ? dl * mlp_act_grad(tb.Z3[r0 * MLP_H + col]) : 0.f;
        acc[nt][2 + e] = v1 ? dh * mlp_act_grad(tb.Z3[r1 * MLP_H + col]) : 0.f;
      }
    for (int kt = 0; kt < 8; ++kt) {
      af[kt][0] = pack_bf16(acc[2 * kt][0], acc[2 * kt][1]);
      af[kt][1] = pack_bf16(acc[2 * kt][2], acc[2 * kt][3]);
      af[kt][2] = pack_bf16(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
      af[kt][3] = pack_bf16(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
      const int c0 = kt * 16 + tig * 2;
      if (v0) { *reinterpret_cast<uint32_t *>(&tb.dZ3[r0 * MLP_H + c0]) = af[kt][0]; *reinterpret_cast<uint32_t *>(&tb.dZ3[r0 * MLP_H + c0 + 8]) = af[kt][2]; }
      if (v1) { *reinterpret_cast<uint32_t *>(&tb.dZ3[r1 * MLP_H + c0]) = af[kt][1]; *reinterpret_cast<uint32_t *>(&tb.dZ3[r1 * MLP_H + c0 + 8]) = af[kt][3]; }
    }
    // da2 = dz3 W3 (W3^T in the W3 slot), dz2 = da2 * act'(z2)
    mlp_layer_mma(M.W3, af, acc);
    for (int nt = 0; nt < 16; ++nt)
      for (int e = 0; e < 2; ++e) {
        const int col = nt * 8 + tig * 2 + e;
        acc[nt][e] = v0 ? acc[nt][e] * mlp_act_grad(tb.Z2[r0 * MLP_H + col]) : 0.f;
        acc[nt][2 + e] = v1 ? acc[nt][2 + e] * mlp_act_grad(tb.Z2[r1 * MLP_H + col]) : 0.f;
      }
    for (int kt = 0; kt < 8; ++kt) {
      af[kt][0] = pack_bf16(acc[2 * kt][0], acc[2 * kt][1]);
      af[kt][1] = pack_bf16(acc[2 * kt][2], acc[2 * kt][3]);
      af[kt][2] = pack_bf16(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
      af[kt][3] = pack_bf16(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
      const int c0 = kt * 16 + tig * 2;
      if (v0) { *reinterpret_cast<uint32_t *>(&tb.dZ2[r0 * MLP_H + c0]) = af[kt][0]; *reinterpret_cast<uint32_t *>(&tb.dZ2[r0 * MLP_H + c0 + 8]) = af[kt][2]; }
      if (v1) { *reinterpret_cast<uint32_t *>(&tb.dZ2[r1 * MLP_H + c0]) = af[kt][1]; *reinterpret_cast<uint32_t *>(&tb.dZ2[r1 * MLP_H + c0 + 8]) = af[kt][3]; }
    }
    // da1 = dz2 W2, dz1 = da1 * act'(z1)
    mlp_layer_mma(M.W2, af, acc);
    for (int nt = 0; nt < 16; ++nt)
      for (int e = 0; e < 2; ++e) {
        const int col = nt * 8 + tig * 2 + e;
        if (v0) tb.dZ1[r0 * MLP_H + col] = acc[nt][e] * mlp_act_grad(tb.Z1[r0 * MLP_H + col]);
        if (v1) tb.dZ1[r1 * MLP_H + col] = acc[nt][2 + e] * mlp_act_grad(tb.Z1[r1 * MLP_H + col]);
      }
  }
}

// ---- weight gradients of the 128 x 128 layers on the tensor cores ----------------------------
// dW[o][i] = sum_r dZ[r][o] A[r][i]: M = o, N = i, K = r.  Block (bx, by) owns a 32 x 32 block of
// dW, bz a slice of the batch; partial results go to part[bz][o][i].
__global__ void __launch_bounds__(32)
k_mlp_wgrad(const __nv_bfloat16 *__restrict__ dZ, const __nv_bfloat16 *__restrict__ A, int B, int kslices,
            float *__restrict__ part) {
  const unsigned lane = threadIdx.x & 31u, g = lane >> 2, tig = lane & 3u;
  const int o0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  const int per = ((B + kslices - 1) / kslices + 15) / 16 * 16;
  const int r_begin = blockIdx.z * per, r_end = min(B, r_begin + per);
  float acc[2][4][4];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const unsigned short *dz = reinterpret_cast<const unsigned short *>(dZ);
  const unsigned short *aa = reinterpret_cast<const unsigned short *>(A);
  for (int r = r_begin; r < r_end; r += 16) {
    auto ldz = [&](int row, int col) -> uint32_t { return row < r_end ? (uint32_t)dz[row * MLP_H + col] : 0u; };
    auto lda = [&](int row, int col) -> uint32_t { return row < r_end ? (uint32_t)aa[row * MLP_H + col] : 0u; };
    uint32_t af[2][4], bf[4][2];
    for (int mt = 0; mt < 2; ++mt) {
      const int m = o0 + mt * 16 + g;
      const int k = r + tig * 2;
      af[mt][0] = ldz(k, m) | (ldz(k + 1, m) << 16);
      af[mt][1] = ldz(k, m + 8) | (ldz(k + 1, m + 8) << 16);
      af[mt][2] = ldz(k + 8, m) | (ldz(k + 9, m) << 16);
      af[mt][3] = ldz(k + 8, m + 8) | (ldz(k + 9, m + 8) << 16);
    }
    for (int nt = 0; nt < 4; ++nt) {
      const int n = i0 + nt * 8 + g;
      const int k = r + tig * 2;
      bf[nt][0] = lda(k, n) | (lda(k + 1, n) << 16);
      bf[nt][1] = lda(k + 8, n) | (lda(k + 9, n) << 16);
    }
    for (int mt = 0; mt < 2; ++mt)
      for (int nt = 0; nt < 4; ++nt) mma_bf16_16816(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
  }
  float *out = part + (size_t)blockIdx.z * MLP_H * MLP_H;
  for (int mt = 0; mt < 2; ++mt)
    for (int nt = 0; nt < 4; ++nt) {
      const int m = o0 + mt * 16 + g, n = i0 + nt * 8 + tig * 2;
      out[m * MLP_H + n] = acc[mt][nt][0];
      out[m * MLP_H + n + 1] = acc[mt][nt][1];
      out[(m + 8) * MLP_H + n] = acc[mt][nt][2];
      out[(m + 8) * MLP_H + n + 1] = acc[mt][nt][3];
    }
}

// the small gradients (W1, all biases, W4) and the reduction of the dW2/dW3 partials:
// one thread per parameter, a fixed loop over the batch (deterministic)
__global__ void k_mlp_small_grads(MlpTrainBufs tb, const float *__restrict__ part2, const float *__restrict__ part3,
                                  int kslices, float *__restrict__ grad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= MLP_NPARAM) return;
  float s = 0.f;
  if (t < MLP_OFF_B1) {                       // W1[o][m] = sum_r dZ1[r][o] X[idx r][m]
    const int o = (t - MLP_OFF_W1) / MLP_IN, m = (t - MLP_OFF_W1) % MLP_IN;
    for (int r = 0; r < tb.B; ++r) s += tb.dZ1[r * MLP_H + o] * tb.X[4 * tb.idx[r] + m];
  } else if (t < MLP_OFF_W2) {                // b1
    const int o = t - MLP_OFF_B1;
    for (int r = 0; r < tb.B; ++r) s += tb.dZ1[r * MLP_H + o];
  } else if (t < MLP_OFF_B2) {
    for (int k = 0; k < kslices; ++k) s += part2[(size_t)k * MLP_H * MLP_H + (t - MLP_OFF_W2)];
  } else if (t < MLP_OFF_W3) {                // b2
    const int o = t - MLP_OFF_B2;
    for (int r = 0; r < tb.B; ++r) s += __bfloat162float(tb.dZ2[r * MLP_H + o]);
  } else if (t < MLP_OFF_B3) {
    for (int k = 0; k < kslices; ++k) s += part3[(size_t)k * MLP_H * MLP_H + (t - MLP_OFF_W3)];
  } else if (t < MLP_OFF_W4) {                // b3
    const int o = t - MLP_OFF_B3;
    for (int r = 0; r < tb.B; ++r) s += __bfloat162float(tb.dZ3[r * MLP_H + o]);
  } else if (t < MLP_OFF_B4) {                // W4[o][i] = sum_r dY[r][o] A3[r][i]
    const int o = (t - MLP_OFF_W4) / MLP_H, i = (t - MLP_OFF_W4) % MLP_H;
    for (int r = 0; r < tb.B; ++r) s += tb.dY[2 * r + o] * tb.A3[r * MLP_H + i];
  } else {
    const int o = t - MLP_OFF_B4;
    for (int r = 0; r < tb.B; ++r) s += tb.dY[2 * r + o];
  }
  grad[t] = s;
}

__global__ void k_mlp_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                           const float *__restrict__ grad, float lr, float b1, float b2, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= MLP_NPARAM) return;
  const float gr = grad[t];
  const float mm = b1 * m[t] + (1.0f - b1) * gr;
  const float vv = b2 * v[t] + (1.0f - b2) * gr * gr;
  m[t] = mm;
  v[t] = vv;
  p[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
}

// ---- batched inference on given inputs (validation and the debug entry point) ---------------
__global__ void __launch_bounds__(MLP_WARPS * 32)
k_mlp_infer(const float *__restrict__ p, const __nv_bfloat16 *__restrict__ w2, const __nv_bfloat16 *__restrict__ w3,
            const float *__restrict__ X, int64_t N, float *__restrict__ Yout) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MlpSmem &M = *reinterpret_cast<MlpSmem *>(smraw);
  mlp_load_smem(M, p, w2, w3);
  const unsigned lane = threadIdx.x & 31u, g = lane >> 2, tig = lane & 3u;
  const int warp = threadIdx.x >> 5;
  const int64_t tiles = (N + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * MLP_WARPS + warp; tile < tiles; tile += (int64_t)gridDim.x * MLP_WARPS) {
    const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
    float xl[MLP_IN], xh[MLP_IN], yl[MLP_OUT], yh[MLP_OUT];
    for (int m = 0; m < MLP_IN; ++m) {
      xl[m] = r0 < N ? X[4 * r0 + m] : 0.f;
      xh[m] = r1 < N ? X[4 * r1 + m] : 0.f;
    }
    mlp_forward16(M, xl, xh, yl, yh);
    if (tig == 0) {
      for (int o = 0; o < MLP_OUT; ++o) {
        if (r0 < N) Yout[2 * r0 + o] = yl[o];
        if (r1 < N) Yout[2 * r1 + o] = yh[o];
      }
    }
  }
}

// ================= host side =====================================================================
static cudaError_t set_smem_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  const int sz = (int)sizeof(MlpSmem);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_forward_train, cudaFuncAttributeMaxDynamicSharedMemorySize, sz);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, sz);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, sz);
  if (e == cudaSuccess) done = true;
  return e;
}

cudaError_t mlp_refresh(MlpDev &d, cudaStream_t s) {
  k_mlp_refresh<<<(MLP_H * MLP_H + 255) / 256, 256, 0, s>>>(d.p, d.w2, d.w3, d.w2t, d.w3t);
  return cudaGetLastError();
}

cudaError_t mlp_infer(const MlpDev &d, const float *X, int64_t N, float *Y, cudaStream_t s) {
  cudaError_t e = set_smem_attr();
  if (e != cudaSuccess || N <= 0) return e;
  int64_t blocks = ((N + 15) / 16 + MLP_WARPS - 1) / MLP_WARPS;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_mlp_infer<<<(unsigned)blocks, MLP_WARPS * 32, sizeof(MlpSmem), s>>>(d.p, d.w2, d.w3, X, N, Y);
  return cudaGetLastError();
}

cudaError_t mlp_make_data(const MlpDataSpec &spec, int64_t N, unsigned long long seed, float *X, float *Y,
                          cudaStream_t s) {
  k_mlp_data<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(N, seed, spec, X, Y);
  return cudaGetLastError();
}

cudaError_t mlp_train_batch(MlpDev &d, const float *X, const float *Y, const int *idx, int B, MlpWork &w, float lr,
                            int t_adam, cudaStream_t s, int64_t *launches) {
  cudaError_t e = set_smem_attr();
  if (e != cudaSuccess) return e;
  MlpTrainBufs tb;
  tb.X = X;
  tb.Y = Y;
  tb.idx = idx;
  tb.B = B;
  tb.A1 = w.A1;
  tb.A2 = w.A2;
  tb.Z1 = w.Z1;
  tb.Z2 = w.Z2;
  tb.Z3 = w.Z3;
  tb.A3 = w.A3;
  tb.dY = w.dY;
  tb.loss = w.loss;
  tb.dZ3 = w.dZ3;
  tb.dZ2 = w.dZ2;
  tb.dZ1 = w.dZ1;
  const int blocks = MLP_TRAIN_BLOCKS;
  k_mlp_forward_train<<<blocks, MLP_WARPS * 32, sizeof(MlpSmem), s>>>(d.p, d.w2, d.w3, tb);
  k_mlp_backward<<<blocks, MLP_WARPS * 32, sizeof(MlpSmem), s>>>(d.p, d.w2t, d.w3t, tb);
  const dim3 gg(MLP_H / 32, MLP_H / 32, MLP_KSLICES);
  k_mlp_wgrad<<<gg, 32, 0, s>>>(w.dZ2, w.A1, B, MLP_KSLICES, w.part2);
  k_mlp_wgrad<<<gg, 32, 0, s>>>(w.dZ3, w.A2, B, MLP_KSLICES, w.part3);
  k_mlp_small_grads<<<(MLP_NPARAM + 127) / 128, 128, 0, s>>>(tb, w.part2, w.part3, MLP_KSLICES, w.grad);
  const float b1 = 0.9f, b2 = 0.999f;
  k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(d.p, d.m, d.v, w.grad, lr, b1, b2,
                                                      1.0f - powf(b1, (float)t_adam), 1.0f - powf(b2, (float)t_adam));
  k_mlp_refresh<<<(MLP_H * MLP_H + 255) / 256, 256, 0, s>>>(d.p, d.w2, d.w3, d.w2t, d.w3t);
  if (launches) *launches += 7;
  return cudaGetLastError();
}

// plain forward+backward on a given batch (gradient check entry point): grad receives dL/dp
cudaError_t mlp_grad(MlpDev &d, const float *X, const float *Y, const int *idx, int B, MlpWork &w, cudaStream_t s) {
  cudaError_t e = set_smem_attr();
  if (e != cudaSuccess) return e;
  MlpTrainBufs tb;
  tb.X = X; tb.Y = Y; tb.idx = idx; tb.B = B;
  tb.A1 = w.A1; tb.A2 = w.A2; tb.Z1 = w.Z1; tb.Z2 = w.Z2; tb.Z3 = w.Z3; tb.A3 = w.A3;
  tb.dY = w.dY; tb.loss = w.loss; tb.dZ3 = w.dZ3; tb.dZ2 = w.dZ2; tb.dZ1 = w.dZ1;
  k_mlp_forward_train<<<MLP_TRAIN_BLOCKS, MLP_WARPS * 32, sizeof(MlpSmem), s>>>(d.p, d.w2, d.w3, tb);
  k_mlp_backward<<<MLP_TRAIN_BLOCKS, MLP_WARPS * 32, sizeof(MlpSmem), s>>>(d.p, d.w2t, d.w3t, tb);
  const dim3 gg(MLP_H / 32, MLP_H / 32, MLP_KSLICES);
  k_mlp_wgrad<<<gg, 32, 0, s>>>(w.dZ2, w.A1, B, MLP_KSLICES, w.part2);
  k_mlp_wgrad<<<gg, 32, 0, s>>>(w.dZ3, w.A2, B, MLP_KSLICES, w.part3);
  k_mlp_small_grads<<<(MLP_NPARAM + 127) / 128, 128, 0, s>>>(tb, w.part2, w.part3, MLP_KSLICES, w.grad);
  return cudaGetLastError();
}
