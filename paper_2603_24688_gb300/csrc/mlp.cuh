// Learned surrogate of the rate integrals: a 4 -> 128 -> 128 -> 128 -> 2 MLP whose activation
// is the squared ReLU, act(z) = max(z, 0)^2.
// The two 128 x 128 layers run on the tensor cores (bf16 inputs, float32 accumulation,
// mma.sync m16n8k16); the first and last layers are float32 on the CUDA cores.  One warp
// evaluates 16 rows at a time; the accumulator fragment of one layer is, after the
// activation, exactly the A fragment of the next layer, so activations never leave the
// registers.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

#define MLP_IN 4
#define MLP_H 128
#define MLP_OUT 2
// float32 parameter block: W1[H][IN] b1[H] W2[H][H] b2[H] W3[H][H] b3[H] W4[OUT][H] b4[OUT]
#define MLP_OFF_W1 0
#define MLP_OFF_B1 (MLP_OFF_W1 + MLP_H * MLP_IN)
#define MLP_OFF_W2 (MLP_OFF_B1 + MLP_H)
#define MLP_OFF_B2 (MLP_OFF_W2 + MLP_H * MLP_H)
#define MLP_OFF_W3 (MLP_OFF_B2 + MLP_H)
#define MLP_OFF_B3 (MLP_OFF_W3 + MLP_H * MLP_H)
#define MLP_OFF_W4 (MLP_OFF_B3 + MLP_H)
#define MLP_OFF_B4 (MLP_OFF_W4 + MLP_OUT * MLP_H)
#define MLP_NPARAM (MLP_OFF_B4 + MLP_OUT)

// Shared-memory image of the network used by the kernels (bf16 copies of W2, W3).
struct MlpSmem {
  __nv_bfloat16 W2[MLP_H * MLP_H];
  __nv_bfloat16 W3[MLP_H * MLP_H];
  float W1[MLP_H * MLP_IN];
  float b1[MLP_H], b2[MLP_H], b3[MLP_H];
  float W4[MLP_OUT * MLP_H];
  float b4[MLP_OUT];
};

// Squared ReLU: no special function, so the layer epilogues stay off the MUFU pipe; training
// and inference use the same function.  Its derivative 2 max(z, 0) is continuous.
__device__ __forceinline__ float mlp_act(float z) {
  const float r = fmaxf(z, 0.0f);
  return r * r;
}
__device__ __forceinline__ float mlp_act_grad(float z) { return 2.0f * fmaxf(z, 0.0f); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x = lo (low 16 bits)
  return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One 128 -> 128 layer on 16 rows: acc[nt][0..3] = a . W^T (W row-major [out][in] in smem as
// bf16; out tile nt covers columns nt*8 .. nt*8+7).  A fragments come packed as
// afrag[kt][0..3] for the 8 k16 blocks.
__device__ __forceinline__ void mlp_layer_mma(const __nv_bfloat16 *__restrict__ W, const uint32_t afrag[8][4],
                                              float acc[16][4]) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned g = lane >> 2, tig = lane & 3u;
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
    acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
    const __nv_bfloat16 *wrow = W + (nt * 8 + g) * MLP_H + tig * 2;
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t *>(wrow + kt * 16);
      const uint32_t b1 = *reinterpret_cast<const uint32_t *>(wrow + kt * 16 + 8);
      mma_bf16_16816(acc[nt], afrag[kt], b0, b1);
    }
  }
}

// bias + activation on an accumulator set, packed into the next layer's A fragments
__device__ __forceinline__ void mlp_act_pack(float acc[16][4], const float *__restrict__ bias, uint32_t afrag[8][4]) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned tig = lane & 3u;
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
    const float bb0 = bias[nt * 8 + tig * 2], bb1 = bias[nt * 8 + tig * 2 + 1];
    acc[nt][0] = mlp_act(acc[nt][0] + bb0);
    acc[nt][1] = mlp_act(acc[nt][1] + bb1);
    acc[nt][2] = mlp_act(acc[nt][2] + bb0);
    acc[nt][3] = mlp_act(acc[nt][3] + bb1);
  }
#pragma unroll
  for (int kt = 0; kt < 8; ++kt) {
    afrag[kt][0] = pack_bf16(acc[2 * kt][0], acc[2 * kt][1]);
    afrag[kt][1] = pack_bf16(acc[2 * kt][2], acc[2 * kt][3]);
    afrag[kt][2] = pack_bf16(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
    afrag[kt][3] = pack_bf16(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
  }
}

// Forward of 16 rows.  x_lo / x_hi: the 4 inputs of rows g and g + 8 (g = lane / 4).
// Returns y for rows g (y_lo) and g + 8 (y_hi), identical in the 4 lanes of a quad.
__device__ __forceinline__ void mlp_forward16(const MlpSmem &M, const float x_lo[MLP_IN], const float x_hi[MLP_IN],
                                              float y_lo[MLP_OUT], float y_hi[MLP_OUT]) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned tig = lane & 3u;
  float acc[16][4];
  uint32_t afrag[8][4];
  // layer 1 (float32): z1 = W1 x + b1 at this lane's fragment positions
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int col = nt * 8 + tig * 2 + e;
      float zl = 0.0f, zh = 0.0f;
#pragma unroll
      for (int m = 0; m < MLP_IN; ++m) {
        zl += M.W1[col * MLP_IN + m] * x_lo[m];
        zh += M.W1[col * MLP_IN + m] * x_hi[m];
      }
      acc[nt][e] = zl;
      acc[nt][2 + e] = zh;
    }
  }
  mlp_act_pack(acc, M.b1, afrag);
  mlp_layer_mma(M.W2, afrag, acc);
  mlp_act_pack(acc, M.b2, afrag);
  mlp_layer_mma(M.W3, afrag, acc);
  // layer 3 activation (float32) and the output layer on the CUDA cores
  float pl[MLP_OUT] = {0.f, 0.f}, ph[MLP_OUT] = {0.f, 0.f};
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int col = nt * 8 + tig * 2 + e;
      const float al = mlp_act(acc[nt][e] + M.b3[col]);
      const float ah = mlp_act(acc[nt][2 + e] + M.b3[col]);
#pragma unroll
      for (int o = 0; o < MLP_OUT; ++o) {
        pl[o] += M.W4[o * MLP_H + col] * al;
        ph[o] += M.W4[o * MLP_H + col] * ah;
      }
    }
  }
#pragma unroll
  for (int o = 0; o < MLP_OUT; ++o) {
    pl[o] += __shfl_xor_sync(DMB_FULL, pl[o], 1);
    pl[o] += __shfl_xor_sync(DMB_FULL, pl[o], 2);
    ph[o] += __shfl_xor_sync(DMB_FULL, ph[o], 1);
    ph[o] += __shfl_xor_sync(DMB_FULL, ph[o], 2);
    y_lo[o] = pl[o] + M.b4[o];
    y_hi[o] = ph[o] + M.b4[o];
  }
}

// Surrogate inputs and outputs.  Inputs: log10(s)/2, log10(tau)/2, log10(m_chi/m_p), n/4 with
// s = w/varsigma, tau = varsigma^2/v0^2.  Outputs: the residuals
// log FA - log EA and log FB - log EB against the envelopes E = (1 + p x + q x^2 + r x^3)^m
// (x = s^2/2, m = (n+1)/6 for FA and (n+3)/6 for FB) that carry the exact large-x power and the
// first two Taylor coefficients at x = 0.
struct MlpDomain {
  float s2_lo, s2_hi, tau_lo, tau_hi, m_lo, m_hi;   // training box (s^2 = w^2 / varsigma^2)
  float envA[4], envB[4];   // envelope (p, q, r, m) of FA and FB for the run's n
  float inv_v0sq, log_m, n4;   // inv_v0sq: 1 / v0^2 (power law) or 1 / v_c^2 (screened law)
  int scr;                     // 1: the screened law sigma0 / (1 + (v / v_c)^2)^2
};

// Inputs of a pair from s^2 = w^2 / varsigma^2 and varsigma^2, logarithms by the hardware log2
// (relative error about 2^-22, far below the bf16 parts the network sees); returns whether the
// pair lies in the training box.  Both inference engines use this, so their fallbacks agree.
__device__ __forceinline__ bool mlp_inputs(const MlpDomain &d, float s2, float sig2, float x[MLP_IN]) {
  const float log10_2 = 0.30102999566398120f;
  const float tau = sig2 * d.inv_v0sq;
  x[0] = (0.25f * log10_2) * __log2f(fmaxf(s2, 1e-30f));   // log10(s) / 2
  x[1] = (0.5f * log10_2) * __log2f(fmaxf(tau, 1e-30f));   // log10(tau) / 2
  x[2] = d.log_m;
  x[3] = d.n4;
  return s2 >= d.s2_lo && s2 <= d.s2_hi && tau >= d.tau_lo && tau <= d.tau_hi;
}

// FA = e^{y0} (1 + p x + q x^2 + r x^3)^m, FB likewise, x = s^2 / 2: one hardware exp and log per
// output.
// The screened law divides both envelopes by (1 + q (2x + 3))^2, q = varsigma^2 / v_c^2: sigma/sigma0
// at the pair's mean-square speed, which carries the law's v^-4 fall (the n = -4 behaviour of FA,
// FB at large q), so the network again learns an O(1) correction.
__device__ __forceinline__ void mlp_outputs(const MlpDomain &d, float s2, float sig2, const float y[MLP_OUT],
                                            float &FA, float &FB) {
  const float x = 0.5f * s2;
  const float ls = d.scr ? -2.0f * __logf(fmaf(sig2 * d.inv_v0sq, s2 + 3.0f, 1.0f)) : 0.0f;
  const float pA = fmaf(x, fmaf(x, fmaf(x, d.envA[2], d.envA[1]), d.envA[0]), 1.0f);
  const float pB = fmaf(x, fmaf(x, fmaf(x, d.envB[2], d.envB[1]), d.envB[0]), 1.0f);
  FA = __expf(fmaf(d.envA[3], __logf(pA), y[0] + ls));
  FB = __expf(fmaf(d.envB[3], __logf(pB), y[1] + ls));
}

// ---- batched inference on pairs: 32 rows per warp ---------------------------------------------
// Weights in shared memory with rows padded to 136 bf16 (272 bytes) so that ldmatrix reads of 8
// rows hit distinct banks; activations of a warp's 32 rows are staged the same way.
#define MLP_LDW 136
struct MlpSmemPad {
  __nv_bfloat16 W2[MLP_H * MLP_LDW];
  __nv_bfloat16 W3[MLP_H * MLP_LDW];
  float W1[MLP_H * MLP_IN];
  float b1[MLP_H], b2[MLP_H], b3[MLP_H];
  float W4[MLP_OUT * MLP_H];
  float b4[MLP_OUT];
};

__device__ __forceinline__ void ldmatrix_x4(uint32_t r[4], const void *p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// One 128 -> 128 layer for 32 rows (two m16 tiles) reading A from the warp's activation buffer
// act (row-major, stride MLP_LDW) and W (row-major [out][in], stride MLP_LDW); writes
// act(a W^T + bias) back into act (bf16) when `last` is false; when it is true the float32
// activations go straight into the output layer: yacc[m][h][o] += W4[o][col] a (partial over
// this lane's columns; rows m*16 + g + 8h).
__device__ __forceinline__ void mlp_layer32(const __nv_bfloat16 *__restrict__ W, const float *__restrict__ bias,
                                            __nv_bfloat16 *act, bool last, const float *__restrict__ W4,
                                            float yacc[2][2][MLP_OUT]) {
  const unsigned lane = threadIdx.x & 31u, g = lane >> 2, tig = lane & 3u;
  // A fragments of both m tiles for all 8 k blocks (ldmatrix: lanes 0-15 rows 0-15 at k,
  // lanes 16-31 rows 0-15 at k + 8)
  uint32_t af[2][8][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
      const __nv_bfloat16 *pa = act + (m * 16 + (lane & 15)) * MLP_LDW + kt * 16 + (lane >> 4) * 8;
      uint32_t r[4];
      ldmatrix_x4(r, pa);
      // ldmatrix order: (rows 0-7, k lo), (rows 8-15, k lo), (rows 0-7, k hi), (rows 8-15, k hi)
      af[m][kt][0] = r[0];
      af[m][kt][1] = r[1];
      af[m][kt][2] = r[2];
      af[m][kt][3] = r[3];
    }
  __syncwarp();
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
    float c[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int kt = 0; kt < 8; kt += 2) {
      // B fragments of k blocks kt and kt + 1: matrices (n rows, k lo/hi) of both blocks
      const __nv_bfloat16 *pb = W + (nt * 8 + (lane & 7)) * MLP_LDW + kt * 16 + (lane >> 3) * 8;
      uint32_t b[4];
      ldmatrix_x4(b, pb);
      mma_bf16_16816(c[0], af[0][kt], b[0], b[1]);
      mma_bf16_16816(c[1], af[1][kt], b[0], b[1]);
      mma_bf16_16816(c[0], af[0][kt + 1], b[2], b[3]);
      mma_bf16_16816(c[1], af[1][kt + 1], b[2], b[3]);
    }
    const int col = nt * 8 + tig * 2;
    const float bb0 = bias[col], bb1 = bias[col + 1];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const float v0 = mlp_act(c[m][0] + bb0), v1 = mlp_act(c[m][1] + bb1);
      const float v2 = mlp_act(c[m][2] + bb0), v3 = mlp_act(c[m][3] + bb1);
      if (last) {
#pragma unroll
        for (int o = 0; o < MLP_OUT; ++o) {
          const float w0 = W4[o * MLP_H + col], w1 = W4[o * MLP_H + col + 1];
          yacc[m][0][o] += w0 * v0 + w1 * v1;
          yacc[m][1][o] += w0 * v2 + w1 * v3;
        }
      } else {
        *reinterpret_cast<uint32_t *>(act + (m * 16 + g) * MLP_LDW + col) = pack_bf16(v0, v1);
        *reinterpret_cast<uint32_t *>(act + (m * 16 + g + 8) * MLP_LDW + col) = pack_bf16(v2, v3);
      }
    }
  }
  __syncwarp();
}
