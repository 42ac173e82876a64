// Surrogate inference on the 5th-generation tensor cores (tcgen05): tiles of 128 rows, the
// three hidden layers as 128 x 128 x K MMAs with bf16 operands in shared memory and the float32
// accumulator in tensor memory; the activation and the bf16 repacking run on the CUDA cores
// between the layers, the output layer in float32.
//
// One CTA per SM holds the bf16 weights once and runs NWG independent warpgroups of 128
// threads; warpgroup g owns TMEM columns [128 g, 128 g + 128) and its own activation buffers,
// so while one warpgroup runs its epilogue another one's MMAs run.
//
// With TSA (two warpgroups) the activations stay in tensor memory: the A operand of every
// layer is read by the MMA from TMEM, written by the epilogue with tcgen05.st (two bf16 per
// 32-bit column, row = lane), so the loop stores nothing to shared memory and needs no proxy
// fence.  Warpgroup g then owns columns [256 g, 256 g + 192): A in the first 64 (K = 128 bf16),
// the accumulator in the next 128; three such groups would not fit in the 512 columns.
// Thread t of a warpgroup owns row t of its tile: it forms the row's inputs, reads the row's
// accumulator (TMEM lane t) and writes the row's activations.
//
// Layer 1 (4 -> 128) runs on the tensor cores too, exactly enough for float32 inputs: with
// x = x_hi + x_lo and W1 = W_hi + W_lo (bf16 parts) and the bias b1 = b_hi + b_lo, one K = 16
// MMA forms [x_hi, x_hi, x_lo, 1, 1, 0, 0] . [W_hi, W_lo, W_hi, b_hi, b_lo, 0, 0] (groups of 4
// columns, then single ones); the dropped x_lo . W_lo leaves an error of about 2^-17 of |x| |W|.
//
// The activation is the squared ReLU, so the epilogue of a hidden layer is one multiply and
// half a conversion per activation: t = z |z|, then cvt.rn.relu.bf16x2 packs max(t, 0) =
// max(z, 0)^2 of two columns.  The MMAs of layers 2 and 3 produce z with the bias included:
// one more K = 16 slice multiplies a constant operand row [1, 1, 0, ...] with
// [b_hi, b_lo, 0, ...] (bias split into bf16 parts, exact to about 2^-17).  The output layer
// runs in float32 on packed two-wide FMAs.
//
// Operand layout (no swizzle, K-major): 8 x 16-byte core matrices; element (row, k) of a
// 128-row operand sits at (k / 8) * 2048 + row * 16 + (k % 8) * 2 bytes, so the descriptor of
// the K = 16 slice ks starts at 4096 ks with leading-dimension offset 2048 (next 8 columns) and
// stride-dimension offset 128 (next 8 rows).
#include <cuda_bf16.h>

#include "mlp_tc.cuh"
#include "physics.cuh"

#define TC_ROWS 128
#define TC_SLICE 2048     // bytes between the 8-column chunks of a 128-row operand
#define TC_OPER 32768     // one 128 x 128 bf16 operand
#define TC_OPER1 4096     // one 128 x 16 bf16 operand (layer 1)

// Instruction descriptor of tcgen05.mma kind::f16: D float32 (bits 4-5 = 1), A and B bf16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at bits 17-22, M / 16 at bits 24-28.
#define TC_IDESC ((1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24))

// shared-memory layout (bytes)
template <int NWG>
struct TcLayout {
  static constexpr int W2 = 0;
  static constexpr int W3 = W2 + TC_OPER;
  static constexpr int A = W3 + TC_OPER;                 // NWG activation operands (slice 0 of each also
                                                         // holds the layer-1 operand of a new tile)
  static constexpr int W1 = A + NWG * TC_OPER;           // split W1 and b1 (128 x 16)
  static constexpr int ONE = W1 + TC_OPER1;              // constant operand rows [1, 1, 0, ...] (128 x 16)
  static constexpr int BB = ONE + TC_OPER1;              // bias operands [b_hi, b_lo, 0, ...] of layers 2, 3
  static constexpr int W4 = BB + 2 * TC_OPER1;           // [2][128] float
  static constexpr int B4 = W4 + 1024;                   // 2 floats (16 bytes)
  static constexpr int BAR = B4 + 16;                    // NWG mbarriers (8-byte aligned)
  static constexpr int TSLOT = BAR + NWG * 8;            // TMEM base address
  static constexpr int TOTAL = (TSLOT + 16 + 1023) / 1024 * 1024;
};
static_assert(TcLayout<4>::TOTAL <= 232448, "shared memory of the tensor-core surrogate");
static_assert(TcLayout<3>::BAR % 8 == 0, "mbarrier alignment");

// ---- PTX wrappers ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Tests the phase; while it is incomplete the thread may sleep up to about 0.1 ms (the
// suspend-time hint, in ns) and wakes when the phase completes, so waiting threads take few
// issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0u;
}

// Waits for the phase with the given parity to complete; gives up after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void wg_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
// barrier of the warpgroup that also returns whether v holds in all 128 threads
__device__ __forceinline__ bool wg_sync_and(int id, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, %2, 128, q;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id)
      : "memory");
  return r != 0u;
}

// Shared-memory matrix descriptor: start address, leading- and stride-dimension byte offsets
// (all >> 4), descriptor version 1 at bit 46, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;
  return d;
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate)
      : "memory");
}

// the same MMA with A read from tensor memory (lane = row, column c = elements 2c, 2c + 1)
__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive float32 columns of this thread's TMEM lane; the wait is tied to the registers
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// 32 columns without the wait: the registers are valid after tmem_wait_ld and reg_tie32
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t r[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// orders the uses of r after the preceding tmem_wait_ld
__device__ __forceinline__ void reg_tie32(uint32_t r[32]) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}

// 16 (8) consecutive 32-bit columns of this thread's TMEM lane; completed by tmem_wait_st
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t r[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t r[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// bf16x2 of (max(lo, 0), max(hi, 0)), lo in the low half, each rounded to nearest even
__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ uint32_t bf16_bits(float x) {
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  return (uint32_t) * reinterpret_cast<const uint16_t *>(&b);
}

__device__ __forceinline__ float as_f32(float x) { return x; }
__device__ __forceinline__ float as_f32(uint32_t x) { return __uint_as_float(x); }

// Output layer, four columns: y_o += W4[o][c] max(z_c, 0)^2 for c = c0 .. c0 + 3 (z as float or
// raw bits, w = W4 + c0 in shared memory, 16-byte aligned); columns (c0, c0 + 1) go to
// accumulator k & 3 and (c0 + 2, c0 + 3) to (k + 1) & 3.  One 16-byte load per output row and
// four columns.
template <typename Z>
__device__ __forceinline__ void out_layer4(const Z *z, const float *w, int k, float2 y0[4], float2 y1[4]) {
  const float4 wa = *reinterpret_cast<const float4 *>(w);
  const float4 wb = *reinterpret_cast<const float4 *>(w + MLP_H);
  const float2 r0 = make_float2(fmaxf(as_f32(z[0]), 0.0f), fmaxf(as_f32(z[1]), 0.0f));
  const float2 r1 = make_float2(fmaxf(as_f32(z[2]), 0.0f), fmaxf(as_f32(z[3]), 0.0f));
  const float2 a0 = __fmul2_rn(r0, r0), a1 = __fmul2_rn(r1, r1);
  y0[k & 3] = __ffma2_rn(make_float2(wa.x, wa.y), a0, y0[k & 3]);
  y1[k & 3] = __ffma2_rn(make_float2(wb.x, wb.y), a0, y1[k & 3]);
  y0[(k + 1) & 3] = __ffma2_rn(make_float2(wa.z, wa.w), a1, y0[(k + 1) & 3]);
  y1[(k + 1) & 3] = __ffma2_rn(make_float2(wb.z, wb.w), a1, y1[(k + 1) & 3]);
}

// ---- row gather, in dependent stages --------------------------------------------------------
// MODE_X: Vi = X[q] (the four network inputs).  MODE_PAIRS: k = prow[q] is the row of q; the
// pair is p = q (rows are all gas, k = j) or p = row_ptr[list[k]] + q - R_ptr[k] (listed rows);
// Vi, Vj are the sorted velocity copies of its DM particle i = rows[p] and gas particle j.
struct RowFetch {
  int64_t q = -1, k = 0, p = 0;
  uint32_t i = 0, j = 0;
  float4 Vi = make_float4(0.f, 0.f, 0.f, 0.f), Vj = make_float4(0.f, 0.f, 0.f, 0.f);
};

template <int MODE>
__device__ __forceinline__ void fetch_stage(const TcArgs &a, int64_t q, int stage, RowFetch &f) {
  if (stage == 0) {
    f.q = q < a.n ? q : -1;
    if (f.q < 0) return;
    if (MODE == 0) {
      f.p = q;
      f.Vi = *reinterpret_cast<const float4 *>(a.X + 4 * q);
    } else {
      f.k = a.prow[q];
      if (a.list == nullptr) {
        f.p = q;
        f.j = (uint32_t)f.k;
        f.i = a.rows[q];
      }
    }
    return;
  }
  if (MODE == 0 || f.q < 0) return;
  if (a.list == nullptr) {
    if (stage == 1) {
      f.Vj = a.G_V[f.j];
      f.Vi = a.D_V[f.i];
    }
    return;
  }
  if (stage == 1) {
    f.j = a.list[f.k];
    f.p = a.row_ptr[f.j] + (f.q - a.R_ptr[f.k]);
  } else if (stage == 2) {
    f.i = a.rows[f.p];
    f.Vj = a.G_V[f.j];
  } else {
    f.Vi = a.D_V[f.i];
  }
}

// ---- the kernel -----------------------------------------------------------------------------
// MODE_X: rows are the caller's inputs X[n][4], outputs the raw network outputs Y[n][2].
// MODE_PAIRS: rows are gas-major pairs (processing order q over a row-start prefix R_ptr),
// outputs the normalised rates (FA, FB) at the pair's index p; out-of-box rows take the
// quadrature (counted), cold gas is skipped (the mean field uses the exact cold limit).
// MODE_MF: the same rows, and the rates go straight into the gas mean field: the pair's
// geometry (displacement, distance, overlap g, M_i g) is formed while the last layer's MMA runs,
// the rates (or the cold limit) after the output layer, and the row's six terms are summed per
// gas row over each warp's 32 rows into the per-segment sums.
enum { MODE_X = 0, MODE_PAIRS = 1, MODE_MF = 2 };

template <int NWG, int MODE, bool TSA>
__global__ void __launch_bounds__(NWG * 128, 1) k_mlp_tc(TcArgs a) {
  static_assert(!TSA || NWG == 2, "activations in tensor memory: two warpgroups of 192 columns");
  typedef TcLayout<NWG> Ly;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x;
  const int g = tid >> 7;             // warpgroup
  const int t = tid & 127;            // row of the tile
  const int w = t >> 5;               // warp within the warpgroup: TMEM lanes 32 w .. 32 w + 31
  const uint32_t sbase = smem_u32(sm);

  // ---- weights into the operand layout ---------------------------------------------------
  for (int q = tid; q < 2 * MLP_H * (MLP_H / 8); q += blockDim.x) {
    const int which = q / (MLP_H * (MLP_H / 8));
    const int r = q % (MLP_H * (MLP_H / 8));
    const int n = r % MLP_H, c = r / MLP_H;           // output row n, 8-column chunk c
    const __nv_bfloat16 *src = (which == 0 ? a.w2 : a.w3) + n * MLP_H + c * 8;
    const uint4 v = *reinterpret_cast<const uint4 *>(src);
    *reinterpret_cast<uint4 *>(sm + (which == 0 ? Ly::W2 : Ly::W3) + c * TC_SLICE + n * 16) = v;
  }
  for (int n = tid; n < MLP_H; n += blockDim.x) {
    uint32_t hl[4];
#pragma unroll
    for (int m = 0; m < MLP_IN; m += 2) {
      const float w0 = a.p[MLP_OFF_W1 + n * MLP_IN + m], w1 = a.p[MLP_OFF_W1 + n * MLP_IN + m + 1];
      const float h0 = __bfloat162float(__float2bfloat16_rn(w0)), h1 = __bfloat162float(__float2bfloat16_rn(w1));
      hl[m / 2] = bf16_bits(w0) | (bf16_bits(w1) << 16);
      hl[2 + m / 2] = bf16_bits(w0 - h0) | (bf16_bits(w1 - h1) << 16);
    }
    // bias as [b_hi, b_lo, 0, 0, 0, 0, 0, 0] (bf16 parts)
    auto bias_chunk = [](float b) {
      const float bh = __bfloat162float(__float2bfloat16_rn(b));
      return make_uint4(bf16_bits(b) | (bf16_bits(b - bh) << 16), 0u, 0u, 0u);
    };
    const uint4 b1c = bias_chunk(a.p[MLP_OFF_B1 + n]);
    // chunk 0 = [W_hi(4), W_lo(4)], chunk 1 = [W_hi(4), b_hi, b_lo, 0, 0]
    *reinterpret_cast<uint4 *>(sm + Ly::W1 + 0 * TC_SLICE + n * 16) = make_uint4(hl[0], hl[1], hl[2], hl[3]);
    *reinterpret_cast<uint4 *>(sm + Ly::W1 + 1 * TC_SLICE + n * 16) = make_uint4(hl[0], hl[1], b1c.x, 0u);
    // constant rows [1, 1, 0, ...] and the bias rows of layers 2 and 3
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(sm + Ly::ONE + 0 * TC_SLICE + n * 16) = make_uint4(0x3F803F80u, 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(sm + Ly::ONE + 1 * TC_SLICE + n * 16) = zero;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      *reinterpret_cast<uint4 *>(sm + Ly::BB + l * TC_OPER1 + 0 * TC_SLICE + n * 16) =
          bias_chunk(a.p[(l == 0 ? MLP_OFF_B2 : MLP_OFF_B3) + n]);
      *reinterpret_cast<uint4 *>(sm + Ly::BB + l * TC_OPER1 + 1 * TC_SLICE + n * 16) = zero;
    }
  }
  float *W4 = reinterpret_cast<float *>(sm + Ly::W4);
  float *b4 = reinterpret_cast<float *>(sm + Ly::B4);
  for (int c = tid; c < MLP_H; c += blockDim.x) {
    W4[c] = a.p[MLP_OFF_W4 + c];
    W4[MLP_H + c] = a.p[MLP_OFF_W4 + MLP_H + c];
  }
  if (tid < MLP_OUT) b4[tid] = a.p[MLP_OFF_B4 + tid];
  const uint32_t bar = sbase + Ly::BAR + 8 * g;
  if (tid == 0) {
    for (int k = 0; k < NWG; ++k) mbar_init(sbase + Ly::BAR + 8 * k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + Ly::TSLOT);
  const uint32_t ncols = (NWG <= 2 && !TSA) ? 256u : 512u;
  static_assert(NWG * 128 <= 512, "tensor memory holds at most four 128-column accumulators");
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + Ly::TSLOT),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();   // the weights were written by the generic proxy; the MMAs read them
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // lane 0 of this group's accumulator (and, with TSA, of its A operand)
  const uint32_t a_tmem = tmem + 256u * (uint32_t)g;
  const uint32_t d_tmem = TSA ? a_tmem + 64u : tmem + 128u * (uint32_t)g;
  const uint32_t my_lanes = d_tmem + ((uint32_t)(32 * w) << 16);
  const uint32_t my_a = a_tmem + ((uint32_t)(32 * w) << 16);
  const uint32_t sA = sbase + Ly::A + g * TC_OPER;   // the layer-1 operand is slice 0 of A
  // the operands' descriptors, built once: a K = 16 slice further is 2 TC_SLICE bytes on, which
  // adds (2 TC_SLICE) >> 4 to the start-address field (shared addresses stay below 2^18 bytes)
  const uint64_t dA = smem_desc(sA, TC_SLICE, 128), dW1 = smem_desc(sbase + Ly::W1, TC_SLICE, 128);
  const uint64_t dW2 = smem_desc(sbase + Ly::W2, TC_SLICE, 128), dW3 = smem_desc(sbase + Ly::W3, TC_SLICE, 128);
  const uint64_t dONE = smem_desc(sbase + Ly::ONE, TC_SLICE, 128);
  const uint64_t dBB2 = smem_desc(sbase + Ly::BB, TC_SLICE, 128), dBB3 = smem_desc(sbase + Ly::BB + TC_OPER1, TC_SLICE, 128);
  const uint64_t dks = (uint64_t)((2 * TC_SLICE) >> 4);
  unsigned char *pA = sm + Ly::A + g * TC_OPER;
  unsigned char *pA1 = pA;
  const int bar_id = 1 + g;
  uint32_t phase = 0;
  unsigned fallback = 0;
  bool ok = true;
  bool skip_commit = a.skip_commit != 0 && blockIdx.x == 0 && g == 0;
  const uint64_t wait_ns = a.wait_ns ? a.wait_ns : 2000000000ull;
  const float alpha = (float)a.rc.alpha;
  const float inv_v0 = (float)(1.0 / a.rc.v0), inv_vc2 = (float)a.rc.inv_vc2;
  if (a.n_dev != nullptr) a.n = min(a.n, *a.n_dev);   // rows counted on the device (captured steps)
  const int64_t n_tiles = (a.n + TC_ROWS - 1) / TC_ROWS;
  const int64_t stride = (int64_t)gridDim.x * NWG;

  // The inputs of the next tile are gathered while this tile's MMAs run: stage 0 is issued
  // behind the layer-1 MMA, stage 1 behind layer 2 and stages 2-3 behind layer 3.
  RowFetch nxt;
  int64_t T = (int64_t)blockIdx.x * NWG + g;
  fetch_stage<MODE>(a, T * TC_ROWS + t, 0, nxt);
  fetch_stage<MODE>(a, 0, 1, nxt);
  fetch_stage<MODE>(a, 0, 2, nxt);
  fetch_stage<MODE>(a, 0, 3, nxt);
  for (; T < n_tiles && ok; T += stride) {
    // ---- this tile's row inputs (gathered one tile ahead) --------------------------------
    float x[MLP_IN] = {0.f, 0.f, 0.f, 0.f};
    const int64_t p = nxt.p;
    float s2 = 0.f;                                   // (w / varsigma)^2
    float sg2 = 0.f;                                  // varsigma^2
    bool use = false, in_dom = false;
    // MODE_MF: the row's gas row k (the segment key; all ones for no row), its particles, the
    // relative velocity w = v_i - V_j, v_i.w, and later M_i g_ij
    uint32_t key = 0xFFFFFFFFu, cur_i = 0u, cur_j = 0u;
    float wx = 0.f, wy = 0.f, wz = 0.f, vdw = 0.f, tM = 0.f;
    if (nxt.q >= 0) {
      if (MODE == MODE_X) {
        x[0] = nxt.Vi.x; x[1] = nxt.Vi.y; x[2] = nxt.Vi.z; x[3] = nxt.Vi.w;
        use = in_dom = true;
      } else {
        const float sig = nxt.Vj.w;
        wx = nxt.Vi.x - nxt.Vj.x;
        wy = nxt.Vi.y - nxt.Vj.y;
        wz = nxt.Vi.z - nxt.Vj.z;
        if (MODE == MODE_MF) {
          key = (uint32_t)nxt.k;
          cur_i = nxt.i;
          cur_j = nxt.j;
          vdw = nxt.Vi.x * wx + nxt.Vi.y * wy + nxt.Vi.z * wz;
        }
        if (sig > 0.0f) {
          const float sig2 = sig * sig;
          sg2 = sig2;
          s2 = __fdividef(wx * wx + wy * wy + wz * wz, sig2);
          in_dom = mlp_inputs(a.dom, s2, sig2, x);
          use = true;
        }
      }
    }
    const int64_t qn = (T + stride) * TC_ROWS + t;    // the next tile's row
    // layer-1 operand row: chunk 0 = [x_hi, x_hi], chunk 1 = [x_lo, 1, 1, 0, 0]
    {
      uint32_t hi2[2], lo2[2];
#pragma unroll
      for (int m = 0; m < MLP_IN; m += 2) {
        const float h0 = __bfloat162float(__float2bfloat16_rn(x[m]));
        const float h1 = __bfloat162float(__float2bfloat16_rn(x[m + 1]));
        hi2[m / 2] = bf16_bits(x[m]) | (bf16_bits(x[m + 1]) << 16);
        lo2[m / 2] = bf16_bits(x[m] - h0) | (bf16_bits(x[m + 1] - h1) << 16);
      }
      if (TSA) {
        const uint32_t r8[8] = {hi2[0], hi2[1], hi2[0], hi2[1], lo2[0], lo2[1], 0x3F803F80u, 0u};
        tmem_st8(my_a, r8);
      } else {
        *reinterpret_cast<uint4 *>(pA1 + 0 * TC_SLICE + t * 16) = make_uint4(hi2[0], hi2[1], hi2[0], hi2[1]);
        *reinterpret_cast<uint4 *>(pA1 + 1 * TC_SLICE + t * 16) = make_uint4(lo2[0], lo2[1], 0x3F803F80u, 0u);
      }
    }
    // ---- three layers ------------------------------------------------------------------------
    // output-layer partial sums: four independent two-wide accumulators per output
    float2 y0[4], y1[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) y0[u] = y1[u] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int layer = 0; layer < 3; ++layer) {
      if (TSA)
        tmem_wait_st();   // this thread's row of the A operand is in tensor memory
      else
        fence_async_smem();
      tc_fence_before();
      wg_sync(bar_id);
      if (t == 0) {
        tc_fence_after();
        if (layer == 0) {
          if (TSA)
            tc_mma_ts(d_tmem, a_tmem, dW1, 0u);
          else
            tc_mma(d_tmem, dA, dW1, 0u);
        } else {
          const uint64_t dW = layer == 1 ? dW2 : dW3;
#pragma unroll
          for (int ks = 0; ks < MLP_H / 16; ++ks) {
            if (TSA)
              tc_mma_ts(d_tmem, a_tmem + 8u * ks, dW + dks * ks, ks > 0 ? 1u : 0u);
            else
              tc_mma(d_tmem, dA + dks * ks, dW + dks * ks, ks > 0 ? 1u : 0u);
          }
          // + b through the constant slice
          tc_mma(d_tmem, dONE, layer == 1 ? dBB2 : dBB3, 1u);
        }
        // (fault injection only: the first layer-1 commit of group 0 in CTA 0 is left out)
        if (!(skip_commit && layer == 0)) tc_commit(bar);
      }
      skip_commit = false;
      // the next tile's gather behind this MMA
      if (layer == 0) {
        fetch_stage<MODE>(a, qn, 0, nxt);
      } else if (layer == 1) {
        fetch_stage<MODE>(a, 0, 1, nxt);
      } else {
        fetch_stage<MODE>(a, 0, 2, nxt);
        fetch_stage<MODE>(a, 0, 3, nxt);
        if (MODE == MODE_MF && key != 0xFFFFFFFFu) {
          // the pair's overlap while the last MMA runs (Eq. gas-dVdt's g_ij, the kernels'
          // canonical displacement and distance)
          const float4 Pi = a.D_P[cur_i], Li = a.D_L[cur_i], Pj = a.G_P[cur_j], Lj = a.G_L[cur_j];
          const BoxSide side = a.bx.boxes != nullptr ? a.bx.boxes[a.G_bid[cur_j]] : box_side<GEOM_BOX>(a.bx, 0);
          float dx, dy, dz;
          pair_dx<float>(Pi, Li, Pj, Lj, a.bx.periodic, side, dx, dy, dz);
          const float d = sqrt_pair(dist2_rn<float>(dx, dy, dz));
          tM = Li.w * overlap_g<float>(a.gtab, d, Pi.w, Pj.w);
        }
      }
      // the group's first warp waits (bounded) for the MMA while the other three wait at the
      // group's barrier, which also makes the group agree on the outcome, so that a timeout is
      // seen by all 128
      const bool done = wg_sync_and(bar_id, w == 0 ? mbar_wait_bounded(bar, phase, wait_ns) : true);
      if (!done) {
        // the MMAs this group issued may still be in flight: a new commit tracks them, and the
        // group waits for it (bounded again) before it leaves and the CTA frees tensor memory
        if (t == 0) tc_commit(bar);
        (void)wg_sync_and(bar_id, w == 0 ? mbar_wait_bounded(bar, phase, wait_ns) : true);
        ok = false;
        break;
      }
      phase ^= 1u;
      tc_fence_after();
      if (TSA) {
        // the whole row of z at once (one wait for four loads): with two warpgroups each warp
        // has the registers, and the epilogue's latency is what limits it
        uint32_t r[MLP_H];
#pragma unroll
        for (int cc = 0; cc < MLP_H / 32; ++cc) tmem_ld32_nowait(my_lanes + 32u * cc, r + 32 * cc);
        tmem_wait_ld();
#pragma unroll
        for (int cc = 0; cc < MLP_H / 32; ++cc) reg_tie32(r + 32 * cc);
        if (layer < 2) {
#pragma unroll
          for (int cc = 0; cc < MLP_H / 32; ++cc) {
            uint32_t pk[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const float z0 = __uint_as_float(r[32 * cc + 2 * k]), z1 = __uint_as_float(r[32 * cc + 2 * k + 1]);
              pk[k] = pack_relu_bf16(z0 * fabsf(z0), z1 * fabsf(z1));
            }
            tmem_st16(my_a + 16u * cc, pk);
          }
        } else {
#pragma unroll
          for (int k = 0; k < MLP_H / 2; k += 2) out_layer4(r + 2 * k, W4 + 2 * k, k, y0, y1);
        }
      } else {
#pragma unroll 1
        for (int cc = 0; cc < MLP_H / 32; ++cc) {
          float v[32];
          tmem_ld32(my_lanes + 32u * cc, v);   // z with the bias
          if (layer < 2) {
            uint32_t pk[16];
#pragma unroll
            for (int k = 0; k < 16; ++k)
              pk[k] = pack_relu_bf16(v[2 * k] * fabsf(v[2 * k]), v[2 * k + 1] * fabsf(v[2 * k + 1]));
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4)
              *reinterpret_cast<uint4 *>(pA + (4 * cc + c4) * TC_SLICE + t * 16) =
                  make_uint4(pk[4 * c4], pk[4 * c4 + 1], pk[4 * c4 + 2], pk[4 * c4 + 3]);
          } else {
#pragma unroll
            for (int k = 0; k < 16; k += 2) out_layer4(v + 2 * k, W4 + 32 * cc + 2 * k, k, y0, y1);
          }
        }
      }
    }
    if (!ok) break;
    tc_fence_before();   // this tile's TMEM reads are done before the next tile's MMA
    // ---- outputs -----------------------------------------------------------------------------
    const float2 s0 = __fadd2_rn(__fadd2_rn(y0[0], y0[1]), __fadd2_rn(y0[2], y0[3]));
    const float2 s1 = __fadd2_rn(__fadd2_rn(y1[0], y1[1]), __fadd2_rn(y1[2], y1[3]));
    const float y[MLP_OUT] = {(s0.x + s0.y) + b4[0], (s1.x + s1.y) + b4[1]};
    if (MODE == MODE_X) {
      if (use) {
        a.Y[2 * p] = y[0];
        a.Y[2 * p + 1] = y[1];
      }
    } else if (MODE == MODE_MF) {
      float c[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (key != 0xFFFFFFFFu) {
        const float w2 = wx * wx + wy * wy + wz * wz;
        float FA, FB;
        if (use) {
          if (in_dom) {
            mlp_outputs(a.dom, s2, sg2, y, FA, FB);
          } else {
            rates_quad<float>(0.5f * s2, a.rc.n, alpha, FA, FB, sg2 * inv_vc2);
            ++fallback;
          }
        } else {   // cold gas: the exact limit A = sigma(w) w, B = sigma(w) w^3
          const float wn = sqrt_t(w2);
          const float sn = sigma_ratio<float>(wn, a.rc.n, inv_v0, inv_vc2);
          FA = sn * wn;
          FB = sn * wn * w2;
        }
        const float tA = tM * FA;
        c[0] = tA * wx;
        c[1] = tA * wy;
        c[2] = tA * wz;
        c[3] = tA * w2;
        c[4] = tM * FB;
        c[5] = tA * vdw;
      }
      // sums over the warp's rows of the same gas row: the keys ascend along the lanes, so after
      // the step with offset o lane l holds the sum over [l, l + 2o) within its row; the first
      // lane of each row writes it
      const unsigned lane = (unsigned)t & 31u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t ko = __shfl_down_sync(DMB_FULL, key, o);
        const bool same = lane + (unsigned)o < 32u && ko == key;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
          const float v = __shfl_down_sync(DMB_FULL, c[m], o);
          if (same) c[m] += v;
        }
      }
      const uint32_t kp = __shfl_up_sync(DMB_FULL, key, 1);
      if (key != 0xFFFFFFFFu && (lane == 0u || kp != key)) {
        float2 *dst = reinterpret_cast<float2 *>(a.part + 6 * ((T * TC_ROWS + t) / 32 + (int64_t)key));
        dst[0] = make_float2(c[0], c[1]);
        dst[1] = make_float2(c[2], c[3]);
        dst[2] = make_float2(c[4], c[5]);
      }
    } else if (use) {
      float FA, FB;
      if (in_dom) {
        mlp_outputs(a.dom, s2, sg2, y, FA, FB);
      } else {
        rates_quad<float>(0.5f * s2, a.rc.n, alpha, FA, FB, sg2 * (float)a.rc.inv_vc2);
        ++fallback;
      }
      a.rates[p] = make_float2(FA, FB);
    }
  }
  if (!ok && t == 0) atomicOr(a.status, DMB_BAD_TIMEOUT);
  if (MODE != MODE_X) {
    fallback = warp_sum<unsigned>(fallback);
    if ((tid & 31) == 0 && fallback && a.fallback_count) atomicAdd(a.fallback_count, (unsigned long long)fallback);
  }
  tc_fence_before();
  __syncthreads();
  if (tid < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// row k of every processing index q: prow[q] = k for q in [R_ptr[k], R_ptr[k + 1]) (warp per row)
__global__ void k_pair_rows(const int64_t *__restrict__ R_ptr, int64_t n_rows, uint32_t *__restrict__ prow) {
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_rows; k += nw)
    for (int64_t q = R_ptr[k] + lane; q < R_ptr[k + 1]; q += 32) prow[q] = (uint32_t)k;
}

static bool g_tc_attr = false;

cudaError_t mlp_tc_prepare() {
  if (g_tc_attr) return cudaSuccess;
  const void *fns[9] = {(const void *)k_mlp_tc<2, MODE_X, true>,      (const void *)k_mlp_tc<2, MODE_PAIRS, true>,
                        (const void *)k_mlp_tc<2, MODE_MF, true>,     (const void *)k_mlp_tc<3, MODE_X, false>,
                        (const void *)k_mlp_tc<3, MODE_PAIRS, false>, (const void *)k_mlp_tc<3, MODE_MF, false>,
                        (const void *)k_mlp_tc<4, MODE_X, false>,     (const void *)k_mlp_tc<4, MODE_PAIRS, false>,
                        (const void *)k_mlp_tc<4, MODE_MF, false>};
  const int smem[9] = {TcLayout<2>::TOTAL, TcLayout<2>::TOTAL, TcLayout<2>::TOTAL,
                       TcLayout<3>::TOTAL, TcLayout<3>::TOTAL, TcLayout<3>::TOTAL,
                       TcLayout<4>::TOTAL, TcLayout<4>::TOTAL, TcLayout<4>::TOTAL};
  for (int k = 0; k < 9; ++k) {
    const cudaError_t e = cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, smem[k]);
    if (e != cudaSuccess) return e;
  }
  g_tc_attr = true;
  return cudaSuccess;
}

template <int NWG, int MODE, bool TSA = false>
static cudaError_t launch_tc(const TcArgs &a, cudaStream_t s) {
  const int smem = TcLayout<NWG>::TOTAL;
  const cudaError_t e = mlp_tc_prepare();
  if (e != cudaSuccess) return e;
  const int64_t n_tiles = (a.n + TC_ROWS - 1) / TC_ROWS;
  int64_t blocks = (n_tiles + NWG - 1) / NWG;
  if (blocks > 152) blocks = 152;
  if (blocks < 1) blocks = 1;
  TcArgs b = a;
  if (b.skip_commit) b.wait_ns = 1000000ull;   // the injected timeout: 1 ms
  k_mlp_tc<NWG, MODE, TSA><<<(unsigned)blocks, NWG * 128, smem, s>>>(b);
  return cudaGetLastError();
}

// nwg: 2..4 independent warpgroups (one tile each)
template <int MODE>
static cudaError_t launch_any(const TcArgs &a, int nwg, cudaStream_t s) {
  switch (nwg) {
    case 2: return launch_tc<2, MODE, true>(a, s);
    case 3: return launch_tc<3, MODE>(a, s);
    default: return launch_tc<4, MODE>(a, s);
  }
}

cudaError_t mlp_tc_infer(TcArgs a, int nwg, cudaStream_t s, int64_t *launches) {
  if (a.n <= 0) return cudaSuccess;
  if (launches) *launches += 1;
  return launch_any<MODE_X>(a, nwg, s);
}

cudaError_t mlp_tc_pair_rates(TcArgs a, uint32_t *prow, int nwg, cudaStream_t s, int64_t *launches) {
  if (a.n <= 0 || a.n_rows <= 0) return cudaSuccess;
  int64_t blocks = (a.n_rows * 32 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_pair_rows<<<(unsigned)blocks, 256, 0, s>>>(a.R_ptr, a.n_rows, prow);
  a.prow = prow;
  if (launches) *launches += 2;
  return launch_any<MODE_PAIRS>(a, nwg, s);
}

// acc_j = cA sum(M_i g FA w), du_j/dt = cA sum(M_i g FA w^2) - cB sum(M_i g FB) and the expected
// DM energy change M_j (cB sum(M_i g FB) - cA sum(M_i g FA v_i.w)) (no dt) of row k, from the
// slots q / 32 + k of its processing positions q, summed in float64 in slot order.
__global__ void k_tc_mf_finish(const int64_t *__restrict__ R_ptr, int64_t n_rows, const uint32_t *__restrict__ list,
                               const float4 *__restrict__ G_K, const float4 *__restrict__ G_L,
                               const uint32_t *__restrict__ G_perm, const float *__restrict__ part,
                               double *__restrict__ acc, double *__restrict__ dudt, double *__restrict__ e_exp) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_rows) return;
  const int64_t j = list ? (int64_t)list[k] : k;
  const int64_t q0 = R_ptr[k], q1 = R_ptr[k + 1];
  double sum[6] = {0, 0, 0, 0, 0, 0};
  if (q1 > q0) {
    for (int64_t u = (q0 >> 5) + k; u <= ((q1 - 1) >> 5) + k; ++u) {
      const float2 *src = reinterpret_cast<const float2 *>(part + 6 * u);
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const float2 v = src[m];
        sum[2 * m] += (double)v.x;
        sum[2 * m + 1] += (double)v.y;
      }
    }
  }
  const float4 K = G_K[j];
  const double cA = (double)K.x, cB = (double)K.y;
  const uint32_t c = G_perm[j];
  acc[3 * (int64_t)c + 0] = cA * sum[0];
  acc[3 * (int64_t)c + 1] = cA * sum[1];
  acc[3 * (int64_t)c + 2] = cA * sum[2];
  dudt[c] = cA * sum[3] - cB * sum[4];
  if (e_exp) e_exp[j] = (double)G_L[j].w * (cB * sum[4] - cA * sum[5]);
}

cudaError_t mlp_tc_meanfield(TcArgs a, uint32_t *prow, int nwg, const float4 *G_K, const uint32_t *G_perm,
                             double *acc, double *dudt, double *e_exp, cudaStream_t s, int64_t *launches) {
  if (a.n_rows <= 0) return cudaSuccess;
  if (a.n > 0) {
    int64_t blocks = (a.n_rows * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_pair_rows<<<(unsigned)blocks, 256, 0, s>>>(a.R_ptr, a.n_rows, prow);
    a.prow = prow;
    if (launches) *launches += 2;
    cudaError_t e;
    switch (nwg) {
      case 2: e = launch_tc<2, MODE_MF, true>(a, s); break;
      case 3: e = launch_tc<3, MODE_MF>(a, s); break;
      default: e = launch_tc<4, MODE_MF>(a, s); break;
    }
    if (e != cudaSuccess) return e;
  }
  k_tc_mf_finish<<<(unsigned)((a.n_rows + 255) / 256), 256, 0, s>>>(a.R_ptr, a.n_rows, a.list, G_K, a.G_L, G_perm,
                                                                    a.part, acc, dudt, e_exp);
  if (launches) *launches += 1;
  return cudaGetLastError();
}
