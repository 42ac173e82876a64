// Shared device types and helpers of the CUDA path (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dmb.h"

#define DMB_WARP 32
#define DMB_LEAF 32          // particles per tree leaf (one warp's worth)
#define DMB_MAX_LEVELS 8     // 32^7 leaves suffice for 2^31 particles
#define DMB_FULL 0xffffffffu

// overlap table: delta nodes on [0, 2], q nodes on [0, 1]
#define DMB_GT_ND 1025                 // delta nodes on [0, 2]
#define DMB_GT_NQ 513                  // q nodes on [0, 1]
#define DMB_GT_CELLS (DMB_GT_ND - 1)

// ---- float / double traits --------------------------------------------------------
template <typename R> struct Vec;
template <> struct Vec<float> {
  typedef float4 v4;
  static __host__ __device__ __forceinline__ float4 make(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
};
template <> struct Vec<double> {
  typedef double4_32a v4;
  static __host__ __device__ __forceinline__ double4_32a make(double a, double b, double c, double d) { return make_double4_32a(a, b, c, d); }
};

// Arithmetic that the compiler may not contract into FMAs: used where two kernels must
// reach bit-identical results from the same inputs (the pair predicate and distance).
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// ---- sorted species on the device -------------------------------------------------
// Positions are split as x - origin = hi + lo with hi an integer multiple of a power of two
// Delta (so hi differences are exact in float32) and lo in [0, Delta).
template <typename R> struct SpeciesView {
  int64_t n;
  const typename Vec<R>::v4 *P;   // (hi_x, hi_y, hi_z, h)
  const typename Vec<R>::v4 *L;   // (lo_x, lo_y, lo_z, M)
  const typename Vec<R>::v4 *V;   // (vx, vy, vz, varsigma [gas] | 0 [dm])
  const typename Vec<R>::v4 *K;   // gas: (cA, cB, kP0, e = mu/(m_chi + mu)); dm: unused
  const uint32_t *id;             // stable id
  const uint32_t *perm;           // sorted position -> caller index
  const uint16_t *bid;            // batched boxes: box index per sorted particle (else null)
  const int2 *leaf_box;           // batched boxes: lowest and highest box index per leaf (else null)
  // 32-ary tree: level 0 = leaves of DMB_LEAF consecutive sorted particles, node i of level
  // l > 0 groups nodes 32i .. 32i+31 of level l-1; level l occupies [off[l], off[l] + cnt[l])
  const float4 *bmin;             // (min xyz, h_max of the particles below)
  const float4 *bmax;             // (max xyz, unused)
  int32_t levels;                 // number of levels; the root is level levels-1 (one node)
  int32_t off[DMB_MAX_LEVELS];
  int32_t cnt[DMB_MAX_LEVELS];
};

// Sides of one periodic box in the split representation (float hi + float lo, and float64).
struct BoxSide {
  float Lhi[3], Llo[3];
  double L[3];
};

// Periodic boxes: one (the context's), or a table of per-box sides for batched boxes, each
// particle carrying its box index.
struct BoxSplit {
  int periodic;
  float Lhi[3], Llo[3];
  double L[3];
  float pad;
  const BoxSide *boxes;           // batched mode: device table indexed by box id, else null
  __device__ __forceinline__ BoxSide side(int box) const {
    if (boxes != nullptr) return boxes[box];
    BoxSide s;
    for (int k = 0; k < 3; ++k) { s.Lhi[k] = Lhi[k]; s.Llo[k] = Llo[k]; s.L[k] = L[k]; }
    return s;
  }
};

// Geometry of a launch, fixed at compile time so that the open and single-box paths carry no
// per-box data: open (no periodicity), one periodic box, or batched periodic boxes.
enum { GEOM_OPEN = 0, GEOM_BOX = 1, GEOM_BOXES = 2 };

template <int GEOM>
__device__ __forceinline__ BoxSide box_side(const BoxSplit &bx, int box) {
  if (GEOM == GEOM_BOXES) return bx.boxes[box];
  BoxSide s;
  for (int k = 0; k < 3; ++k) { s.Lhi[k] = bx.Lhi[k]; s.Llo[k] = bx.Llo[k]; s.L[k] = bx.L[k]; }
  return s;
}

inline int geom_of(const BoxSplit &bx) { return !bx.periodic ? GEOM_OPEN : (bx.boxes ? GEOM_BOXES : GEOM_BOX); }

// Canonical pair displacement x_a - x_b (minimum image in the pair's periodic box when
// periodic), identical bits whichever kernel computes it and antisymmetric in (a, b).
template <typename R>
__device__ __forceinline__ void pair_dx(const typename Vec<R>::v4 &Pa, const typename Vec<R>::v4 &La,
                                        const typename Vec<R>::v4 &Pb, const typename Vec<R>::v4 &Lb, int periodic,
                                        const BoxSide &bs, R &dx, R &dy, R &dz) {
  R hx = sub_rn(Pa.x, Pb.x), hy = sub_rn(Pa.y, Pb.y), hz = sub_rn(Pa.z, Pb.z);   // exact
  R lx = sub_rn(La.x, Lb.x), ly = sub_rn(La.y, Lb.y), lz = sub_rn(La.z, Lb.z);
  if (periodic) {
    if (sizeof(R) == 8) {  // float64 path: the box side is exact in double
      if (hx > (R)(0.5 * bs.L[0])) hx = sub_rn(hx, (R)bs.L[0]); else if (hx < (R)(-0.5 * bs.L[0])) hx = add_rn(hx, (R)bs.L[0]);
      if (hy > (R)(0.5 * bs.L[1])) hy = sub_rn(hy, (R)bs.L[1]); else if (hy < (R)(-0.5 * bs.L[1])) hy = add_rn(hy, (R)bs.L[1]);
      if (hz > (R)(0.5 * bs.L[2])) hz = sub_rn(hz, (R)bs.L[2]); else if (hz < (R)(-0.5 * bs.L[2])) hz = add_rn(hz, (R)bs.L[2]);
    } else {
      // hi differences in (L/2, L) minus the float side are exact (Sterbenz); the low part
      // of the side goes with lo
      const R L0 = (R)bs.Lhi[0], L1 = (R)bs.Lhi[1], L2 = (R)bs.Lhi[2];
      if (hx > (R)0.5 * L0) { hx = sub_rn(hx, L0); lx = sub_rn(lx, (R)bs.Llo[0]); }
      else if (hx < (R)-0.5 * L0) { hx = add_rn(hx, L0); lx = add_rn(lx, (R)bs.Llo[0]); }
      if (hy > (R)0.5 * L1) { hy = sub_rn(hy, L1); ly = sub_rn(ly, (R)bs.Llo[1]); }
      else if (hy < (R)-0.5 * L1) { hy = add_rn(hy, L1); ly = add_rn(ly, (R)bs.Llo[1]); }
      if (hz > (R)0.5 * L2) { hz = sub_rn(hz, L2); lz = sub_rn(lz, (R)bs.Llo[2]); }
      else if (hz < (R)-0.5 * L2) { hz = add_rn(hz, L2); lz = add_rn(lz, (R)bs.Llo[2]); }
    }
  }
  dx = add_rn(hx, lx);
  dy = add_rn(hy, ly);
  dz = add_rn(hz, lz);
}

template <typename R>
__device__ __forceinline__ R dist2_rn(R dx, R dy, R dz) {
  return add_rn(add_rn(mul_rn(dx, dx), mul_rn(dy, dy)), mul_rn(dz, dz));
}

// Pair predicate d_ab < h_a + h_b, evaluated as d^2 < (h_a + h_b)^2 with fixed rounding.
template <typename R>
__device__ __forceinline__ bool pair_test(R d2, R ha, R hb) {
  R r = add_rn(ha, hb);
  return d2 < mul_rn(r, r);
}

// ---- small utilities -----------------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(DMB_FULL, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(DMB_FULL, v, o));
  return v;
}

// 128-bit unsigned fixed point with 64 fractional bits: exact, order-independent sums of
// the Monte Carlo probabilities.
struct U128 {
  unsigned long long lo, hi;
};
__device__ __forceinline__ U128 u128_add(U128 a, U128 b) {
  U128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}
__device__ __forceinline__ bool u128_lt(U128 a, U128 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ U128 u128_shfl_xor(U128 a, int o) {
  U128 r;
  r.lo = __shfl_xor_sync(DMB_FULL, a.lo, o);
  r.hi = __shfl_xor_sync(DMB_FULL, a.hi, o);
  return r;
}
__device__ __forceinline__ U128 warp_sum_u128(U128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = u128_add(v, u128_shfl_xor(v, o));
  return v;
}
// Exact conversion of a non-negative float/double to the fixed-point format (values below
// 2^-64 of a unit truncate; values >= 2^63 saturate).
__device__ __forceinline__ U128 to_fixed(double p) {
  U128 r = {0ull, 0ull};
  if (!(p > 0.0)) return r;
  if (p >= 9.2233720368547758e18) { r.hi = 0x7fffffffffffffffull; r.lo = ~0ull; return r; }
  int e;
  double m = frexp(p, &e);                       // p = m 2^e, m in [0.5, 1)
  unsigned long long mant = (unsigned long long)ldexp(m, 53);   // 53-bit integer
  int sh = e - 53 + 64;                          // value = mant * 2^(e-53); fixed = value * 2^64
  if (sh >= 64) { r.hi = mant << (sh - 64); r.lo = 0; if (sh - 64 > 0) r.hi |= 0; }
  else if (sh > 0) { r.hi = mant >> (64 - sh); r.lo = mant << sh; }
  else if (sh > -64) { r.lo = mant >> (-sh); }
  return r;
}
// float version from the bits alone (no float64 or conversion instructions): p = m 2^(e-150)
// with the 24-bit significand m, so the fixed-point value is m << (e - 86).
__device__ __forceinline__ U128 to_fixed(float p) {
  U128 r = {0ull, 0ull};
  const uint32_t b = __float_as_uint(p);
  const int e = (int)((b >> 23) & 0xffu);
  if ((b >> 31) || e == 0) return r;              // negative, zero or subnormal
  if (e >= 255) { r.hi = 0x7fffffffffffffffull; r.lo = ~0ull; return r; }
  const unsigned long long m = (unsigned long long)((b & 0x7fffffu) | 0x800000u);
  const int sh = e - 86;
  if (sh > 103) { r.hi = 0x7fffffffffffffffull; r.lo = ~0ull; }   // >= 2^39: saturate
  else if (sh >= 64) r.hi = m << (sh - 64);
  else if (sh > 40) { r.lo = m << sh; r.hi = m >> (64 - sh); }
  else if (sh >= 0) r.lo = m << sh;
  else if (sh > -24) r.lo = m >> (-sh);
  return r;
}
__device__ __forceinline__ double fixed_to_double(U128 a) {
  return ldexp((double)a.hi, 0) + ldexp((double)a.lo, -64);
}
// floor(r * a) for a 64-bit fraction r = R 2^-64 and a fixed-point a.
__device__ __forceinline__ U128 u128_scale(unsigned long long R, U128 a) {
  U128 r;
  unsigned long long p_hi_lo = R * a.hi;
  unsigned long long p_hi_hi = __umul64hi(R, a.hi);
  unsigned long long p_lo_hi = __umul64hi(R, a.lo);
  r.lo = p_hi_lo + p_lo_hi;
  r.hi = p_hi_hi + (r.lo < p_hi_lo ? 1ull : 0ull);
  return r;
}
