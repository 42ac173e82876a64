// Exclusive scan and LSD radix sort written for this library (no CUB).
#include "sort_scan.cuh"

#define SCAN_BLOCK 1024
#define SCAN_ITEMS 4
#define SCAN_TILE (SCAN_BLOCK * SCAN_ITEMS)

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *smem_warp, T *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? smem_warp[lane] : (T)0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) smem_warp[lane] = w;
  }
  __syncthreads();
  const T warp_off = warp > 0 ? smem_warp[warp - 1] : (T)0;
  if (total) *total = smem_warp[nw - 1];
  __syncthreads();
  return warp_off + x - v;
}

// pass 1: per-tile sums
template <typename TIn>
__global__ void k_scan_tile_sums(const TIn *__restrict__ in, int64_t n, int64_t *__restrict__ sums) {
  __shared__ int64_t sw[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int64_t i = base + (int64_t)k * SCAN_BLOCK + threadIdx.x;
    if (i < n) s += (int64_t)in[i];
  }
  int64_t tot;
  block_exclusive_scan<int64_t>(s, sw, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// pass 2: exclusive scan of the tile sums in one block (looping over chunks)
__global__ void k_scan_sums(int64_t *__restrict__ sums, int64_t m) {
  __shared__ int64_t sw[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < m; base += SCAN_BLOCK) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < m ? sums[i] : 0;
    int64_t tot;
    const int64_t ex = block_exclusive_scan<int64_t>(v, sw, &tot);
    if (i < m) sums[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[m] = carry;
}

// pass 3: per-tile scan plus the tile offset (blocked: thread t owns SCAN_ITEMS consecutive)
template <typename TIn>
__global__ void k_scan_tiles(const TIn *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                             const int64_t *__restrict__ sums) {
  __shared__ int64_t sw[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = (base + k < n) ? (int64_t)in[base + k] : 0;
    s += v[k];
  }
  int64_t ex = block_exclusive_scan<int64_t>(s, sw, nullptr) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

int64_t scan_tmp_elems(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 2; }

template <typename TIn>
static cudaError_t exclusive_scan_impl(const TIn *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s,
                                       int64_t *launches) {
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    return cudaGetLastError();
  }
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  k_scan_tile_sums<TIn><<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(in, n, tmp);
  k_scan_sums<<<1, SCAN_BLOCK, 0, s>>>(tmp, tiles);
  k_scan_tiles<TIn><<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(in, out, n, tmp);
  if (launches) *launches += 3;
  return cudaGetLastError();
}

cudaError_t exclusive_scan_u32_i64(const uint32_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s,
                                   int64_t *launches) {
  return exclusive_scan_impl<uint32_t>(in, out, n, tmp, s, launches);
}

// ---- radix sort --------------------------------------------------------------------
#define RS_THREADS 256
#define RS_ITEMS 8
#define RS_TILE (RS_THREADS * RS_ITEMS)
#define RS_BINS 256

int64_t radix_hist_elems(int64_t n) { return (int64_t)RS_BINS * ((n + RS_TILE - 1) / RS_TILE) + 1; }

// digit-major histogram: hist[digit * tiles + tile]
__global__ void k_radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, uint32_t *__restrict__ hist,
                             int64_t tiles) {
  __shared__ uint32_t h[RS_BINS];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
  for (int k = 0; k < RS_ITEMS; ++k) {
    const int64_t i = base + (int64_t)k * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// stable scatter: items of a tile are ranked in index order (round k covers
// [base + k*256, base + k*256 + 256), within a round by thread index)
__global__ void k_radix_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
                                const int64_t *__restrict__ hscan, int64_t tiles) {
  __shared__ int64_t gbase[RS_BINS];
  __shared__ uint32_t run[RS_BINS];
  __shared__ uint32_t wcnt[RS_THREADS / 32][RS_BINS];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  gbase[t] = hscan[(int64_t)t * tiles + blockIdx.x];
  run[t] = 0;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int k = 0; k < RS_ITEMS; ++k) {
#pragma unroll
    for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][t] = 0;
    __syncthreads();
    const int64_t i = base + (int64_t)k * RS_THREADS + t;
    const bool valid = i < n;
    uint64_t key = 0;
    uint32_t val = 0;
    unsigned digit = 0;
    if (valid) {
      key = kin[i];
      val = vin[i];
      digit = (unsigned)(key >> shift) & 255u;
    }
    // lanes with equal digits; invalid lanes get distinct sentinels
    const unsigned tag = valid ? digit : (0x1000u + lane);
    const unsigned peers = __match_any_sync(0xffffffffu, tag);
    const unsigned rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
    __syncthreads();
    // per digit: exclusive prefix over warps, plus the running count of earlier rounds
    {
      uint32_t s = run[t];
#pragma unroll
      for (int w = 0; w < RS_THREADS / 32; ++w) {
        const uint32_t c = wcnt[w][t];
        wcnt[w][t] = s;
        s += c;
      }
      run[t] = s;
    }
    __syncthreads();
    if (valid) {
      const int64_t dst = gbase[digit] + wcnt[warp][digit] + rank;
      kout[dst] = key;
      vout[dst] = val;
    }
    __syncthreads();
  }
}

cudaError_t radix_sort_pairs(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t n, int bits,
                             uint32_t *hist, int64_t *hist_scan, int64_t *scan_tmp, cudaStream_t s,
                             int64_t *launches) {
  if (n <= 1) return cudaSuccess;
  const int64_t tiles = (n + RS_TILE - 1) / RS_TILE;
  int passes = (bits + 7) / 8;
  if (passes & 1) passes += 1;  // an even number of passes leaves the result in (k0, v0)
  uint64_t *ka = k0, *kb = k1;
  uint32_t *va = v0, *vb = v1;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_radix_hist<<<(unsigned)tiles, RS_THREADS, 0, s>>>(ka, n, shift, hist, tiles);
    cudaError_t e = exclusive_scan_u32_i64(hist, hist_scan, (int64_t)RS_BINS * tiles, scan_tmp, s, launches);
    if (e != cudaSuccess) return e;
    k_radix_scatter<<<(unsigned)tiles, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, hist_scan, tiles);
    if (launches) *launches += 2;
    uint64_t *tk = ka; ka = kb; kb = tk;
    uint32_t *tv = va; va = vb; vb = tv;
  }
  return cudaGetLastError();
}
