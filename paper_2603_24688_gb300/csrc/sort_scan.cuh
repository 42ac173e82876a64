// Device-wide exclusive scan and LSD radix sort of (uint64 key, uint32 value) pairs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Exclusive scan of uint32 counts into int64 offsets, out has n + 1 entries (out[n] = total).
// tmp must hold scan_tmp_elems(n) int64 values.
int64_t scan_tmp_elems(int64_t n);
cudaError_t exclusive_scan_u32_i64(const uint32_t *in, int64_t *out, int64_t n, int64_t *tmp,
                                   cudaStream_t s, int64_t *launches);

// Stable LSD radix sort by the low `bits` bits of the keys, 8 bits per pass, ping-ponging
// between (k0, v0) and (k1, v1); the result ends in (k0, v0).  hist must hold
// radix_hist_elems(n) uint32 values and scan_tmp the matching scan scratch.
int64_t radix_hist_elems(int64_t n);
cudaError_t radix_sort_pairs(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t n, int bits,
                             uint32_t *hist, int64_t *hist_scan, int64_t *scan_tmp, cudaStream_t s,
                             int64_t *launches);
