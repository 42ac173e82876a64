// Hierarchical timesteps: particles carry a power-of-two timestep bin b (dt_i = 2^b dt_min) and
// are active at substep s when s mod 2^b == 0.  The active set of any substep is then the
// bins b <= nu(s) (nu the number of trailing zero bits of s), so ordering every species by
// (bin, sorted index) once makes each substep's active set a prefix of that list, with all of
// its sizes known on the host.
#pragma once
#include "grid.cuh"

#define DMB_NBINS 64   // bins 0 .. 63

// keys[s] = bin of sorted particle s (caller-order bins through perm), vals[s] = s; a bin
// above 63 raises DMB_BAD_VALUE.
cudaError_t launch_bin_keys(const uint8_t *bin, const uint32_t *perm, int64_t n, uint64_t *keys, uint32_t *vals,
                            uint32_t *status, cudaStream_t s, int64_t *launches);
// start[b] (b = 0 .. 64) = first position of the bin-sorted keys whose bin is >= b (start[64] = n).
cudaError_t launch_bin_bounds(const uint64_t *keys, int64_t n, int64_t *start, cudaStream_t s, int64_t *launches);
// For row k = list[k] of a CSR (row_ptr): its pair count and, when seg > 0, its number of
// segments of at most seg pairs (an empty row has none).
cudaError_t launch_list_counts(const uint32_t *list, int64_t n, const int64_t *row_ptr, int seg, uint32_t *len,
                               uint32_t *segs, cudaStream_t s, int64_t *launches);
// Segment table of the listed rows: seg_row[u] = list[k], seg_begin[u] = row start + (u - seg_ptr[k]) seg.
cudaError_t launch_list_seg_map(const uint32_t *list, int64_t n, const int64_t *row_ptr, const int64_t *seg_ptr,
                                int seg, uint32_t *seg_row, int64_t *seg_begin, cudaStream_t s, int64_t *launches);
// out[b] = arr[start[b]] for b = 0 .. 64.
cudaError_t launch_pick(const int64_t *arr, const int64_t *start, int64_t *out, cudaStream_t s, int64_t *launches);

// Kick of the active gas of a substep: row k is sorted gas list[k] (caller index perm[list[k]])
// with dt_j = 2^bin dt_min; the caller's V and T are updated (u clamped at 0), the sorted copies
// V = (v, varsigma) and K are refreshed for the next substep, and the block partials of the
// kick sums are written as by the full-step kick.
template <typename R>
cudaError_t launch_kick_gas_list(double *vel, double *T, const double *mu, const double *mass, const double *acc,
                                 const double *dudt, const double *e_exp, const uint32_t *list, int64_t n_list,
                                 const uint32_t *perm, const uint8_t *bin, double dt_min, RunConst rc,
                                 typename Vec<R>::v4 *Vs, typename Vec<R>::v4 *Ks, double *block_sums, int blocks,
                                 cudaStream_t s, int64_t *launches);

// Device step counter of captured substeps: set it, or advance it by one (the last launch of a
// captured substep, so that the next replay runs the next substep).
cudaError_t launch_step_set(unsigned long long *step, unsigned long long value, cudaStream_t s, int64_t *launches);
cudaError_t launch_step_advance(unsigned long long *step, cudaStream_t s, int64_t *launches);

// New timestep bins of n particles from the criterion ratios of Eq. prob_criterion (the rule of
// dmb_rebin_dm); *changed (device) is increased by the number of bins that moved.
cudaError_t launch_rebin(const float *ratio, uint8_t *bin, int64_t n, int max_bin, unsigned long long substep,
                         const uint8_t *active, unsigned long long *changed, cudaStream_t s, int64_t *launches);
