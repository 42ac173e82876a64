// Kicks and float64 conservation sums.
#pragma once
#include "common.cuh"

#define KICK_THREADS 256
#define KICK_NSUM 6   // sum M a dt (3), gas energy change, u clamps, sum e_exp

cudaError_t launch_kick_gas(double *vel, double *T, const double *mu, const double *mass, const double *acc,
                            const double *dudt, const double *e_exp, int64_t n, double dt, double kT_over_mp,
                            double *block_sums, int blocks, cudaStream_t s, int64_t *launches,
                            const uint32_t *gate = nullptr);

// gate (device, may be null): when nonzero the kick changes nothing (a captured step that overflowed).
// Gather the per-block partials of the MC and kick kernels into the 16 step sums.
cudaError_t launch_final_sums(const double *mc_blocks, const double *mc_max, int mc_nb, const double *kick_blocks,
                              int kick_nb, double dt, double n_pairs, double *sums, cudaStream_t s,
                              int64_t *launches, const int64_t *n_pairs_dev = nullptr);

cudaError_t launch_pairs_out(const int64_t *row_ptr, const uint32_t *rows, const uint32_t *gas_perm,
                             const uint32_t *dm_perm, int64_t ng, int64_t capacity, uint32_t *out, cudaStream_t s,
                             int64_t *launches);
