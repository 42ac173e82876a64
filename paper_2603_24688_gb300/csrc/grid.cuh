// Spatial index: shared frame, Morton keys, sorted float copies, chunk tree.
#pragma once
#include "common.cuh"

struct Frame {
  double origin[3];
  double span;       // side of the cube holding all particles (periodic: max box side)
  double delta;      // power of two with span <= 2^23 delta: quantum of the hi parts
  double inv_delta;  // 1 / delta (exact)
  double key_scale;  // 2^bits / span
  float pad;         // padding of tree boxes (covers float rounding of the coordinates)
  int bits;          // Morton bits per axis
  double hmax_dm, hmax_gas;
};

// Physical constants of a run, precomputed on the host in float64.
struct RunConst {
  double S;          // sigma0 [kpc^2] * Msun / m_p
  double m_chi;      // m_chi / m_p
  double v0;         // km/s
  double alpha;      // alpha_n = 2^((n+5)/2) Gamma(3 + n/2) / sqrt(pi)
  double kT_over_mp; // k_B / m_p in (km/s)^2 / K
  int n;
  int rate_mode;     // dmb_rate_mode
  // sigma_bar / sigma: the gas exchange rates take the momentum-transfer cross section,
  // 1 - beta / 3 for dsigma/dOmega proportional to 1 + beta cos theta (1 when isotropic)
  double sbar = 1.0;
  // velocity law of sigma: 0 the power law sigma0 (v / v0)^n; 1 the screened law
  // sigma0 / (1 + (v / v_c)^2)^2, whose runs carry n = 0 and alpha = alpha_0 (the App. B
  // normalisation of the n = 0 closed forms), so that FA, FB become functions of x and
  // varsigma^2 / v_c^2 and the gas coefficients keep their n = 0 form
  int xsec = 0;
  double inv_vc2 = 0.0;   // 1 / v_c^2, (km/s)^-2 (0 for the power law)
};

// Per-gas coefficients of the sorted copy K = (cA, cB, kP0, e) from varsigma (km/s), the gas
// particle mass M (Msun) and mu (m_p): a_j = cA sum M_i g FA w and du_j/dt = cA sum M_i g FA w^2
// - cB sum M_i g FB with the normalised rates FA, FB (Eqs. gas-dVdt, gas-dTdt and the App. B
// closed forms), kP0 = (M_j / mu_j) sigma0 of Eq. dm-update-prob and e = mu_j / (m_chi + mu_j).
__host__ __device__ inline void gas_coeffs(const RunConst &rc, double sig, double M, double mu, double &cA,
                                           double &cB, double &kP0, double &e) {
  // float64 division and pow are slow on this GPU (its float64 pipe runs at about 1/70 of
  // float32): one reciprocal per particle and an integer power by squaring
  const double inv_mpm = 1.0 / (rc.m_chi + mu);
  e = mu * inv_mpm;
  if (sig > 0.0) {
    const double r = sig / rc.v0;
    double sn = 1.0, b = r;                                    // (varsigma / v0)^|n|
    for (int k = rc.n < 0 ? -rc.n : rc.n; k > 0; k >>= 1) {
      if (k & 1) sn *= b;
      b *= b;
    }
    if (rc.n < 0) sn = 1.0 / sn;
    const double t = rc.S * rc.sbar * rc.alpha * sn * sig * inv_mpm;
    cA = t / 3.0;
    cB = t * sig * sig * e;
  } else {  // cold gas: A = sigma(w) w, B = sigma(w) w^3
    cA = rc.S * rc.sbar * inv_mpm;
    cB = cA * e;
  }
  kP0 = M / mu * rc.S;                                         // (M_j / mu_j) sigma0 Msun/m_p
}

// Batched boxes: per-box parameters used by the key and gather kernels (device table).
struct BoxParamDev {
  double L[3];        // periodic sides, kpc
  double S;           // sigma0 [kpc^2] * Msun / m_p of this box
  double m_chi;       // m_chi / m_p of this box
  double offset_x;    // x offset of the box's slot in the shared virtual space
};

struct BatchArgs {
  const uint32_t *box_of;       // caller: box index per particle (null: single box)
  const BoxParamDev *bp;        // device table
  int box_bits;                 // bits of the box index in the key
};

// Status bits raised by the device checks.
enum : uint32_t {
  DMB_BAD_VALUE = 1u,      // NaN / Inf or a non-positive h, M, mu, or negative T
  DMB_BAD_PERIODIC = 2u,   // h_i + h_j >= box / 2 (minimum image ambiguous)
  DMB_BAD_DOMAIN = 4u,     // rate provider outside its domain
  DMB_BAD_OVERFLOW = 8u,   // a pair list or stack overflowed
  DMB_BAD_TIMEOUT = 16u,   // a bounded wait on the tensor cores gave up
};

cudaError_t launch_frame(const double *dm_pos, const double *dm_h, int64_t ndm, const double *gas_pos,
                         const double *gas_h, int64_t ngas, int periodic, const double box[3], double *part,
                         int64_t part_elems, Frame *frame, uint32_t *status, cudaStream_t s, int64_t *launches);

cudaError_t launch_morton(const double *pos, int64_t n, int periodic, const double box[3], const Frame *frame,
                          BatchArgs ba, uint64_t *keys, uint32_t *vals, cudaStream_t s, int64_t *launches);

template <typename R>
cudaError_t launch_gather(const double *pos, const double *vel, const double *mass, const double *h,
                          const double *T, const double *mu, const uint32_t *id, int64_t n, const uint32_t *perm,
                          int periodic, const double box[3], const Frame *frame, RunConst rc, BatchArgs ba,
                          typename Vec<R>::v4 *P, typename Vec<R>::v4 *L, typename Vec<R>::v4 *V,
                          typename Vec<R>::v4 *K, uint32_t *sid, uint16_t *bid, uint32_t *status, cudaStream_t s,
                          int64_t *launches);

// Level layout of the 32-ary tree for n particles; returns the number of nodes.
int tree_layout(int64_t n, int *levels, int off[DMB_MAX_LEVELS], int cnt[DMB_MAX_LEVELS]);

template <typename R>
cudaError_t launch_tree(const typename Vec<R>::v4 *P, const typename Vec<R>::v4 *L, int64_t n, const Frame *frame,
                        float4 *bmin, float4 *bmax, int levels, const int *off, const int *cnt, const uint16_t *bid,
                        int2 *leaf_box, cudaStream_t s, int64_t *launches);
