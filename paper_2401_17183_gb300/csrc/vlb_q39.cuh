// vlb_q39.cuh -- the D3Q39 velocity set: moment isotropy up to 6th order, as
// the paper asks for the full Navier-Stokes limit (Eq. 10), with T0 = 2/3, so
// that the equilibrium of Eq. 33 reproduces every moment of Eq. 32 including
// the third, Q^eq. Speeds reach 3 lattice units; this set runs on meshes whose
// axes are all periodic (halfway bounce-back is defined for one-cell links).
//
// Directions: 0 the rest vector, 1..19 the positive half listed in cpos()
// (the 3 unit axis vectors, the 4 corners with c^1 = +1, the 3 axis vectors of
// length 2, the 6 vectors (+-2, +-2, 0) and permutations with a positive first
// non-zero component, the 3 axis vectors of length 3), 20..38 their opposites
// in the same order (a + 19 = abar). Weights by |c|^2 = 0, 1, 3, 4, 8, 9:
// 1/12, 1/12, 1/27, 2/135, 1/432, 1/1620.
#pragma once

#include "vlb_internal.cuh"

namespace vlb {

template <>
struct Lat<39> {
  static constexpr int D = 3, H = 19;
  __host__ __device__ static constexpr int cpos(int a, int d) {
    // rows a = 1..19 of the positive half, three components each
    return d == 0 ? (a == 1 || (a >= 4 && a <= 7) ? 1 : a == 8 || (a >= 11 && a <= 14) ? 2 : a == 17 ? 3 : 0)
         : d == 1 ? (a == 2 || a == 4 || a == 5 ? 1 : a == 6 || a == 7 ? -1 : a == 9 || a == 11 || a == 15 || a == 16 ? 2
                     : a == 12 ? -2 : a == 18 ? 3 : 0)
                  : (a == 3 || a == 4 || a == 6 ? 1 : a == 5 || a == 7 ? -1 : a == 10 || a == 13 || a == 15 ? 2
                     : a == 14 || a == 16 ? -2 : a == 19 ? 3 : 0);
  }
  __host__ __device__ static constexpr int c(int a, int d) {
    return a == 0 ? 0 : a <= H ? cpos(a, d) : -cpos(a - H, d);
  }
};

constexpr double kT0_39 = 2.0 / 3.0;

__host__ __device__ constexpr int q39_c2(int a) {
  return Lat<39>::c(a, 0) * Lat<39>::c(a, 0) + Lat<39>::c(a, 1) * Lat<39>::c(a, 1) +
         Lat<39>::c(a, 2) * Lat<39>::c(a, 2);
}

__host__ __device__ constexpr double q39_w(int a) {
  return q39_c2(a) == 0   ? 1.0 / 12.0
         : q39_c2(a) == 1 ? 1.0 / 12.0
         : q39_c2(a) == 3 ? 1.0 / 27.0
         : q39_c2(a) == 4 ? 2.0 / 135.0
         : q39_c2(a) == 8 ? 1.0 / 432.0
                          : 1.0 / 1620.0;
}

// launches of the D3Q39 path (FP64 populations, periodic meshes)
cudaError_t q39_mesh_stats(const vlb_mesh *m, double *d_partial, int64_t nblk, cudaStream_t s);
// per-cell chord data of the force map into sim->d_coef (12 doubles per cell)
cudaError_t q39_prepare(const vlb_sim *sim, cudaStream_t s);
cudaError_t q39_init(const vlb_sim *sim, const double *d_rho, const double *d_u, cudaStream_t s);
cudaError_t q39_step(const vlb_sim *sim, int odd, cudaStream_t s);
cudaError_t q39_moments(const vlb_sim *sim, double *d_out, double *d_partial, int64_t nblk, cudaStream_t s);
cudaError_t q39_get_state(const vlb_sim *sim, double *d_N, cudaStream_t s);
cudaError_t q39_set_state(const vlb_sim *sim, const double *d_N, cudaStream_t s);

}  // namespace vlb
