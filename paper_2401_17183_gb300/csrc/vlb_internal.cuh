// vlb_internal.cuh -- shared internals of libvlb (device lattice tables, the
// per-cell collision of section 2.2, mesh/simulation objects and launcher
// declarations). Not part of the public C-ABI (include/vlb.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/vlb.h"

namespace vlb {

// --------------------------------------------------------------------------
// Velocity sets. Section 2.1 lists D3Q19 {0, +-e_i, +-e_i +-e_j}; D2Q9 is its
// planar restriction. The library orders each set so that the opposite of
// direction a (1 <= a <= H) is a + H, which lets every kernel treat the
// (a, abar) pair as one unit.
//   D2Q9 : 1 (1,0) 2 (0,1) 3 (1,1) 4 (-1,1)           and their negatives
//   D3Q19: 1 (1,0,0) 2 (0,1,0) 3 (0,0,1) 4 (1,1,0) 5 (1,-1,0) 6 (1,0,1)
//          7 (1,0,-1) 8 (0,1,1) 9 (0,1,-1)             and their negatives
// Weights: the standard ones with T0 = 1/3 (they meet Eq. 10 to 4th order).
template <int Q>
struct Lat;

template <>
struct Lat<9> {
  static constexpr int D = 2, H = 4;
  // positive half, a = 1..4
  __host__ __device__ static constexpr int cpos(int a, int d) {
    return d == 0 ? (a == 1 || a == 3 ? 1 : a == 4 ? -1 : 0) : d == 1 ? (a == 1 ? 0 : 1) : 0;
  }
  __host__ __device__ static constexpr int c(int a, int d) {
    return a == 0 ? 0 : a <= H ? cpos(a, d) : -cpos(a - H, d);
  }
};

template <>
struct Lat<19> {
  static constexpr int D = 3, H = 9;
  // positive half, a = 1..9
  __host__ __device__ static constexpr int cpos(int a, int d) {
    return d == 0   ? (a == 1 || a == 4 || a == 5 || a == 6 || a == 7 ? 1 : 0)
           : d == 1 ? (a == 2 || a == 4 || a == 8 || a == 9 ? 1 : a == 5 ? -1 : 0)
                    : (a == 3 || a == 6 || a == 8 ? 1 : a == 7 || a == 9 ? -1 : 0);
  }
  __host__ __device__ static constexpr int c(int a, int d) {
    return a == 0 ? 0 : a <= H ? cpos(a, d) : -cpos(a - H, d);
  }
};

template <int Q>
__host__ __device__ constexpr int lat_nnz(int a) {
  return (Lat<Q>::c(a, 0) != 0) + (Lat<Q>::c(a, 1) != 0) + (Lat<Q>::c(a, 2) != 0);
}

// the k-th non-zero component axis of c_a (k = 0, 1), or -1
template <int Q>
__host__ __device__ constexpr int nz_axis(int a, int k) {
  int n = 0;
  for (int i = 0; i < 3; i++)
    if (Lat<Q>::c(a, i) != 0) {
      if (n == k) return i;
      n++;
    }
  return -1;
}

template <int Q, typename R>
__host__ __device__ constexpr R lat_w(int a) {
  return Q == 9 ? (a == 0 ? R(4) / R(9) : lat_nnz<Q>(a) == 1 ? R(1) / R(9) : R(1) / R(36))
                : (a == 0 ? R(1) / R(3) : lat_nnz<Q>(a) == 1 ? R(1) / R(18) : R(1) / R(36));
}

template <int Q>
__host__ __device__ constexpr int lat_opp(int a) {
  return a == 0 ? 0 : (a <= Lat<Q>::H ? a + Lat<Q>::H : a - Lat<Q>::H);
}

// index of the symmetric pair (i, j) in a packed D(D+1)/2 array
template <int D>
__host__ __device__ constexpr int sym(int i, int j) {
  return D == 2 ? i + j : (i < j ? i : j) == 0 ? (i > j ? i : j) : (i < j ? i : j) == 1 ? 2 + (i > j ? i : j) : 5;
}

// index of the ordered off-diagonal pair (k, l), k != l, in a D(D-1) array
template <int D>
__host__ __device__ constexpr int offd(int k, int l) {
  return k * (D - 1) + (l < k ? l : l - 1);
}

// --------------------------------------------------------------------------
// Coefficient record of one cell (or one column in plane mode). Records are
// stored one after another (record r at coef + r * RS). Everything in a
// record is a function of the cell geometry and tau alone, formed once in
// FP64 and rounded to the storage type. The record falls into groups, each
// starting on a multiple of four elements (16 bytes or more), so that a
// group can be read with vector loads: the set-up of a collision, the link
// coefficients, the chord matrix and the coefficients of one evaluation of
// the map.
//
// Link coefficients are stored per pair (p, pbar = p + H) as
// am M_p and ad D_p with M_p = K_p + K_pbar, D_p = K_p - K_pbar and the weights
// am = -(2 - 1/tau)/4, ad = (1/tau)/4 that they carry in the constant part
// of the map (see collide_cell): components 0 and 1 of pair p as one 16-byte
// quad (am M^0, am M^1, ad D^0, ad D^1), then (D = 3) the component-2 pairs
// (am M^2, ad D^2). The last group holds the coefficients of the fixed-point
// map of Eq. 27 written as a polynomial in U~, premultiplied by the chord
// matrix (see build_record), so that one chord step costs a few dozen products
// instead of a pass over all directions.
__host__ __device__ constexpr int round4(int n) { return (n + 3) / 4 * 4; }
__host__ __device__ constexpr int round2(int n) { return (n + 1) / 2 * 2; }

template <int Q>
struct CoefLayout {
  static constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
  static constexpr int NS = D * (D + 1) / 2;   // symmetric pairs
  static constexpr int NO = D * (D - 1);       // ordered off-diagonal pairs
  static constexpr int NQ = NS + NO;           // monomials of U~ in one chord step
  // set-up of a collision
  static constexpr int J = 0;                  // J (Eq. 5)
  static constexpr int GH = 1;                 // (g^ij - delta^ij) / 2 packed (Eq. 8)
  static constexpr int BODY = GH + NS;         // G^i = G . g^i
  static constexpr int KW = BODY + D;          // sum_a w_a K^i_a (reference-state part of J F)
  static constexpr int KWL = KW + D;           // its low part: KW + KWL = the FP64 value
  static constexpr int FR = KWL + D;           // F of the rest state at rho = 1 (start value)
  static constexpr int CE = FR + D;            // constant term of the map
  static constexpr int PO1 = CE + D;           // D x D: coefficient of U (row-major)
  static constexpr int IJ = PO1 + D * D;       // 1 / J
  // link coefficients (see above)
  static constexpr int MPD = round4(IJ + 1);
  // blocks of D rows (component i of Phi) of n coefficients each, stored with
  // rows 0 and 1 interleaved (k-th pair at base + 2k, 8-byte aligned, for
  // packed FP32 arithmetic) and row 2 after them (see row())
  static constexpr int HM = round4(MPD + 2 * H * D);  // D x D: chord matrix (I - L)^-1 minus I
  // H PE and H PO2 side by side: column s < NS is the coefficient of
  // U~^k U~^l (s = sym(k, l)), column NS + offd(k, l) that of (U~^k)^2 U~^l
  static constexpr int QM = round4(HM + round2(D * D));
  // element k of row i of the block that starts at base and has n per row
  __host__ __device__ static constexpr int row(int base, int n, int i, int k) {
    return i < 2 ? base + 2 * k + i : base + 2 * n + (i - 2) * n + k;
  }
  // the local rest state (rho = 1, U = 0) of Eq. 33, for the final pass:
  // RR + p (p = 0..H) its deviation from the uniform reference,
  // J w_p (1 + x_p) - w_p n_ref (even in the direction), RR + H + 1 the sum of
  // those deviations over all Q directions, and RW + p the weight of the rest
  // state, w_p (1 + x_p). Both follow from J and g^ij; with one record per
  // cell the step recomputes them rather than streaming them (see
  // rest_state), so a per-cell record is read up to RR only.
  static constexpr int RR = round4(QM + D * NQ);
  static constexpr int RW = RR + round4(H + 2);
  // wall velocity U_w^i (read in the wall cells of moving walls only), in the
  // padding after the chord matrix or after the map coefficients, so that a
  // per-cell record ends at RR
  static constexpr int UW = QM - (HM + D * D) >= D   ? HM + D * D
                            : RR - (QM + D * NQ) >= D ? QM + D * NQ
                                                      : -1;
  static_assert(UW >= 0, "no padding gap holds the wall velocity");
  // 16-bit populations relative to the rest state (reference VLB_REF_REST,
  // plane mode). A location (slot, cell) holding a population of direction a
  // stores N_a - o_a, o_a = J w_a (1 + x_a) of the column that holds the
  // location, rounded to FP32 (even in the direction). The collision then
  // works on e_a = N_a - o_a(own column) directly; it needs
  //   SR + i  sum_p am M^i_p 2 (o_p - w_p n_ref), the part of the pair sums
  //           of the deviations that the rest state carries,
  //   MDV     sum_a (o_a - w_a n_ref), so that m - n_ref = sum_a e_a + MDV,
  //   MNV     sum_a o_a - J, so that m - J = sum_a e_a + MNV,
  // and, for odd steps, the differences to the columns that a population is
  // read from (slot abar of q - c_a) and written to (slot a of q + c_a):
  //   DIN + a   o_a(column of q - c_a) - o_a(own),
  //   DOUT + a  o_a(own) - o_a(column of q + c_a),
  // both zero for a link through a wall (the cell's own slot). Kernels that
  // do not read 16-bit rest-relative populations stage the record up to SREST.
  static constexpr int SREST = round4(RW + H + 1);
  static constexpr int SR = SREST;
  static constexpr int MDV = SR + D;
  static constexpr int MNV = MDV + 1;
  static constexpr int DIN = round4(MNV + 1);
  static constexpr int DOUT = DIN + Q;
  static constexpr int NC = DOUT + Q;
  __host__ __device__ static constexpr int mp(int p, int i) {
    return i < 2 ? MPD + 4 * (p - 1) + i : MPD + 4 * H + 2 * (p - 1);
  }
  __host__ __device__ static constexpr int dk(int p, int i) {
    return i < 2 ? MPD + 4 * (p - 1) + 2 + i : MPD + 4 * H + 2 * (p - 1) + 1;
  }
  // record stride in elements of type R: a multiple of four elements, so that
  // every record and group starts on a 16-byte boundary. One record per
  // column (PLANE) holds everything; one record per cell ends at RR (the rest
  // state is formed from J and g^ij, the 16-bit rest-relative block needs
  // plane mode), which for D3Q19 FP32 is 544 bytes, 17 whole 32-byte sectors.
  template <typename R, bool PLANE = true>
  static constexpr int stride() {
    return PLANE ? round4(NC) : RR;
  }
};

constexpr double kT0 = 1.0 / 3.0;

// max that propagates NaN from either side (a NaN residual never converges);
// FP32 in one instruction (PTX max.NaN)
template <typename R>
__device__ __forceinline__ R maxnan(R a, R b) {
  return (a > b || a != a) ? a : b;
}
template <>
__device__ __forceinline__ float maxnan<float>(float a, float b) {
  float r;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float absr(float x) { return fabsf(x); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double absr(double x) { return fabs(x); }

// population storage types: FP64, FP32, IEEE half, bfloat16
template <typename R, typename S>
__device__ __forceinline__ R load_s(S x) {
  return static_cast<R>(x);
}
template <>
__device__ __forceinline__ float load_s<float, __half>(__half x) {
  return __half2float(x);
}
template <>
__device__ __forceinline__ double load_s<double, __half>(__half x) {
  return (double)__half2float(x);
}
template <>
__device__ __forceinline__ float load_s<float, __nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}
template <>
__device__ __forceinline__ double load_s<double, __nv_bfloat16>(__nv_bfloat16 x) {
  return (double)__bfloat162float(x);
}
template <typename S, typename R>
__device__ __forceinline__ S store_s(R x) {
  return static_cast<S>(x);
}
template <>
__device__ __forceinline__ __half store_s<__half, float>(float x) {
  return __float2half_rn(x);
}
template <>
__device__ __forceinline__ __half store_s<__half, double>(double x) {
  return __double2half(x);
}
template <>
__device__ __forceinline__ __nv_bfloat16 store_s<__nv_bfloat16, float>(float x) {
  return __float2bfloat16_rn(x);
}
template <>
__device__ __forceinline__ __nv_bfloat16 store_s<__nv_bfloat16, double>(double x) {
  return __double2bfloat16(x);
}

// --------------------------------------------------------------------------
// Equilibrium of Eq. 33 for one cell, specialised to velocity sets whose
// components are in {-1, 0, 1}. With
//   B^ij  = (g^ij - delta^ij) T0 + U~^i U~^j,
//   C^ijk = T0 [(g^ij U~^k - delta^ij U^k) + cyclic] + U~^i U~^j U~^k,
// the bracket of Eq. 33 is
//   1 + c.U/T0 + (c.B.c/T0 - tr B)/(2 T0) + (C[c,c,c] - 3 T0 c^i C^ijj)/(6 T0^3).
// On such sets (c^k)^3 = c^k, and the last term reduces to
//   (9/2) sum_{k != l} C^kkl c^l (3 (c^k)^2 - 1):
// the C^kkk terms of C[c,c,c] and of c^i C^ijj cancel, and C^123 never meets
// a velocity with three non-zero components on D3Q19. So only C^kkl (k != l)
// is formed. The struct holds the direction-independent parts.
template <int Q, typename R>
struct EqParts {
  static constexpr int D = Lat<Q>::D;
  R B[D][D];
  R trB;
  R C2[D][D];   // C2[k][l] = C^kkl, k != l
};

template <int Q, typename R>
__device__ __forceinline__ void eq_parts(const R (&gd)[Lat<Q>::D * (Lat<Q>::D + 1) / 2],
                                         const R (&U)[Lat<Q>::D], const R (&dU)[Lat<Q>::D],
                                         EqParts<Q, R> &e) {
  // gd = g^ij - delta^ij and U~ = U + dU; every difference of large terms is
  // written out so that only small quantities are rounded
  constexpr int D = Lat<Q>::D;
  const R T0 = R(kT0);
  R Ut[D];
#pragma unroll
  for (int i = 0; i < D; i++) Ut[i] = U[i] + dU[i];
  e.trB = R(0);
#pragma unroll
  for (int i = 0; i < D; i++)
#pragma unroll
    for (int j = 0; j < D; j++) e.B[i][j] = gd[sym<D>(i, j)] * T0 + Ut[i] * Ut[j];
#pragma unroll
  for (int i = 0; i < D; i++) e.trB += e.B[i][i];
#pragma unroll
  for (int i = 0; i < D; i++) {
#pragma unroll
    for (int j = 0; j < D; j++) {
      if (i == j) continue;
      // C^iij = T0 [(g^ii U~^j - U^j) + 2 g^ij U~^i] + U~^i U~^i U~^j
      e.C2[i][j] = T0 * ((gd[sym<D>(i, i)] * Ut[j] + dU[j]) + R(2) * gd[sym<D>(i, j)] * Ut[i]) +
                   Ut[i] * Ut[i] * Ut[j];
    }
  }
}

// even part of the bracket of Eq. 33 (terms with an even power of c) for
// direction a. Called inside fully unrolled loops, so a and every c(a, i) are
// compile-time constants and the zero terms fold away.
template <int Q, typename R>
__device__ __forceinline__ R eq_even(const EqParts<Q, R> &e, int a) {
  constexpr int D = Lat<Q>::D;
  R cbc = R(0);
#pragma unroll
  for (int i = 0; i < D; i++) {
    const int ci = Lat<Q>::c(a, i);
    if (ci == 0) continue;
#pragma unroll
    for (int j = 0; j < D; j++) {
      const int cj = Lat<Q>::c(a, j);
      if (cj == 0) continue;
      if (ci * cj > 0)
        cbc += e.B[i][j];
      else
        cbc -= e.B[i][j];
    }
  }
  return R(1) + (R(3) * cbc - e.trB) * R(1.5);
}

// odd part of the bracket of Eq. 33 for direction a:
//   c.U / T0 + (9/2) sum_{k != l} C^kkl c^l (3 (c^k)^2 - 1)
template <int Q, typename R>
__device__ __forceinline__ R eq_odd(const EqParts<Q, R> &e, const R (&U)[Lat<Q>::D], int a) {
  constexpr int D = Lat<Q>::D;
  R cu = R(0), cc = R(0);
#pragma unroll
  for (int l = 0; l < D; l++) {
    const int cl = Lat<Q>::c(a, l);
    if (cl == 0) continue;
    cu += cl > 0 ? U[l] : -U[l];
#pragma unroll
    for (int k = 0; k < D; k++) {
      if (k == l) continue;
      // 3 (c^k)^2 - 1 is 2 for an in-plane k and -1 otherwise
      const int f = Lat<Q>::c(a, k) != 0 ? 2 : -1;
      cc += R(f * cl) * e.C2[k][l];
    }
  }
  return R(3) * cu + R(4.5) * cc;
}

// Storage reference of population a at a cell: with VLB_REF_REST the rest
// state of Eq. 33 on the cell's metric, J w_a (1 + even part at U = 0), rounded
// to FP32 (every kernel that stores or reads 16-bit populations uses this one
// value); else w_a n_ref. ginv is the cell's packed g^ij.
template <int Q>
__device__ __forceinline__ double rest_ref(double J, const double *ginv, int a) {
  constexpr int D = Lat<Q>::D, NS = D * (D + 1) / 2;
  double gd[NS], z[D];
#pragma unroll
  for (int i = 0; i < NS; i++) gd[i] = ginv[i];
#pragma unroll
  for (int i = 0; i < D; i++) {
    gd[sym<D>(i, i)] -= 1.0;
    z[i] = 0.0;
  }
  EqParts<Q, double> e;
  eq_parts<Q, double>(gd, z, z, e);
  const int p = a <= Lat<Q>::H ? a : a - Lat<Q>::H;
  return (double)(float)(J * lat_w<Q, double>(a) * eq_even<Q, double>(e, p));
}

// Where the storage reference of a location comes from (kernels outside the
// time step, which read populations by location).
struct RefCtx {
  int32_t rest;          // VLB_REF_REST in use
  double nref;           // uniform reference
  const double *J;       // FP64 geometry (rest)
  const double *ginv;
  int64_t nfast;         // plane mode: a column's geometry is that of its first cell
};

template <int Q>
__device__ __forceinline__ double ref_at(const RefCtx &r, int slot, int64_t cell) {
  if (!r.rest) return lat_w<Q, double>(slot) * r.nref;
  constexpr int NS = Lat<Q>::D * (Lat<Q>::D + 1) / 2;
  const int64_t c0 = (cell / r.nfast) * r.nfast;
  return rest_ref<Q>(r.J[c0], r.ginv + c0 * NS, slot);
}

// --------------------------------------------------------------------------
// Mesh and simulation objects (host side).
struct MeshDev {
  int32_t dim;
  int32_t q;
  int64_t n[3];
  int32_t bc[3];
  double shift[3][3];
  double rot[3][9];
  int32_t has_rot[3];
  double dx;
  int32_t wall_links;  // VLB_WALL_LINKS_ZERO or VLB_WALL_LINKS_GHOST
  const double *x;     // device positions
};

}  // namespace vlb

struct vlb_mesh {
  vlb::MeshDev md;
  int64_t ncell;
  double *d_x = nullptr;
  double *d_J = nullptr;     // [ncell]
  double *d_gl = nullptr;    // [ncell][dim][dim]
  double *d_gu = nullptr;    // [ncell][dim][dim]
  double *d_ginv = nullptr;  // [ncell][NS]
  double *d_K = nullptr;     // [ncell][q][dim]
  vlb_mesh_stats stats;
  int device = 0;
};

struct vlb_sim {
  const vlb_mesh *mesh = nullptr;
  vlb_params p;
  cudaStream_t stream = nullptr;
  void *d_f = nullptr;        // populations [q][ncell]
  void *d_coef = nullptr;     // coefficient records, record r at r * nc elements
  int64_t ncoef = 0;
  int32_t nc = 0;
  int32_t plane = 0;
  int64_t t = 0;
  double nref = 0.0;          // populations are stored as N_a - w_a nref, nref = rho_0 J_ref
  int32_t ref_rest = 0;       // 16-bit storage relative to the local rest state
  int *d_err = nullptr;       // sticky kernel error flags
  double *d_fields = nullptr; // moments output staging: rho [ncell], u and u~ [ncell][dim]
  double *d_partial = nullptr;
  double *d_totals = nullptr;
  int64_t partial_blocks = 0;
  double *d_io = nullptr;     // host<->device staging for init/state, grown on demand
  size_t io_bytes = 0;
};

struct vlb_batch {
  std::vector<vlb_sim *> sims;
  cudaStream_t stream = nullptr;
  int device = 0;
  int64_t run = 0;            // tiles per block
  int64_t nitems = 0;         // blocks per launch
  int64_t cells = 0;
  void *d_args = nullptr;     // StepArgs[nsims]
  void *d_items = nullptr;    // BatchItem[nitems]
  size_t items_cap = 0;
  cudaGraphExec_t graph = nullptr;  // 32 launches, even parity first
  int64_t graph_run = 0;      // run length the graph was built for
  int32_t shape = 0;          // block shape (index into the batch's shape table)
  int32_t graph_shape = -1;   // shape the graph was built for
};

namespace vlb {

// storage type of a precision, as a type tag for generic host dispatch
template <typename T>
struct TypeTag {
  using type = T;
};
template <typename F>
inline auto with_storage(int32_t precision, F &&fn) {
  switch (precision) {
    case VLB_F64: return fn(TypeTag<double>{});
    case VLB_F16: return fn(TypeTag<__half>{});
    case VLB_BF16: return fn(TypeTag<__nv_bfloat16>{});
    default: return fn(TypeTag<float>{});
  }
}
inline size_t storage_bytes(int32_t precision) {
  return precision == VLB_F64 ? 8 : precision == VLB_F32 ? 4 : 2;
}
// arithmetic (and coefficient) type: FP64 only for VLB_F64
inline bool arith_f64(int32_t precision) { return precision == VLB_F64; }

inline RefCtx make_ref(const vlb_sim *sim) {
  RefCtx r;
  r.rest = sim->ref_rest;
  r.nref = sim->nref;
  r.J = sim->mesh->d_J;
  r.ginv = sim->mesh->d_ginv;
  r.nfast = sim->plane ? sim->mesh->md.n[sim->mesh->md.dim - 1] : 1;
  return r;
}

// error flags raised by kernels
enum : int { ERR_NOCONV = 1, ERR_NONFINITE = 2, ERR_GEOM = 4 };

// launchers (each returns a cudaError_t from the launch)
cudaError_t launch_geometry(const vlb_mesh *m, int *d_err, cudaStream_t s);
cudaError_t launch_mesh_stats(const vlb_mesh *m, double *d_partial, int64_t nblk, cudaStream_t s);
cudaError_t launch_plane_check(const vlb_mesh *m, int *d_flag, cudaStream_t s);
cudaError_t launch_pack_coef(const vlb_sim *sim, cudaStream_t s);
cudaError_t launch_init(const vlb_sim *sim, const double *d_rho, const double *d_u, cudaStream_t s);
cudaError_t launch_step(const vlb_sim *sim, int odd, cudaStream_t s);
cudaError_t launch_moments(const vlb_sim *sim, double *d_out, int64_t nblk, cudaStream_t s);
// conservation totals (mass, P, M) of a D2Q9/D3Q19 simulation into d_totals[7]
// through per-block partial sums in d_partial (room for nblk_max x 7 doubles)
cudaError_t launch_totals(const vlb_sim *sim, double *d_partial, int64_t nblk_max, double *d_totals,
                          cudaStream_t s);
cudaError_t launch_finish_totals(const double *d_partial, int64_t nblk, double *d_totals,
                                 cudaStream_t s);
cudaError_t launch_get_state(const vlb_sim *sim, double *d_N, cudaStream_t s);
cudaError_t launch_set_state(const vlb_sim *sim, const double *d_N, cudaStream_t s);

// records a thread-local error message for vlb_last_error() and returns code
int set_error(int code, const char *fmt, ...);

constexpr int kMomThreads = 256;
constexpr int kStatThreads = 256;

}  // namespace vlb
