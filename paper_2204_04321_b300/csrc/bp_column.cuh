// Per-column assembly body shared by the single-mesh kernel and the ensemble's persistent kernel.
// Fused finite-element assembly of the first-order Stokes residual and Jacobian
// (paper Sec. 3.2: Gather -> Interpolate -> Evaluate -> Scatter, here one kernel).
//
// One thread walks one column of wedges (a base triangle times all layers) from the bed up.
// The value path is FP64 and uses the extruded structure of the wedge: x, y do not depend
// on zeta, so for N_{a,k} = lambda_a(xi, eta) psi_k(zeta)
//     grad N_{a,k} = psi_k Lambda_a + lambda_a psi_k' Z,   Z = grad zeta = (2/h)(-grad z|zeta, 1),
// with Lambda_a the constant 2D gradient of the barycentric coordinate, h the local layer
// thickness and grad z|zeta the (constant) slope of the zeta-level surface.  The velocity
// gradient at a quadrature point is then
//     u_z = sum_a lambda_a (u_top - u_bot)_a / h,   u_xy = grad_2D u(zeta) - u_z grad z|zeta.
// Sums over the 6 quadrature points are factored into sums over the 2 zeta levels and the 3
// triangle points.  Values shared by consecutive wedges of a column (the level velocities
// and their 2D gradients, the top-face residual) are carried in registers.
//
// Jacobian (Sec. 3.2; the paper differentiates with forward-mode dual numbers, SFad):
//   K_ij = sum_q c_q [eta B^{c_i c_j}(grad N_i, grad N_j) + eta' p_i p_j],
//   eta = 2 mu, eta' = d eta / d eps_e^2, p_i = eps_{c_i} . grad N_i = d eps_e^2 / dU_i,
//   B^{uu}(X, Y) = 2 X_x Y_x + X_y Y_y / 2 + X_z Y_z / 2,  B^{uv} = X_x Y_y + X_y Y_x / 2,
//   B^{vu} = X_x Y_y / 2 + X_y Y_x,  B^{vv} = X_x Y_x / 2 + 2 X_y Y_y + X_z Y_z / 2,
// formed either with literal 12-lane dual numbers (BP_JAC_DUAL, one lane per element dof) or
// sum-factorised over the wedge's quadrature structure (BP_JAC_FACTORED).  The lane type TL is
// double (BP_F64) or float (BP_F32); the residual stays FP64 either way.
#pragma once

#include <cmath>
#include <type_traits>

#include "bp_ds.cuh"
#include "bp_internal.cuh"

namespace {

constexpr int MODE_RES = 0;
constexpr int MODE_DUAL = 1;
constexpr int MODE_FACT = 2;

struct AsmArgs {
  const double2* xy;
  const double* bed;
  const double* thick;
  const double* sigma;      // [L + 1] levels, then [L] inverse layer thicknesses
  const int32_t* tri;
  const int32_t* slots;
  const double* basal;
  const int64_t* vstart;
  const int32_t* vdeg;
  const int32_t* tri_list;  // nullable: the triangles of one colour
  int32_t count;            // columns handled by this launch
  int32_t L;
  // tail split (atomic scatter): threads [0, nwhole) take whole columns; the last count - nwhole
  // columns are taken in nseg layer segments each, by the threads that follow (nseg 0: no split)
  int32_t nwhole, nseg;
  double cA, delta;
  const double* Bn;  // nullable: [nv][L + 1] nodal hardness A^(-1/3) (rate-factor field); else cA
  const double* U;
  double* R;
  void* J;
};

// The column and layer segment [l0, l1) of thread idx of a launch (see AsmArgs::nwhole); false for
// threads past the end.
__device__ __forceinline__ bool column_segment(const AsmArgs& A, int idx, int& t, int& l0, int& l1) {
  if (A.nseg <= 1) {
    if (idx >= A.count) return false;
    t = idx, l0 = 0, l1 = A.L;
    return true;
  }
  if (idx < A.nwhole) {
    t = idx, l0 = 0, l1 = A.L;
    return true;
  }
  const int nrest = A.count - A.nwhole, j = idx - A.nwhole;
  if (j >= nrest * A.nseg) return false;
  const int sgm = j / nrest;
  t = A.nwhole + (j - sgm * nrest);
  l0 = sgm * A.L / A.nseg;
  l1 = (sgm + 1) * A.L / A.nseg;
  return true;
}

__device__ __forceinline__ constexpr double psi(int k, int z) {  // psi_k at zeta level z
  return (k == z) ? BP_QP_P : BP_QP_Q;
}
__device__ __forceinline__ constexpr double dpsi(int k) { return k == 0 ? -0.5 : 0.5; }
__device__ __forceinline__ constexpr double lam(int a, int tp) {  // lambda_a at triangle point tp
  return (a == tp) ? 2.0 / 3.0 : 1.0 / 6.0;
}
__device__ __forceinline__ constexpr int uidx(int i, int j) {  // upper-triangle index, i <= j < 12
  return i * 12 - (i * (i - 1)) / 2 + (j - i);
}
__device__ __forceinline__ constexpr int uidx6(int i, int j) {  // upper-triangle index, i <= j < 6
  return i * 6 - (i * (i - 1)) / 2 + (j - i);
}

template <bool ATOMIC, class T>
__device__ __forceinline__ void scatter_add(T* p, T v) {
  if constexpr (ATOMIC) {
    atomicAdd(p, v);
  } else {
    *p += v;
  }
}

// FP64 value -> lane type.  FP32 lanes convert on the integer pipe (f32_of): the FP64 pipe, which
// would otherwise run the conversions, is the one the value path fills.
template <class TL>
__device__ __forceinline__ TL to_lane(const double x) {
  return TL(x);
}
template <>
__device__ __forceinline__ float to_lane<float>(const double x) {
  return f32_of(x);
}
template <>
__device__ __forceinline__ f64x2 to_lane<f64x2>(const double x) {  // hi + lo, both split on the integer pipe
  return ds_of(x);
}

// A value-path quantity (type TV) as a lane (type TL): no conversion when the types agree; a pair
// gives an FP32 lane its rounded sum.
template <class TL, class TV>
__device__ __forceinline__ TL lane_from(const TV x) {
  if constexpr (std::is_same<TL, TV>::value) {
    return x;
  } else if constexpr (std::is_same<TV, f64x2>::value) {
    static_assert(std::is_same<TL, float>::value, "pairs feed FP32 or paired lanes");
    return x.hi + x.lo;
  } else {
    return to_lane<TL>(x);
  }
}
// Value-path helpers for TV = double (FP64 value path) and TV = float (the all-FP32 variant).
__device__ __forceinline__ double inv_cbrt_t(const double x) { return inv_cbrt(x); }
__device__ __forceinline__ float inv_cbrt_t(const float x) { return rcbrtf(x); }
__device__ __forceinline__ double fma_t(const double a, const double b, const double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(const float a, const float b, const float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double to_r(const double x) { return x; }
__device__ __forceinline__ double to_r(const float x) { return f64_of(x); }
// Double-single value path (TV = f64x2): the quadrature-point arithmetic of the residual in pairs
// of FP32 numbers (~2^-47 relative per operation), FP64-accurate on the FP32 pipe.
__device__ __forceinline__ f64x2 fma_t(const f64x2 a, const f64x2 b, const f64x2 c) { return a * b + c; }
__device__ __forceinline__ double to_r(const f64x2 x) { return ds_value(x); }
__device__ __forceinline__ f64x2 inv_cbrt_t(const f64x2 x) { return ds_inv_cbrt(x); }

// Element of a 2- or 3-array by an index that may be a compile-time constant (a register access)
// or a warp-uniform runtime value (a select), and the matching writes.
template <class T>
__device__ __forceinline__ T sel2(const T (&a)[2], const int i) {
  return i ? a[1] : a[0];
}
template <class T>
__device__ __forceinline__ T sel3(const T (&a)[3], const int i) {
  return i == 0 ? a[0] : (i == 1 ? a[1] : a[2]);
}
template <class T>
__device__ __forceinline__ void put2(T (&a)[2], const int i, const T v) {
  if (i)
    a[1] = v;
  else
    a[0] = v;
}
template <class T>
__device__ __forceinline__ void put3(T (&a)[3], const int i, const T v) {
  if (i == 0)
    a[0] = v;
  else if (i == 1)
    a[1] = v;
  else
    a[2] = v;
}

// storage type of a lane type in the Jacobian array, and the conversion
template <class TL>
struct LaneStore {
  using type = TL;
  static __device__ __forceinline__ TL cast(const TL v) { return v; }
};
template <>
struct LaneStore<f64x2> {
  using type = double;
  // hi + lo in FP64: the two widenings repack the fields on the integer pipe, one FP64 addition
  static __device__ __forceinline__ double cast(const f64x2 v) { return f64_of(v.hi) + f64_of(v.lo); }
};

// acc + x or acc - x with the sign known at compile time after unrolling
template <class TL>
__device__ __forceinline__ TL add_signed(const TL acc, const TL x, const bool negative) {
  return negative ? acc - x : acc + x;
}

// Accumulation into the element matrix: K += a b and K +/- x.  With paired-FP32 lanes the accumulator
// stays unnormalised: hi carries the FP32 sum and lo the exact rounding errors of the additions
// (TwoSum) plus the low-order parts of the products (TwoProd through fmaf), so each update skips the
// renormalisation of a full pair addition; the scatter sums hi and lo in FP64.
template <class TL>
__device__ __forceinline__ void acc_fma(TL& K, const TL a, const TL b) {
  K += a * b;
}
template <class TL>
__device__ __forceinline__ void acc_add(TL& K, const TL x, const bool negative) {
  K = add_signed(K, x, negative);
}
template <>
__device__ __forceinline__ void acc_fma<f64x2>(f64x2& K, const f64x2 a, const f64x2 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = K.hi + p;
  const float bb = s - K.hi;
  K.lo += ((K.hi - (s - bb)) + (p - bb)) + e;
  K.hi = s;
}
template <>
__device__ __forceinline__ void acc_add<f64x2>(f64x2& K, const f64x2 x0, const bool negative) {
  const f64x2 x = negative ? -x0 : x0;
  const float s = K.hi + x.hi;
  const float bb = s - K.hi;
  K.lo += ((K.hi - (s - bb)) + (x.hi - bb)) + x.lo;
  K.hi = s;
}

// ------------------------------------------------------------------ dual numbers
// Forward-mode dual number with an FP64 value and NL derivative lanes of type TL.
template <class TL, int NL>
struct Dual {
  double v;
  TL d[NL];
};
template <class TL, int NL>
__device__ __forceinline__ Dual<TL, NL> operator+(const Dual<TL, NL>& a, const Dual<TL, NL>& b) {
  Dual<TL, NL> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < NL; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <class TL, int NL>
__device__ __forceinline__ Dual<TL, NL> operator*(const Dual<TL, NL>& a, const Dual<TL, NL>& b) {
  Dual<TL, NL> r;
  r.v = a.v * b.v;
  const TL av = to_lane<TL>(a.v), bv = to_lane<TL>(b.v);
#pragma unroll
  for (int k = 0; k < NL; ++k) r.d[k] = a.d[k] * bv + av * b.d[k];
  return r;
}
template <class TL, int NL>
__device__ __forceinline__ Dual<TL, NL> operator*(double s, const Dual<TL, NL>& a) {
  Dual<TL, NL> r;
  r.v = s * a.v;
  const TL ts = to_lane<TL>(s);
#pragma unroll
  for (int k = 0; k < NL; ++k) r.d[k] = ts * a.d[k];
  return r;
}

// p_{(a,k),c} = psi_k alpha_{a,c} -/+ t_{a,c}, the factors of the rank-one part eta' p p^T at
// triangle point tp (node (a, k) -> entries 2 (3k + a) + c): alpha_{a,c} = g_c,xy . Lambda_a with
// alpha_2 = -(alpha_0 + alpha_1) (the barycentric gradients sum to zero), and t_{a,c} = lambda_a(tp)
// tau_c / 2, i.e. tq_c for a != tp and 4 tq_c for a == tp, given tq = tau / 12.
template <class TL>
__device__ __forceinline__ void rank_one_factors(TL (&p)[12], const TL g1x, const TL exy, const TL g2y,
                                                 const TL tq1, const TL tq2, const TL ps0, const TL ps1,
                                                 const int tp, const TL (&clx)[3], const TL (&cly)[3]) {
  TL al1[3], al2[3];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    al1[a] = g1x * clx[a] + exy * cly[a];
    al2[a] = exy * clx[a] + g2y * cly[a];
  }
  al1[2] = -(al1[0] + al1[1]);
  al2[2] = -(al2[0] + al2[1]);
  const TL f1 = TL(4) * tq1, f2 = TL(4) * tq2;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const TL t1a = a == tp ? f1 : tq1, t2a = a == tp ? f2 : tq2;
    p[2 * a] = ps0 * al1[a] - t1a;
    p[2 * a + 1] = ps0 * al2[a] - t2a;
    p[2 * (3 + a)] = ps1 * al1[a] + t1a;
    p[2 * (3 + a) + 1] = ps1 * al2[a] + t2a;
  }
}

// ------------------------------------------------------------------ the column kernel
// Assembles every wedge of the column above base triangle t (one thread).
// PICARD (factored method only): leave out the eta' rank-one part, i.e. assemble the fixed-viscosity
// (Picard) matrix instead of the Jacobian; the residual is unchanged.
// TV is the value-path type: double (the residual in FP64), or float for the all-FP32 variant
// (factored method, FP32 lanes) whose residual carries FP32 rounding: per-column and per-level
// geometry, the 2D velocity gradients and the vertical velocity differences are still formed in
// FP64 and rounded once, everything per quadrature point runs in FP32.
// SBL (factored method): the in-plane coefficients B(Lambda_a, Lambda_b) depend on the triangle only;
// they are formed once per column into shared memory (sbl: this thread's first slot, consecutive
// slots blockDim.x apart; 24 slots) and read per wedge instead of being formed again at every
// level.  With FP64 or FP32 lanes the carried element block takes 21 more slots there.
// STAGE (factored method with SBL, Jacobian not Picard): the rank-one part is applied after the
// value path, in a loop over the 6 quadrature points that is not unrolled: each point's rank-one
// factors (Wp, the three strain combinations, tau_1, tau_2) wait in shared memory (slots 45..80),
// and the element matrix is started only after the value path, so that it is not live there.  For
// the paired-FP32 lanes, whose fully unrolled arithmetic outgrows the instruction cache.
// l0, l1: the layers [l0, l1) of the column this call assembles (a segment; the whole column by
// default).  A segment starts from its bottom level with nothing carried from below and scatters
// its top level's residual and element block itself: every contribution is additive, so the
// segments of one column give the column's sum (with atomics; the coloured scatter takes whole
// columns only).
template <int MODE, class TL, bool ATOMIC, bool PICARD = false, class TV = double, bool SBL = false,
          bool STAGE = false>
__device__ __forceinline__ void assemble_column(const AsmArgs& A, const int t, TL* sbl = nullptr, int l0 = 0,
                                                int l1 = -1) {
  static_assert(std::is_same<TV, double>::value || (MODE == MODE_FACT && std::is_same<TL, float>::value) ||
                    (std::is_same<TV, f64x2>::value && MODE != MODE_DUAL),
                "the FP32 value path exists for the factored method with FP32 lanes only, the double-single "
                "one for the residual and the factored method");
  static_assert(!STAGE || (SBL && MODE == MODE_FACT && !PICARD), "the staged rank-one part needs SBL");
  const int L = A.L;
  if (l1 < 0) l1 = L;

  // ---- column geometry (per base triangle)
  int v[3];
  double x[3], y[3], H[3], bb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v[a] = A.tri[3 * t + a];
    const double2 p = A.xy[v[a]];
    x[a] = p.x;
    y[a] = p.y;
    H[a] = A.thick[v[a]];
    bb[a] = A.bed[v[a]];
  }
  const double d = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);  // 2 * area
  const double inv_d = 1.0 / d;
  double lx[3], ly[3];  // grad lambda_a
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lx[a] = (y[(a + 1) % 3] - y[(a + 2) % 3]) * inv_d;
    ly[a] = (x[(a + 2) % 3] - x[(a + 1) % 3]) * inv_d;
  }
  const double gbx = bb[0] * lx[0] + bb[1] * lx[1] + bb[2] * lx[2];
  const double gby = bb[0] * ly[0] + bb[1] * ly[1] + bb[2] * ly[2];
  const double gHx = H[0] * lx[0] + H[1] * lx[1] + H[2] * lx[2];
  const double gHy = H[0] * ly[0] + H[1] * ly[1] + H[2] * ly[2];
  const double Hs6 = (H[0] + H[1] + H[2]) * (1.0 / 6.0);
  double Hq[3], invHq[3];
#pragma unroll
  for (int tp = 0; tp < 3; ++tp) {
    Hq[tp] = Hs6 + 0.5 * H[tp];
    invHq[tp] = 1.0 / Hq[tp];
  }
  const double d12 = d * (1.0 / 12.0);
  const double d6 = d * (1.0 / 6.0);
  const TL d12L = to_lane<TL>(d12);
  const TV d6V = to_lane<TV>(d6), deltaV = to_lane<TV>(A.delta), cAV = to_lane<TV>(A.cA);
  TV lxV[3], lyV[3];  // grad lambda in value-path precision
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lxV[a] = to_lane<TV>(lx[a]);
    lyV[a] = to_lane<TV>(ly[a]);
  }
  TL clx[3], cly[3];  // grad lambda in lane precision (Jacobian lanes)
  if constexpr (MODE == MODE_FACT) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      clx[a] = to_lane<TL>(lx[a]);
      cly[a] = to_lane<TL>(ly[a]);
    }
  }
  if constexpr (SBL) {  // B(Lambda_a, Lambda_b) for the vertex pairs a <= b (pairs 00 01 02 11 12 22)
    const int bs = blockDim.x;
    int pr = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b, ++pr) {
        const TL xx = clx[a] * clx[b], yy = cly[a] * cly[b];
        const TL xy = clx[a] * cly[b], yx = cly[a] * clx[b];
        sbl[(4 * pr + 0) * bs] = TL(2) * xx + TL(0.5) * yy;
        sbl[(4 * pr + 1) * bs] = xy + TL(0.5) * yx;
        sbl[(4 * pr + 2) * bs] = TL(0.5) * xy + yx;
        sbl[(4 * pr + 3) * bs] = TL(0.5) * xx + TL(2) * yy;
      }
  }

  int64_t ubase[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) ubase[a] = 2LL * v[a] * (L + 1);


  // ---- bottom level
  double ub[3], vb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double2 w = *reinterpret_cast<const double2*>(A.U + ubase[a] + 2 * l0);
    ub[a] = w.x;
    vb[a] = w.y;
  }
  double gubx = ub[0] * lx[0] + ub[1] * lx[1] + ub[2] * lx[2];
  double guby = ub[0] * ly[0] + ub[1] * ly[1] + ub[2] * ly[2];
  double gvbx = vb[0] * lx[0] + vb[1] * lx[1] + vb[2] * lx[2];
  double gvby = vb[0] * ly[0] + vb[1] * ly[1] + vb[2] * ly[2];
  TV carry[3][2] = {{TV(0), TV(0)}, {TV(0), TV(0)}, {TV(0), TV(0)}};  // residual of the bottom level from below
  // rate-factor field: hardness B = A^(-1/3) interpolated at the triangle points of the bottom level
  TV hb[3] = {cAV, cAV, cAV};
  if (A.Bn) {
    const double b0 = A.Bn[(int64_t)v[0] * (L + 1) + l0], b1 = A.Bn[(int64_t)v[1] * (L + 1) + l0],
                 b2 = A.Bn[(int64_t)v[2] * (L + 1) + l0];
    const double bs = (b0 + b1 + b2) * (1.0 / 6.0);
    hb[0] = to_lane<TV>(bs + 0.5 * b0);
    hb[1] = to_lane<TV>(bs + 0.5 * b1);
    hb[2] = to_lane<TV>(bs + 0.5 * b2);
  }

  // Sum-factorised FP64 and FP32 lanes (and paired lanes with the shared-memory table): the next
  // level's velocities are loaded one wedge ahead, and the element-matrix block of the top level is
  // carried to the next wedge (where it is the bottom block of the same J entries) instead of being
  // scattered twice: 108 scalar atomics per wedge (54 float2 ones for FP32 values), not 144.
  constexpr bool kAhead =
      (std::is_same<TL, float>::value || std::is_same<TL, double>::value || (SBL && std::is_same<TL, f64x2>::value)) &&
      MODE == MODE_FACT;
  double2 nxt[3];
  // carried top-top block (upper triangle of local dofs 6..11): in shared memory after the in-plane
  // coefficients with SBL (slots 24..44), else in registers
  TL Kc_r[SBL ? 1 : 21];
  const int kcs = SBL ? (int)blockDim.x : 1;
  TL* const Kc0 = SBL ? sbl + 24 * kcs : Kc_r;
#define KC(k) Kc0[(k) * kcs]
  if constexpr (kAhead) {
#pragma unroll
    for (int a = 0; a < 3; ++a) nxt[a] = *reinterpret_cast<const double2*>(A.U + ubase[a] + 2 * (l0 + 1));
#pragma unroll
    for (int k = 0; k < 21; ++k) KC(k) = TL(0);
  }

  for (int l = l0; l < l1; ++l) {
    double ut[3], vt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double2 w;
      if constexpr (kAhead) {
        w = nxt[a];
      } else {
        w = *reinterpret_cast<const double2*>(A.U + ubase[a] + 2 * (l + 1));
      }
      ut[a] = w.x;
      vt[a] = w.y;
    }
    if constexpr (kAhead) {
      if (l + 2 <= l1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) nxt[a] = *reinterpret_cast<const double2*>(A.U + ubase[a] + 2 * (l + 2));
      }
    }
    const double gutx = ut[0] * lx[0] + ut[1] * lx[1] + ut[2] * lx[2];
    const double guty = ut[0] * ly[0] + ut[1] * ly[1] + ut[2] * ly[2];
    const double gvtx = vt[0] * lx[0] + vt[1] * lx[1] + vt[2] * lx[2];
    const double gvty = vt[0] * ly[0] + vt[1] * ly[1] + vt[2] * ly[2];
    const double s_l = A.sigma[l];
    const double ds = A.sigma[l + 1] - s_l;
    const double invds = A.sigma[L + 1 + l];  // 1 / ds, formed once at upload
    TV ht[3] = {cAV, cAV, cAV};  // hardness at the triangle points of the top level
    if (A.Bn) {
      const double b0 = A.Bn[(int64_t)v[0] * (L + 1) + l + 1], b1 = A.Bn[(int64_t)v[1] * (L + 1) + l + 1],
                   b2 = A.Bn[(int64_t)v[2] * (L + 1) + l + 1];
      const double bs = (b0 + b1 + b2) * (1.0 / 6.0);
      ht[0] = to_lane<TV>(bs + 0.5 * b0);
      ht[1] = to_lane<TV>(bs + 0.5 * b1);
      ht[2] = to_lane<TV>(bs + 0.5 * b2);
    }

    // per zeta level: slope of the level surface and the 2D velocity gradients
    double Gzx[2], Gzy[2];
    TV GzxV[2], GzyV[2], GUx[2], GUy[2], GVx[2], GVy[2];
    const TV gUb[2] = {to_lane<TV>(gubx), to_lane<TV>(guby)}, gUt[2] = {to_lane<TV>(gutx), to_lane<TV>(guty)};
    const TV gVb[2] = {to_lane<TV>(gvbx), to_lane<TV>(gvby)}, gVt[2] = {to_lane<TV>(gvtx), to_lane<TV>(gvty)};
#pragma unroll
    for (int z = 0; z < 2; ++z) {
      const double sz = s_l + psi(1, z) * ds;
      Gzx[z] = gbx + sz * gHx;
      Gzy[z] = gby + sz * gHy;
      GzxV[z] = to_lane<TV>(Gzx[z]);
      GzyV[z] = to_lane<TV>(Gzy[z]);
      GUx[z] = TV(psi(0, z)) * gUb[0] + TV(psi(1, z)) * gUt[0];
      GUy[z] = TV(psi(0, z)) * gUb[1] + TV(psi(1, z)) * gUt[1];
      GVx[z] = TV(psi(0, z)) * gVb[0] + TV(psi(1, z)) * gVt[0];
      GVy[z] = TV(psi(0, z)) * gVb[1] + TV(psi(1, z)) * gVt[1];
    }
    // per triangle point: vertical shear, weights
    const double dus6 = (ut[0] - ub[0] + ut[1] - ub[1] + ut[2] - ub[2]) * (1.0 / 6.0);
    const double dvs6 = (vt[0] - vb[0] + vt[1] - vb[1] + vt[2] - vb[2]) * (1.0 / 6.0);
    double cq[3], invh[3], invh6[3];
    TV uz[3], vz[3], ez[3], cqV[3];
#pragma unroll
    for (int tp = 0; tp < 3; ++tp) {
      invh[tp] = invds * invHq[tp];
      invh6[tp] = invh[tp] * (1.0 / 6.0);
      const TV invhV = to_lane<TV>(invh[tp]);
      uz[tp] = to_lane<TV>(dus6 + 0.5 * (ut[tp] - ub[tp])) * invhV;
      vz[tp] = to_lane<TV>(dvs6 + 0.5 * (vt[tp] - vb[tp])) * invhV;
      ez[tp] = TV(0.25) * (uz[tp] * uz[tp] + vz[tp] * vz[tp]);
      cq[tp] = d12 * ds * Hq[tp];
      cqV[tp] = to_lane<TV>(cq[tp]);
    }

    TV Rl[2][3][2];  // [k][a][c] residual of this wedge
    TL K[78];            // upper triangle of the element matrix
    TL eta_q[2][3];      // 2 mu at the quadrature points (factored Jacobian)
    // FP32 lanes: the per-point weights in FP32, converted once per wedge
    constexpr bool kF32 = std::is_same<TL, float>::value;
    TL cqL[3], invhL[3];
    if constexpr (MODE == MODE_FACT) {
#pragma unroll
      for (int tp = 0; tp < 3; ++tp) {
        cqL[tp] = to_lane<TL>(cq[tp]);
        invhL[tp] = to_lane<TL>(invh[tp]);
      }
    }
    auto start_element_matrix = [&]() {
      if constexpr (MODE != MODE_RES) {
#pragma unroll
        for (int k = 0; k < 78; ++k) K[k] = TL(0);
      }
      if constexpr (kAhead) {  // the previous wedge's top-top block starts this wedge's bottom-bottom block
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
          for (int j = i; j < 6; ++j) K[uidx(i, j)] = KC(uidx6(i, j));
      }
    };
    if constexpr (!STAGE) start_element_matrix();

    if constexpr (MODE == MODE_DUAL) {
      // ---- literal forward mode: 12 lanes, lane j = d / dU_j (j = 2 * (3k + a) + c)
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) Rl[k][a][0] = Rl[k][a][1] = 0.0;
#pragma unroll
      for (int z = 0; z < 2; ++z) {
#pragma unroll
        for (int tp = 0; tp < 3; ++tp) {
          const double Zx = -2.0 * invh[tp] * Gzx[z], Zy = -2.0 * invh[tp] * Gzy[z], Zz = 2.0 * invh[tp];
          double gNd[6][3];  // physical basis gradients, node n = 3k + a (value path, FP64)
          TL gN[6][3];       // the same in lane precision
#pragma unroll
          for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              const double c = lam(a, tp) * dpsi(k);
              gNd[3 * k + a][0] = psi(k, z) * lx[a] + c * Zx;
              gNd[3 * k + a][1] = psi(k, z) * ly[a] + c * Zy;
              gNd[3 * k + a][2] = c * Zz;
#pragma unroll
              for (int r = 0; r < 3; ++r) gN[3 * k + a][r] = to_lane<TL>(gNd[3 * k + a][r]);
            }
          Dual<TL, 12> ux, uy, uzd, vx, vy, vzd;
          ux.v = GUx[z] - uz[tp] * Gzx[z];
          uy.v = GUy[z] - uz[tp] * Gzy[z];
          vx.v = GVx[z] - vz[tp] * Gzx[z];
          vy.v = GVy[z] - vz[tp] * Gzy[z];
          uzd.v = uz[tp];
          vzd.v = vz[tp];
#pragma unroll
          for (int n = 0; n < 6; ++n) {  // seed: d(grad u)/dU_(n,u) = grad N_n, d(grad v)/dU_(n,v) = grad N_n
            ux.d[2 * n] = gN[n][0];
            ux.d[2 * n + 1] = TL(0);
            uy.d[2 * n] = gN[n][1];
            uy.d[2 * n + 1] = TL(0);
            uzd.d[2 * n] = gN[n][2];
            uzd.d[2 * n + 1] = TL(0);
            vx.d[2 * n] = TL(0);
            vx.d[2 * n + 1] = gN[n][0];
            vy.d[2 * n] = TL(0);
            vy.d[2 * n + 1] = gN[n][1];
            vzd.d[2 * n] = TL(0);
            vzd.d[2 * n + 1] = gN[n][2];
          }
          const Dual<TL, 12> exy = 0.5 * (uy + vx);
          const Dual<TL, 12> exz = 0.5 * uzd;
          const Dual<TL, 12> eyz = 0.5 * vzd;
          const Dual<TL, 12> e2 = ux * ux + vy * (vy + ux) + exy * exy + exz * exz + eyz * eyz;
          const double xx = e2.v + A.delta;
          const double r = inv_cbrt(xx);
          Dual<TL, 12> eta;  // eta = B (e2 + delta)^(-1/3), d eta / d e2 = -eta / (3 (e2 + delta))
          eta.v = (psi(0, z) * hb[tp] + psi(1, z) * ht[tp]) * r;
          const TL detad = to_lane<TL>(-(1.0 / 3.0) * eta.v * (r * r * r));
#pragma unroll
          for (int j = 0; j < 12; ++j) eta.d[j] = detad * e2.d[j];
          const Dual<TL, 12> g1x = 2.0 * ux + vy, g2y = ux + 2.0 * vy;
          const double c = cq[tp];
          const TL cL = to_lane<TL>(c);
#pragma unroll
          for (int n = 0; n < 6; ++n) {
#pragma unroll
            for (int comp = 0; comp < 2; ++comp) {
              const int i = 2 * n + comp;
              const Dual<TL, 12>& ga = comp == 0 ? g1x : exy;
              const Dual<TL, 12>& gb = comp == 0 ? exy : g2y;
              const Dual<TL, 12>& gc = comp == 0 ? exz : eyz;
              Dual<TL, 12> pi;  // p_i = g_c . grad N_n
              pi.v = ga.v * gNd[n][0] + gb.v * gNd[n][1] + gc.v * gNd[n][2];
#pragma unroll
              for (int j = 0; j < 12; ++j) pi.d[j] = ga.d[j] * gN[n][0] + gb.d[j] * gN[n][1] + gc.d[j] * gN[n][2];
              const Dual<TL, 12> ri = eta * pi;
              Rl[n / 3][n % 3][comp] += c * ri.v;
#pragma unroll
              for (int j = i; j < 12; ++j) acc_fma(K[uidx(i, j)], cL, ri.d[j]);
            }
          }
        }
      }
    } else {
      // ---- structured value path (+ sum-factorised Jacobian lanes)
      TV P1x[2] = {TV(0), TV(0)}, P1y[2] = {TV(0), TV(0)}, P2x[2] = {TV(0), TV(0)}, P2y[2] = {TV(0), TV(0)};
      TV TW1[3] = {TV(0), TV(0), TV(0)}, TW2[3] = {TV(0), TV(0), TV(0)};
      // One quadrature point (zeta level z, triangle point tp).  The arrays indexed by z and tp are
      // read and written through sel2 / sel3 / put2 / put3: plain register accesses when the
      // indices are compile-time constants (the unrolled loop below), warp-uniform selects when they
      // are not (the double-single value path runs the 6 points in a loop that is not unrolled: its
      // pair arithmetic, ~10 instructions per FP64 one, would not fit the instruction cache 6 times).
      // hardness at the 6 points, psi_0 hb + psi_1 ht (the constant A^(-1/3) without a field), formed
      // once per wedge for the FP64 and FP32 value paths; the double-single path, short of registers,
      // forms it per point
      constexpr bool kHq = !std::is_same<TV, f64x2>::value;
      TV hq[2][3];
      if (!kHq) {
      } else if (A.Bn) {
#pragma unroll
        for (int tp = 0; tp < 3; ++tp) {
          hq[0][tp] = TV(BP_QP_P) * hb[tp] + TV(BP_QP_Q) * ht[tp];
          hq[1][tp] = TV(BP_QP_Q) * hb[tp] + TV(BP_QP_P) * ht[tp];
        }
      } else {
#pragma unroll
        for (int tp = 0; tp < 3; ++tp) hq[0][tp] = hq[1][tp] = cAV;
      }
      auto point = [&](const int z, const int tp) {
        const TV gzx = sel2(GzxV, z), gzy = sel2(GzyV, z);
        const TV uzp = sel3(uz, tp), vzp = sel3(vz, tp);
        const TV ux = sel2(GUx, z) - uzp * gzx;
        const TV uy = sel2(GUy, z) - uzp * gzy;
        const TV vx = sel2(GVx, z) - vzp * gzx;
        const TV vy = sel2(GVy, z) - vzp * gzy;
        const TV exy = TV(0.5) * (uy + vx);
        const TV e2 = fma_t(ux, ux, fma_t(vy, vy + ux, fma_t(exy, exy, sel3(ez, tp))));
        const TV xx = e2 + deltaV;
        const TV r = inv_cbrt_t(xx);
        TV eta;
        if constexpr (kHq) {
          eta = (z ? sel3(hq[1], tp) : sel3(hq[0], tp)) * r;
        } else {
          const TV ps0 = z ? TV(BP_QP_Q) : TV(BP_QP_P), ps1 = z ? TV(BP_QP_P) : TV(BP_QP_Q);  // psi_k at z
          eta = (ps0 * sel3(hb, tp) + ps1 * sel3(ht, tp)) * r;
        }
        const TV W = sel3(cqV, tp) * eta;
        const TV g1x = TV(2.0) * ux + vy, g2y = ux + TV(2.0) * vy;
        put2(P1x, z, fma_t(W, g1x, sel2(P1x, z)));
        put2(P1y, z, fma_t(W, exy, sel2(P1y, z)));
        put2(P2x, z, fma_t(W, exy, sel2(P2x, z)));
        put2(P2y, z, fma_t(W, g2y, sel2(P2y, z)));
        const TV t1 = TV(0.5) * uzp - g1x * gzx - exy * gzy;
        const TV t2 = TV(0.5) * vzp - exy * gzx - g2y * gzy;
        const TV W6 = d6V * eta;
        put3(TW1, tp, fma_t(W6, t1, sel3(TW1, tp)));
        put3(TW2, tp, fma_t(W6, t2, sel3(TW2, tp)));
        if constexpr (MODE == MODE_FACT) {
          // rank-one part eta' p_i p_j with p_{(a,k),c} = psi_k g_c,xy . Lambda_a + lambda_a psi_k' g_c . Z
          TL Wp, tau1, tau2, eq;  // tau1, tau2 hold tau_c / 12 (see rank_one_factors)
          if constexpr (kF32) {  // from r, t1, t2 converted once: FP32 arithmetic only
            const float rf = lane_from<float>(r);
            const float ef = lane_from<float>(eta);
            eq = ef;
            Wp = (-1.0f / 3.0f) * sel3(cqL, tp) * ef * (rf * rf * rf);
            const float ih6 = sel3(invhL, tp) * (1.0f / 6.0f);
            tau1 = ih6 * lane_from<float>(t1);  // tau / 12 (rank_one_factors)
            tau2 = ih6 * lane_from<float>(t2);
          } else if constexpr (std::is_same<TV, f64x2>::value) {  // double-single value path, paired lanes
            eq = eta;
            Wp = TV(-1.0 / 3.0) * W * (r * r * r);
            const TV ih6 = to_lane<TV>(sel3(invh6, tp));
            tau1 = ih6 * t1;  // tau / 12
            tau2 = ih6 * t2;
          } else {
            eq = to_lane<TL>(eta);
            Wp = to_lane<TL>(-(1.0 / 3.0) * W * (r * r * r));
            const double ih6 = sel3(invh6, tp);
            tau1 = to_lane<TL>(ih6 * t1);  // tau / 12
            tau2 = to_lane<TL>(ih6 * t2);
          }
          if (z)
            put3(eta_q[1], tp, eq);
          else
            put3(eta_q[0], tp, eq);
          if constexpr (STAGE) {  // park the point's rank-one factors (slots 45 + 6 q ..)
            const int bs = blockDim.x;
            TL* const sq = sbl + (45 + 6 * (3 * z + tp)) * bs;
            sq[0] = Wp;
            sq[bs] = lane_from<TL>(g1x);
            sq[2 * bs] = lane_from<TL>(exy);
            sq[3 * bs] = lane_from<TL>(g2y);
            sq[4 * bs] = tau1;
            sq[5 * bs] = tau2;
          } else if constexpr (!PICARD) {
            const TL fg1x = lane_from<TL>(g1x), fexy = lane_from<TL>(exy), fg2y = lane_from<TL>(g2y);
            const TL pl0 = z ? TL(BP_QP_Q) : TL(BP_QP_P), pl1 = z ? TL(BP_QP_P) : TL(BP_QP_Q);
            TL p[12];
            rank_one_factors(p, fg1x, fexy, fg2y, tau1, tau2, pl0, pl1, tp, clx, cly);
#pragma unroll
            for (int i = 0; i < 12; ++i) {
              const TL pw = Wp * p[i];
#pragma unroll
              for (int j = i; j < 12; ++j) acc_fma(K[uidx(i, j)], pw, p[j]);
            }
          }
        }
      };
      if constexpr (std::is_same<TV, f64x2>::value) {
#pragma unroll 1
        for (int q = 0; q < 6; ++q) point(q >= 3 ? 1 : 0, q >= 3 ? q - 3 : q);
      } else {
#pragma unroll
        for (int z = 0; z < 2; ++z)
#pragma unroll
          for (int tp = 0; tp < 3; ++tp) point(z, tp);
      }
      // residual: R_{a,k,c} = Lambda_a . sum_z psi_k(z) P_c(z) + psi_k' sum_tp lambda_a(tp) TW_c(tp)
      const TV T1s = (TW1[0] + TW1[1] + TW1[2]) * TV(1.0 / 6.0);
      const TV T2s = (TW2[0] + TW2[1] + TW2[2]) * TV(1.0 / 6.0);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const TV A1x = TV(psi(k, 0)) * P1x[0] + TV(psi(k, 1)) * P1x[1];
        const TV A1y = TV(psi(k, 0)) * P1y[0] + TV(psi(k, 1)) * P1y[1];
        const TV A2x = TV(psi(k, 0)) * P2x[0] + TV(psi(k, 1)) * P2x[1];
        const TV A2y = TV(psi(k, 0)) * P2y[0] + TV(psi(k, 1)) * P2y[1];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          Rl[k][a][0] = lxV[a] * A1x + lyV[a] * A1y + TV(dpsi(k)) * (T1s + TV(0.5) * TW1[a]);
          Rl[k][a][1] = lxV[a] * A2x + lyV[a] * A2y + TV(dpsi(k)) * (T2s + TV(0.5) * TW2[a]);
        }
      }
      if constexpr (STAGE) {
        start_element_matrix();
        const int bs = blockDim.x;
#pragma unroll 1
        for (int q = 0; q < 6; ++q) {
          const int z = q >= 3 ? 1 : 0, tp = q - 3 * z;
          const TL* const sq = sbl + (45 + 6 * q) * bs;
          const TL Wp = sq[0], fg1x = sq[bs], fexy = sq[2 * bs], fg2y = sq[3 * bs], tau1 = sq[4 * bs],
                   tau2 = sq[5 * bs];
          const TL ps0 = z ? TL(BP_QP_Q) : TL(BP_QP_P), ps1 = z ? TL(BP_QP_P) : TL(BP_QP_Q);
          TL p[12];
          rank_one_factors(p, fg1x, fexy, fg2y, tau1, tau2, ps0, ps1, tp, clx, cly);
#pragma unroll
          for (int i = 0; i < 12; ++i) {
            const TL pw = Wp * p[i];
#pragma unroll
            for (int j = i; j < 12; ++j) acc_fma(K[uidx(i, j)], pw, p[j]);
          }
        }
      }
      if constexpr (MODE == MODE_FACT) {
        // eta B(grad N_i, grad N_j) summed over the quadrature, B bilinear:
        //  (I)   Q_km B(Lambda_a, Lambda_b),          Q_km = sum_q W psi_k psi_m
        //  (II)  psi_m' B(Lambda_a, V^k_b),           V^k_b = sum_q W psi_k lambda_b Z_xy
        //  (III) psi_k' B(V^m_a, Lambda_b)
        //  (IV)  psi_k' psi_m' Y_ab,                  Y_ab = sum_q W lambda_a lambda_b B(Z, Z)
        TL Qs[2], E[2][3], F[2][6];
#pragma unroll
        for (int z = 0; z < 2; ++z) {
          Qs[z] = TL(0);
#pragma unroll
          for (int tp = 0; tp < 3; ++tp) Qs[z] += cqL[tp] * eta_q[z][tp];
          const TL es = (eta_q[z][0] + eta_q[z][1] + eta_q[z][2]) * TL(1.0 / 6.0);
          TL ei[3];
#pragma unroll
          for (int tp = 0; tp < 3; ++tp) {
            E[z][tp] = es + TL(0.5) * eta_q[z][tp];
            ei[tp] = eta_q[z][tp] * invhL[tp];
          }
          // F_ab = sum_tp lambda_a lambda_b eta / h, pairs 00 01 02 11 12 22
          int pr = 0;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b) {
              TL f = TL(0);
#pragma unroll
              for (int tp = 0; tp < 3; ++tp) f += (TL)(lam(a, tp) * lam(b, tp)) * ei[tp];
              F[z][pr++] = f;
            }
        }
        TL Q[2][2];
        Q[0][0] = (TL)(BP_QP_P * BP_QP_P) * Qs[0] + (TL)(BP_QP_Q * BP_QP_Q) * Qs[1];
        Q[1][1] = (TL)(BP_QP_Q * BP_QP_Q) * Qs[0] + (TL)(BP_QP_P * BP_QP_P) * Qs[1];
        Q[0][1] = Q[1][0] = (TL)(BP_QP_P * BP_QP_Q) * (Qs[0] + Qs[1]);
        // V^k_b scaled by 1/2 (the magnitude of psi'): V = -(d/12) sum_z psi_k E_b Gz
        TL Vx[2][3], Vy[2][3];
        const TL GzxL[2] = {to_lane<TL>(Gzx[0]), to_lane<TL>(Gzx[1])};
        const TL GzyL[2] = {to_lane<TL>(Gzy[0]), to_lane<TL>(Gzy[1])};
        const TL md12 = -d12L;
        const TL gz0x = md12 * GzxL[0], gz1x = md12 * GzxL[1];
        const TL gz0y = md12 * GzyL[0], gz1y = md12 * GzyL[1];
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const TL w0 = (TL)psi(k, 0) * E[0][b], w1 = (TL)psi(k, 1) * E[1][b];
            Vx[k][b] = w0 * gz0x + w1 * gz1x;
            Vy[k][b] = w0 * gz0y + w1 * gz1y;
          }
        // Y scaled by 1/4 (|psi_k' psi_m'|): (d/12) sum_z F_ab(z) B_zz(z)
        TL Yuu[6], Yvv[6], Yuv[6];
        {
          TL Buu[2], Bvv[2], Buv[2];
#pragma unroll
          for (int z = 0; z < 2; ++z) {
            const TL gx = GzxL[z], gy = GzyL[z];
            Buu[z] = TL(2) * gx * gx + TL(0.5) * gy * gy + TL(0.5);
            Bvv[z] = TL(0.5) * gx * gx + TL(2) * gy * gy + TL(0.5);
            Buv[z] = TL(1.5) * gx * gy;
          }
          const TL s = d12L;
#pragma unroll
          for (int pr = 0; pr < 6; ++pr) {
            Yuu[pr] = s * (F[0][pr] * Buu[0] + F[1][pr] * Buu[1]);
            Yvv[pr] = s * (F[0][pr] * Bvv[0] + F[1][pr] * Bvv[1]);
            Yuv[pr] = s * (F[0][pr] * Buv[0] + F[1][pr] * Buv[1]);
          }
        }
        const TL* flx = clx;
        const TL* fly = cly;
        // per node pair (n1 = (a,k) <= n2 = (b,m)), s = sign of psi':
        //   K += Q_km B(Lambda_a, Lambda_b) + s_k s_m Y_ab + s_m BV[a][k][b] + s_k BV[b][m][a]^T,
        // with BV[a][k][b] = B(Lambda_a, V^k_b).  First the in-plane and Y terms pair by pair ...
#pragma unroll
        for (int n1 = 0; n1 < 6; ++n1) {
#pragma unroll
          for (int n2 = n1; n2 < 6; ++n2) {
            const int ki = n1 / 3, ai = n1 % 3, kj = n2 / 3, bj = n2 % 3;
            const int lo = ai < bj ? ai : bj, hi = ai < bj ? bj : ai;
            const int pr = lo * 3 - (lo * (lo - 1)) / 2 + (hi - lo);
            TL BL[4];
            if constexpr (SBL) {  // B(Lambda_b, Lambda_a) is B(Lambda_a, Lambda_b) with the uv / vu terms swapped
              const int bs = blockDim.x;
              BL[0] = sbl[(4 * pr + 0) * bs];
              BL[1] = sbl[(4 * pr + (ai <= bj ? 1 : 2)) * bs];
              BL[2] = sbl[(4 * pr + (ai <= bj ? 2 : 1)) * bs];
              BL[3] = sbl[(4 * pr + 3) * bs];
            } else {
              const TL xx = flx[ai] * flx[bj], yy = fly[ai] * fly[bj];
              const TL xy = flx[ai] * fly[bj], yx = fly[ai] * flx[bj];
              BL[0] = TL(2) * xx + TL(0.5) * yy;
              BL[1] = xy + TL(0.5) * yx;
              BL[2] = TL(0.5) * xy + yx;
              BL[3] = TL(0.5) * xx + TL(2) * yy;
            }
            const TL Yc[4] = {Yuu[pr], Yuv[pr], Yuv[pr], Yvv[pr]};
            const TL q = Q[ki][kj];
            const bool neg = (ki == 0) != (kj == 0);
#pragma unroll
            for (int ci = 0; ci < 2; ++ci)
#pragma unroll
              for (int cj = 0; cj < 2; ++cj) {
                const int i = 2 * n1 + ci, j = 2 * n2 + cj;
                if (i > j) continue;
                const int cd = 2 * ci + cj;
                acc_fma(K[uidx(i, j)], q, BL[cd]);
                acc_add(K[uidx(i, j)], Yc[cd], neg);
              }
          }
        }
        // ... then the BV terms node by node: the 12 values BV[a][k][.] of node n = (a, k) go to the
        // pairs where n is the first node (the s_m term) and where it is the second (the transposed
        // s_k term), so that only one node's values are live at a time.
#pragma unroll
        for (int n = 0; n < 6; ++n) {
          const int kn = n / 3, an = n % 3;
          TL BVn[3][4];
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const TL xx = flx[an] * Vx[kn][b], yy = fly[an] * Vy[kn][b];
            const TL xy = flx[an] * Vy[kn][b], yx = fly[an] * Vx[kn][b];
            BVn[b][0] = TL(2) * xx + TL(0.5) * yy;
            BVn[b][1] = xy + TL(0.5) * yx;
            BVn[b][2] = TL(0.5) * xy + yx;
            BVn[b][3] = TL(0.5) * xx + TL(2) * yy;
          }
#pragma unroll
          for (int n2 = n; n2 < 6; ++n2) {  // n first: + s_m BV[a][k][b][cd], n2 = (b, m)
            const int kj = n2 / 3, bj = n2 % 3;
#pragma unroll
            for (int ci = 0; ci < 2; ++ci)
#pragma unroll
              for (int cj = 0; cj < 2; ++cj) {
                const int i = 2 * n + ci, j = 2 * n2 + cj;
                if (i > j) continue;
                acc_add(K[uidx(i, j)], BVn[bj][2 * ci + cj], kj == 0);
              }
          }
#pragma unroll
          for (int n1 = 0; n1 <= n; ++n1) {  // n second: + s_k BV[b][m][a][dc], n1 = (a, k)
            const int ki = n1 / 3, ai = n1 % 3;
#pragma unroll
            for (int ci = 0; ci < 2; ++ci)
#pragma unroll
              for (int cj = 0; cj < 2; ++cj) {
                const int i = 2 * n1 + ci, j = 2 * n + cj;
                if (i > j) continue;
                acc_add(K[uidx(i, j)], BVn[ai][2 * cj + ci], ki == 0);
              }
          }
        }
      }
    }

    // ---- basal friction (bottom face of the first layer), memoised 3x3 matrix per triangle
    if (l == 0) {
      const double* Mb = A.basal + 6 * (int64_t)t;
      const double M[3][3] = {{Mb[0], Mb[1], Mb[2]}, {Mb[1], Mb[3], Mb[4]}, {Mb[2], Mb[4], Mb[5]}};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Rl[0][a][0] += to_lane<TV>(M[a][0] * ub[0] + M[a][1] * ub[1] + M[a][2] * ub[2]);
        Rl[0][a][1] += to_lane<TV>(M[a][0] * vb[0] + M[a][1] * vb[1] + M[a][2] * vb[2]);
      }
      if constexpr (MODE != MODE_RES) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = a; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) acc_add(K[uidx(2 * a + c, 2 * b + c)], to_lane<TL>(M[a][b]), false);
      }
    }

    // ---- scatter: residual of the bottom level is complete now; the top level is carried
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      scatter_add<ATOMIC>(A.R + ubase[a] + 2 * l, to_r(Rl[0][a][0] + carry[a][0]));
      scatter_add<ATOMIC>(A.R + ubase[a] + 2 * l + 1, to_r(Rl[0][a][1] + carry[a][1]));
      carry[a][0] = Rl[1][a][0];
      carry[a][1] = Rl[1][a][1];
    }
    if constexpr (MODE != MODE_RES) {
      using ST = typename LaneStore<TL>::type;
      ST* J = static_cast<ST*>(A.J);
      // scatter positions: the vertices' row blocks and the triangle's slots are read here, per
      // wedge, from the (L1-resident) mesh arrays rather than kept live across the level loop,
      // whose registers the element matrix needs
      int64_t vs[3];
      int dg[3], sl[9];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        vs[a] = __ldg(A.vstart + v[a]);
        dg[a] = __ldg(A.vdeg + v[a]);
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) sl[k] = __ldg(A.slots + 9 * t + k);
      int64_t rowbase[6], rowhalf[6];
      int nlev[2], off[2][2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        nlev[k] = bp_nlev(l + k, L);
        const int lmin = (l + k) > 0 ? (l + k - 1) : 0;
#pragma unroll
        for (int m = 0; m < 2; ++m) off[k][m] = l + m - lmin;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          rowbase[3 * k + a] = vs[a] + (int64_t)dg[a] * 4 * bp_levels_before(l + k);
          rowhalf[3 * k + a] = 2LL * nlev[k] * dg[a];
        }
      }
      if constexpr (ATOMIC && std::is_same<ST, float>::value) {
        // FP32 values: the (u, v) column pair of a row and a column node is one aligned float2 in
        // the pattern, added by one vector atomic: 72 per wedge (54 with the carry) instead of 144
        // scalar ones.  The entry points require 8-byte aligned FP32 values.
        if constexpr (kAhead) {
          if (l + 1 < l1) {  // top-top block: carried to the next wedge
#pragma unroll
            for (int i = 6; i < 12; ++i)
#pragma unroll
              for (int j = i; j < 12; ++j) KC(uidx6(i - 6, j - 6)) = K[uidx(i, j)];
          }
        }
#pragma unroll
        for (int i = 0; i < 12; ++i) {
          const int ni = i >> 1, ci = i & 1, ki = ni / 3, ai = ni % 3;
#pragma unroll
          for (int nj = 0; nj < 6; ++nj) {
            const int kj = nj / 3, bj = nj % 3;
            if constexpr (kAhead) {
              if (ni >= 3 && nj >= 3 && l + 1 < l1) continue;  // carried
            }
            const int j0 = 2 * nj, j1 = 2 * nj + 1;
            const float v0 = LaneStore<TL>::cast(K[i <= j0 ? uidx(i, j0) : uidx(j0, i)]);
            const float v1 = LaneStore<TL>::cast(K[i <= j1 ? uidx(i, j1) : uidx(j1, i)]);
            const int64_t p = rowbase[ni] + ci * rowhalf[ni] + 2 * (sl[3 * ai + bj] * nlev[ki] + off[ki][kj]);
            atomicAdd(reinterpret_cast<float2*>(J + p), make_float2(v0, v1));
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < 12; ++i) {
          const int ni = i >> 1, ci = i & 1, ki = ni / 3, ai = ni % 3;
#pragma unroll
          for (int j = i; j < 12; ++j) {
            const int nj = j >> 1, cj = j & 1, kj = nj / 3, bj = nj % 3;
            if constexpr (kAhead) {
              if (i >= 6 && l + 1 < l1) {  // top-top block: carried to the next wedge
                KC(uidx6(i - 6, j - 6)) = K[uidx(i, j)];
                continue;
              }
            }
            const ST val = LaneStore<TL>::cast(K[uidx(i, j)]);
            const int64_t pij = rowbase[ni] + ci * rowhalf[ni] + 2 * (sl[3 * ai + bj] * nlev[ki] + off[ki][kj]) + cj;
            scatter_add<ATOMIC>(J + pij, val);
            if (i != j) {
              const int64_t pji = rowbase[nj] + cj * rowhalf[nj] + 2 * (sl[3 * bj + ai] * nlev[kj] + off[kj][ki]) + ci;
              scatter_add<ATOMIC>(J + pji, val);
            }
          }
        }
      }
    }

    // ---- shift the top level down
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ub[a] = ut[a];
      vb[a] = vt[a];
      hb[a] = ht[a];
    }
    gubx = gutx;
    guby = guty;
    gvbx = gvtx;
    gvby = gvty;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    scatter_add<ATOMIC>(A.R + ubase[a] + 2 * l1, to_r(carry[a][0]));
    scatter_add<ATOMIC>(A.R + ubase[a] + 2 * l1 + 1, to_r(carry[a][1]));
  }
#undef KC
}

}  // namespace
