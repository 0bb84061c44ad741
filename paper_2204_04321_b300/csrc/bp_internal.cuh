// Internal declarations of libbp (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

#include "bp.h"

#define BP_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t bp_err_ = (expr);                           \
    if (bp_err_ != cudaSuccess) {                           \
      bp_set_last_cuda_error(bp_err_, #expr, __LINE__);     \
      return BP_ECUDA;                                      \
    }                                                       \
  } while (0)

void bp_set_last_cuda_error(cudaError_t err, const char* what, int line);

// Quadrature constants of the fixed wedge rule (see bp.h).
// zeta = -+1/sqrt(3): psi_0 = (1 - zeta)/2, psi_1 = (1 + zeta)/2 take the values P and Q.
#define BP_QP_P 0.78867513459481288225457439025098  // (1 + 1/sqrt(3)) / 2
#define BP_QP_Q 0.21132486540518711774542560974902  // (1 - 1/sqrt(3)) / 2

// Newton-Krylov workspace, allocated on the first solver call and owned by the mesh.
struct bp_solver_ws {
  int32_t* dslot = nullptr;   // [nv] rank of the vertex in its own closed neighbourhood
  double* Lm = nullptr;       // [L][4][nv]   E_l G_{l-1}^-1 (block Thomas multipliers), l = 1..L
  double* Ginv = nullptr;     // [L+1][4][nv] inverses of the eliminated diagonal blocks
  double* Fu = nullptr;       // [L][4][nv]   super-diagonal blocks J(l, l+1)
                              // (double, or float in the first half of each array: prec_f32)
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;  // Krylov vectors
  double* J = nullptr;        // [nnz] Jacobian values (double, or float in the first half)
  double* R = nullptr;        // [ndof] residual
  double* Ut = nullptr;       // [ndof] trial iterate of the line search
  double* scal = nullptr;     // [3 (cap + 2)] per Krylov iteration: p.q, r.z, r.r
  int scal_cap = 0;
  int* stop = nullptr;        // Krylov stop flag (1 converged, 2 breakdown, 3 not finite, 4 limit,
                              // 5 a bounded wait for bulk copies gave up)
  double* red = nullptr;      // [8] reduction scalars
  double* sia = nullptr;      // [3 nv] shallow-ice scratch
  double* host = nullptr;     // pinned host mirror of scal / red
  int host_cap = 0;
  bool has_prec = false;
  bool prec_f32 = false;      // factors stored as float (set up from an FP32 Jacobian)
  int* kbase = nullptr;       // CG: first iteration index of the current batch (device)
  double* cgpar = nullptr;    // CG: [0] tolerance eta^2 on r.r / r0.r0, [1] iteration limit (device)
  double* hpar = nullptr;     // pinned staging of cgpar
  void* cg_exec[2] = {nullptr, nullptr};  // instantiated CG batch graphs (FP64, FP32 Krylov)
  void* cg_loop[2] = {nullptr, nullptr};  // instantiated device-driven CG loops (conditional WHILE node)
  bool cg_loop_failed[2] = {false, false};  // the loop graph could not be built: use the batches
  // MDSC two-level preconditioner (allocated on first use); arrays typed like the column factors
  double* mP = nullptr;     // [L][4][nv] semicoarsening prolongation blocks of levels 0..L-1 (top = I)
  double* mAc = nullptr;    // [nbr][4] plane operator P^T J P, 2 x 2 blocks on the vertex neighbourhoods
  double* mDinv = nullptr;  // [nv][4] inverses of its diagonal blocks
  double* mcheb = nullptr;  // Chebyshev coefficients: [0] 1/theta, then per step (rho' rho, 2 rho' / delta)
  double* mlam = nullptr;   // Gershgorin bound of D^-1 A_c (device)
  double *mz1 = nullptr, *mt = nullptr, *ms = nullptr;  // [ndof] fine scratch
  double *mrc = nullptr, *mec = nullptr, *mrr = nullptr, *md0 = nullptr, *md1 = nullptr;  // [2 nv]
  int64_t nbr_total = 0;
  bool has_mdsc = false, mdsc_f32 = false, has_amg = false;
  void* mdsc_loop[2] = {nullptr, nullptr};  // device-driven PCG loops with the MDSC cycle
  // GMRES(m): Krylov basis (m + 1 vectors, double storage) and the Hessenberg column / coefficients
  void* amg = nullptr;        // smoothed-aggregation hierarchy of the MDSC plane solve (built once per mesh)
  void* amg_loop[2] = {nullptr, nullptr};  // device-driven PCG loops with the MDSC-AMG cycle
  double* gm_basis = nullptr;
  double* gm_h = nullptr;
  int gm_cap = 0;
};

struct bp_mesh {
  int device = 0;
  int32_t nv = 0, ntri = 0, nl = 0;
  int64_t ndof = 0, nnz = 0;
  bp_params p{};
  double cA = 0.0;  // A^(-1/3): 2 mu = cA (eps_e^2 + delta)^(-1/3) for n = 3

  // per vertex
  double2* xy = nullptr;
  double* bed = nullptr;
  double* thick = nullptr;
  double* beta = nullptr;
  int64_t* vstart = nullptr;  // first CSR entry of the vertex's row block
  int32_t* vdeg = nullptr;    // |{a} U neighbours(a)|
  int32_t* nbr_ptr = nullptr; // [nv + 1] sorted closed neighbourhoods
  int32_t* nbr_idx = nullptr;
  // per level
  double* sigma = nullptr;    // [L + 1] levels sigma_l, then [L] inverse layer thicknesses 1 / (sigma_{l+1} - sigma_l)
  // per triangle
  int32_t* tri = nullptr;     // [ntri][3]
  int32_t* slots = nullptr;   // [ntri][9]: slot[a][b] = rank of tri[b] in the closed neighbourhood of tri[a]
  double* basal = nullptr;    // [ntri][6]: basal friction matrix entries 00 01 02 11 12 22
  int32_t* color_tris = nullptr;  // [ntri] triangles grouped by colour
  std::vector<int32_t> color_off; // host copy: [ncolors + 1]
  int32_t ncolors = 0;
  // per dof / per entry
  int64_t* rowptr = nullptr;
  int32_t* colidx = nullptr;
  double* load = nullptr;     // [ndof] solution-independent load: driving stress rho g grad s . int N_i
                              // (+ the ocean margin load with BP_MARGIN_OCEAN)
  double* Bnode = nullptr;    // [nv][L + 1] hardness A^(-1/3) of the rate-factor field (NULL: uniform cA)
  double* Bnode_buf = nullptr;  // its storage (kept when the field is switched off)
  int2* bedges = nullptr;     // boundary edges a -> b (ocean margin condition only)
  int nbedges = 0;
  double* rscratch = nullptr; // [ndof] residual scratch for Jacobian calls with R = NULL
  uint16_t* mlp_X = nullptr;  // [nv][16] BF16 features of the learned guess
  float* mlp_Y = nullptr;     // [nv][32] network outputs
  double* mlp_q = nullptr;    // [16][nv] feature quantities (local, ~5 km, ~15 km, scratch)

  int64_t device_bytes = 0;
  std::vector<void*> allocations;
  bp_solver_ws* ws = nullptr;
};

void bp_solver_ws_free(bp_mesh* m);
// nodal area-weighted surface gradient accumulators [3][nv] (sum area * grad s, sum area), in mesh scratch
int bp_nodal_surface_gradient(bp_mesh* m, double** acc, cudaStream_t s);
// ||v||_2 of an ndof vector (synchronous)
int bp_norm2_host(bp_mesh* m, const double* v, cudaStream_t s, double* out);
// scratch of the learned guess: features, outputs, a shallow-ice guess, a residual
// bp_assemble_jacobian with the option to leave out the eta' rank-one part of the sum-factorised
// Jacobian (picard = 1: the fixed-viscosity matrix of a Picard step).
int bp_assemble_jacobian_ex(bp_mesh* m, const double* U, double* R, void* J, int precision, int scatter, int method,
                            int picard, void* stream);
int bp_learned_scratch(bp_mesh* m, uint16_t** X, float** Y, double** Usia, double** R, double** red);

// Allocation helper that records the pointer in the mesh (freed by bp_mesh_free).
template <class T>
int bp_alloc(bp_mesh* m, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  void* p = nullptr;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return BP_ENOMEM;
  }
  m->allocations.push_back(p);
  m->device_bytes += (int64_t)(count * sizeof(T));
  *ptr = static_cast<T*>(p);
  return BP_OK;
}

// Makes the mesh's device current for the scope of a call and restores the caller's device.
struct bp_device_guard {
  int prev = -1;
  explicit bp_device_guard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~bp_device_guard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// The kernels read velocity pairs (u, v) as one 16-byte load.
__host__ __device__ inline bool bp_aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
__host__ __device__ inline bool bp_aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

// Jacobian precision kinds whose values are stored as float (the others store double).
__host__ __device__ inline bool bp_values_f32(int precision) {
  return precision == BP_F32 || precision == BP_F32_ALL || precision == BP_F32_DS;
}

// Node level helpers of the extruded CSR pattern.
__host__ __device__ inline int bp_nlev(int level, int L) { return (level == 0 || level == L) ? 2 : 3; }
__host__ __device__ inline int bp_levels_before(int level) { return level == 0 ? 0 : 3 * level - 1; }
// Binary64 <-> binary32 conversions done on the integer pipe by repacking the IEEE 754 fields
// (sign; exponent rebiased between 1023 and 127; fraction cut from 52 to 23 bits or widened).
// B300 runs conversions from or to FP64 on its narrow FP64 pipe, which the kernels that use these
// keep busy with FP64 arithmetic; the integer pipe is otherwise idle there.
//   f32_of: rounds to nearest with ties away from zero (IEEE rounds ties to even: the two differ
//   only when the 29 dropped bits are exactly 1000...0).  Magnitudes below the FP32 normal range
//   give a signed zero, above it an infinity; NaN stays NaN.
__device__ __forceinline__ float f32_of(const double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7FFu;
  unsigned m = ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  m += (lo >> 28) & 1u;  // the first dropped bit; a carry moves into the exponent
  m = e <= 896u ? 0u : m;
  const unsigned big = (e == 0x7FFu && ((hi & 0xFFFFFu) | lo) != 0u) ? 0x7FC00000u : 0x7F800000u;
  m = e >= 1151u ? big : m;
  return __uint_as_float((hi & 0x80000000u) | m);
}
//   f64_of: exact for normal FP32 numbers, zeros, infinities and NaN; subnormals give a signed zero.
__device__ __forceinline__ double f64_of(const float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned frac = e == 0u ? 0u : (b & 0x7FFFFFu);
  const unsigned E = e == 0u ? 0u : (e == 0xFFu ? 0x7FFu : e + 896u);
  const unsigned hi = (b & 0x80000000u) | (E << 20) | (frac >> 3);
  return __hiloint2double((int)hi, (int)(frac << 29));
}

// x^(-1/3) for the viscosity, FP64-accurate with little FP64 work: an FP32 seed y (rcbrtf, relative
// error ~1e-7) refined once with the binomial series of (1 - e)^(-1/3), e = 1 - x y^3:
//   x^(-1/3) = y (1 - e)^(-1/3) = y (1 + e/3 + 2 e^2/9 + O(e^3)),
// a third-order correction whose truncation error (~e^3 / 6 ~ 1e-21) is far below FP64 rounding;
// 6 FP64 operations, the two conversions on the integer pipe.  Outside the FP32 normal range the
// library rcbrt is used.
__device__ __forceinline__ double inv_cbrt(double x) {
  // the FP32 seed needs x in [2^-99, 2^100): a test of the high word on the integer pipe (negative
  // values, zero, infinities and NaN fail it too), which keeps comparisons off the FP64 pipe
  if ((uint32_t)__double2hiint(x) - (924u << 20) >= (199u << 20)) return rcbrt(x);
  const double y = f64_of(rcbrtf(f32_of(x)));
  const double e = fma(-x * y, y * y, 1.0);
  return fma(y * e, fma(2.0 / 9.0, e, 1.0 / 3.0), y);
}

__host__ __device__ inline int64_t bp_dof(int64_t a, int l, int c, int L) {
  return 2 * (a * (L + 1) + l) + c;
}
