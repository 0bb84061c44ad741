// Newton-Krylov solve of the discrete first-order Stokes system (paper Sec. 3.1, Eq. linearsystem):
// CSR SpMV ("Op*x"), a vertical-line block-tridiagonal preconditioner (the per-line batched LU of
// Sec. 4.4, here used directly as the preconditioner), preconditioned CG with device-resident
// scalars (the Jacobian is symmetric positive definite: it is the Hessian of a convex energy),
// the discrete energy for the damped-Newton line search, and a shallow-ice initial guess.
#include <algorithm>
#include <memory>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "bp_ds.cuh"
#include "bp_internal.cuh"

namespace {

constexpr int MAXL = 64;       // largest layer count the column kernels handle
constexpr int TPR = 4;         // SpMV threads per row pair of FP32 values (grid sizing; spmv_group)
constexpr int NT = 256;        // threads per block of the vector kernels
constexpr int SCAL_CAP = 8192; // Krylov iterations per linear solve (scalar history capacity)
constexpr int GRID_CAP = 148 * 8;  // grid-stride kernels: 8 blocks of NT per SM
constexpr int UPD_NT = 128;        // threads of the staged CG update (one warp solves the block's columns)
constexpr int CG_BATCH = 8;        // CG iterations per replay of the captured batch graph
constexpr int LOOP_BODY = 4;       // CG iterations per pass of the device-driven loop
constexpr int GMRES_MAX_RESTART = 64;  // largest GMRES restart length

// Programmatic dependent launch inside the CG loop: each kernel lets the next one be scheduled at
// once (its blocks then wait on the SM instead of behind the launch latency) and waits for the
// previous kernel's completion and memory before it touches data the previous kernels produce or
// still read.  Both instructions do nothing in a launch without the programmatic attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Bulk asynchronous copies (the non-tensor TMA form): one thread moves a contiguous global range into
// shared memory and the copy signals an mbarrier with its byte count.  Both addresses and the size
// must be multiples of 16 bytes.  Waits are bounded: after BULK_WAIT_SPINS polls the caller gets
// false and flags an error instead of hanging.
constexpr int BULK_WAIT_SPINS = 1 << 22;
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  for (int it = 0; it < BULK_WAIT_SPINS; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (done) return true;
    if (it > 16) __nanosleep(32);
  }
  return false;
}

// B300 issues FP64 at ~1/64 of the FP32 rate, so the vector kernels keep per-element reductions in
// the vector type V and spend FP64 operations only on per-warp / per-block partial sums.
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of v (summed in T within each warp, in FP64 across warps), atomically added to
// *out.  Every thread of the block must call it.
template <class T>
__device__ __forceinline__ void block_add(T v, double* out) {
  __shared__ double sh[NT / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    w = warp_sum(w);
    if (threadIdx.x == 0) atomicAdd(out, w);
  }
  __syncthreads();
}

// ------------------------------------------------------------------ vectors
template <class A, class B>
__global__ void __launch_bounds__(NT) k_dot(const A* __restrict__ a, const B* __restrict__ b, int64_t n,
                                            double* out) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)a[i] * (double)b[i];
  block_add(s, out);
}

template <class V>
__global__ void __launch_bounds__(NT) k_axpy_to(const double* __restrict__ U, const V* __restrict__ d, double alpha,
                                                int64_t n, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = U[i] + alpha * (double)d[i];
}

__global__ void k_find_dslot(const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx, int nv,
                             int32_t* __restrict__ dslot) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  int s = 0;
  for (int k = nbr_ptr[a]; k < nbr_ptr[a + 1]; ++k)
    if (nbr_idx[k] == a) s = k - nbr_ptr[a];
  dslot[a] = s;
}

// ------------------------------------------------------------------ SpMV
// a * b + c with one rounding in the type of the operands (fmaf for FP32: the overload set of fma
// would otherwise be free to promote to FP64)
__device__ __forceinline__ float vfma(const float a, const float b, const float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(const double a, const double b, const double c) { return fma(a, b, c); }
// a matrix value in the vector type: FP32 values widen on the integer pipe (f64_of) when the
// vectors are FP64, so that the FP64 pipe does only the products
template <class V, class M>
__device__ __forceinline__ V mat_v(const M x) {
  if constexpr (std::is_same<V, double>::value && std::is_same<M, float>::value) {
    return f64_of(x);
  } else {
    return (V)x;
  }
}

template <class T>
struct Pair;
template <>
struct Pair<double> {
  using type = double2;
};
template <>
struct Pair<float> {
  using type = float2;
};

// y = A x on the extruded pattern, one row pair per group of G threads (spmv_group).  Rows 2i and 2i + 1 (the u
// and v rows of node i = (a, l)) are adjacent in the CSR arrays and have the same columns: for each b
// of the sorted closed neighbourhood of vertex a, levels lmin .. lmin + nlev - 1, components u, v.
// Column indices are therefore rebuilt from the neighbour list instead of read from colidx (which
// halves the bytes of an FP32 SpMV), x is read as aligned (u, v) pairs and the values of both rows as
// aligned pairs.  The two row sums are folded with one add per lane per step (after the first step
// the lower half of the group carries row 2i, the upper half row 2i + 1).  With DOT, x . y is added
// to *dot (summed in V per thread, in FP64 across threads, one atomic per block; inside the CG
// batch graph the target is scal[3 (kbase + j)]).  Grid-stride over row pairs.
// threads per row pair of the SpMV: 4 for FP32 values (HBM-bound: more row pairs in flight per warp
// would cost registers), 2 for FP64 values (bound by the FP64 pipe, which a group of 4 leaves idle
// on more lanes in the last steps of short rows: FP64 Krylov phase 25.7 -> 24.5 ms at 1M wedges)
template <class M>
__host__ __device__ constexpr int spmv_group() {
  return std::is_same<M, float>::value ? 4 : 2;
}
// resident blocks of NT threads asked of the register allocator: the FP32 product is bound by memory
// latency and needs every warp slot (32 registers: 8 blocks per SM; at 40 registers, 6 blocks, the
// mixed-precision Krylov phase took 12.3 instead of 10.3 ms); the FP64-vector products take up to
// 64 registers (4 blocks) and spill below 48
template <class M, class V>
__host__ __device__ constexpr int spmv_min_blocks() {
  return std::is_same<V, float>::value ? 8 : 4;
}

template <class M, class V, bool DOT>
__global__ void __launch_bounds__(NT, spmv_min_blocks<M, V>()) k_spmv_pairs(const int64_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ nbr_ptr,
                                                   const int32_t* __restrict__ nbr_idx, int L,
                                                   const M* __restrict__ vals, int npairs, const V* __restrict__ x,
                                                   V* __restrict__ y, double* dot, const int* stop,
                                                   const int* kbase, int j) {
  using M2 = typename Pair<M>::type;
  using V2 = typename Pair<V>::type;
  pdl_trigger();
  pdl_wait();
  if (stop && *stop) return;
  if (DOT && kbase) dot += 3 * (*kbase + j);  // CG iteration k = kbase + j writes scal[3k]
  constexpr int G = spmv_group<M>();  // threads per row pair
  const int lane = threadIdx.x % G;
  const bool upper = lane >= G / 2;
  V d = V(0);  // this thread's part of x . y (in V; FP64 only across threads)
  // warp-uniform loop bound: the shuffles below need all 32 lanes of the warp
  const int stride = gridDim.x * (NT / G);
  // the row pair's header (first entry, row length, neighbourhood start) is loaded one grid-stride
  // step ahead, so that its loads are in flight while the previous row pair is summed
  const int first = blockIdx.x * (NT / G) + (threadIdx.x / 32) * (32 / G) + (threadIdx.x % 32) / G;
  int64_t h_s0 = 0, h_s1 = 0;
  int h_nb = 0;
  if (first < npairs) {
    h_s0 = rowptr[2 * (int64_t)first];
    h_s1 = rowptr[2 * (int64_t)first + 1];
    h_nb = nbr_ptr[first / (L + 1)];
  }
  for (int base = blockIdx.x * (NT / G) + (threadIdx.x / 32) * (32 / G); base < npairs; base += stride) {
    const int pr = base + (threadIdx.x % 32) / G;
    const int64_t s0 = h_s0;
    const int half = (int)((h_s1 - s0) >> 1);  // column pairs per row = deg nlev
    const int nbp = h_nb;
    const int prn = pr + stride;
    if (prn < npairs) {
      h_s0 = rowptr[2 * (int64_t)prn];
      h_s1 = rowptr[2 * (int64_t)prn + 1];
      h_nb = nbr_ptr[prn / (L + 1)];
    }
    V y0 = V(0), y1 = V(0);
    if (pr < npairs) {
      const int a = pr / (L + 1);
      const int l = pr - a * (L + 1);
      const int nlev = bp_nlev(l, L);
      const int lmin = l > 0 ? l - 1 : 0;
      const int32_t* nb = nbr_idx + nbp;
      const M2* v0 = reinterpret_cast<const M2*>(vals + s0);
      const M2* v1 = v0 + half;
      // k = sl nlev + dl formed afresh in every step (nlev is 2 or 3: a shift or a multiply-high),
      // so that no step depends on the one before and the unrolled steps' loads are all in flight
      // (unrolled 4 deep for FP64 values, whose FMAs bind; 2 for FP32, where deeper unrolling
      // costs registers and resident warps: measured on the 1M-wedge Newton solve)
      constexpr int UNR = sizeof(M) == sizeof(double) ? 4 : 2;
#pragma unroll UNR
      for (int k = lane; k < half; k += G) {
        const int sl = nlev == 3 ? k / 3 : k >> 1;
        const int dl = k - sl * nlev;
        const int b = __ldg(nb + sl);
        const V2 xx = *reinterpret_cast<const V2*>(x + 2 * ((int64_t)b * (L + 1) + lmin + dl));
        const M2 a0 = v0[k], a1 = v1[k];
        // chained FMAs: one FMA per matrix entry (a sum of two products first would cost a
        // multiply, an FMA and an add per pair, 1.5 instructions per entry on the FP64 pipe)
        y0 = vfma(mat_v<V>(a0.y), xx.y, vfma(mat_v<V>(a0.x), xx.x, y0));
        y1 = vfma(mat_v<V>(a1.y), xx.y, vfma(mat_v<V>(a1.x), xx.x, y1));
      }
    }
    V keep = upper ? y1 : y0;
    keep += __shfl_xor_sync(0xffffffffu, upper ? y0 : y1, G / 2, G);
#pragma unroll
    for (int o = G / 4; o; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o, G);
    if (pr < npairs && (lane == 0 || lane == G / 2)) {
      const int64_t row = 2 * (int64_t)pr + (upper ? 1 : 0);
      y[row] = keep;
      if (DOT) d += x[row] * keep;
    }
  }
  if (DOT && dot) {  // only lanes 0 and G / 2 of each group hold a partial: one warp adds them
    __shared__ double sd[2 * NT / G];
    if (lane == 0 || lane == G / 2) sd[2 * (threadIdx.x / G) + (upper ? 1 : 0)] = (double)d;
    __syncthreads();
    if (threadIdx.x < 32) {
      double w = 0.0;
      for (int i = threadIdx.x; i < 2 * NT / G; i += 32) w += sd[i];
      w = warp_sum(w);
      if (threadIdx.x == 0) atomicAdd(dot, w);
    }
  }
}

// ------------------------------------------------------------------ column preconditioner
__device__ __forceinline__ int64_t col_entry(int64_t vs, int dg, int ds, int l, int c, int lp, int cp, int L) {
  const int nl = bp_nlev(l, L);
  const int lmin = l > 0 ? l - 1 : 0;
  return vs + (int64_t)dg * (4 * bp_levels_before(l) + 2 * c * nl) + 2 * (ds * nl + lp - lmin) + cp;
}

// Block Thomas elimination of the column's block-tridiagonal part of J (2 x 2 blocks; arithmetic and
// factors in F: FP64 for the FP64 path, FP32 for the mixed-precision path, whose factors are FP32
// anyway and whose elimination would otherwise run on the narrow FP64 pipe, divisions included):
//   G_0 = D_0,  Lm_l = E_l G_{l-1}^-1,  G_l = D_l - Lm_l F_{l-1},  store Lm_l, G_l^-1, F_l.
template <class M, class F>
__global__ void __launch_bounds__(128) k_colprec_setup(const M* __restrict__ J, const int64_t* __restrict__ vstart,
                                                       const int32_t* __restrict__ vdeg,
                                                       const int32_t* __restrict__ dslot, int nv, int L,
                                                       F* __restrict__ Lm, F* __restrict__ Ginv,
                                                       F* __restrict__ Fu) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  const int64_t vs = vstart[a];
  const int dg = vdeg[a], ds = dslot[a];
  using A = F;  // arithmetic type
  auto at = [&](int l, int c, int lp, int cp) -> A {
    return (A)J[col_entry(vs, dg, ds, l, c, lp, cp, L)];
  };
  A Gp[4] = {0, 0, 0, 0}, Fp[4] = {0, 0, 0, 0};
  for (int l = 0; l <= L; ++l) {
    A G[4] = {at(l, 0, l, 0), at(l, 0, l, 1), at(l, 1, l, 0), at(l, 1, l, 1)};
    if (l > 0) {
      const A E[4] = {at(l, 0, l - 1, 0), at(l, 0, l - 1, 1), at(l, 1, l - 1, 0), at(l, 1, l - 1, 1)};
      const A Lmat[4] = {E[0] * Gp[0] + E[1] * Gp[2], E[0] * Gp[1] + E[1] * Gp[3],
                         E[2] * Gp[0] + E[3] * Gp[2], E[2] * Gp[1] + E[3] * Gp[3]};
      G[0] -= Lmat[0] * Fp[0] + Lmat[1] * Fp[2];
      G[1] -= Lmat[0] * Fp[1] + Lmat[1] * Fp[3];
      G[2] -= Lmat[2] * Fp[0] + Lmat[3] * Fp[2];
      G[3] -= Lmat[2] * Fp[1] + Lmat[3] * Fp[3];
#pragma unroll
      for (int e = 0; e < 4; ++e) Lm[((int64_t)(l - 1) * 4 + e) * nv + a] = (F)Lmat[e];
    }
    const A idet = A(1) / (G[0] * G[3] - G[1] * G[2]);
    Gp[0] = G[3] * idet;
    Gp[1] = -G[1] * idet;
    Gp[2] = -G[2] * idet;
    Gp[3] = G[0] * idet;
#pragma unroll
    for (int e = 0; e < 4; ++e) Ginv[((int64_t)l * 4 + e) * nv + a] = (F)Gp[e];
    if (l < L) {
      Fp[0] = at(l, 0, l + 1, 0);
      Fp[1] = at(l, 0, l + 1, 1);
      Fp[2] = at(l, 1, l + 1, 0);
      Fp[3] = at(l, 1, l + 1, 1);
#pragma unroll
      for (int e = 0; e < 4; ++e) Fu[((int64_t)l * 4 + e) * nv + a] = (F)Fp[e];
    }
  }
}

template <class F>
struct Prec {
  const F* Lm;
  const F* Ginv;
  const F* Fu;
  int nv, L;
};

// z = P^-1 r on column a (forward and backward block substitution, arithmetic in F); returns (r.z, r.r)
// of the column.  The column's 2(L+1) values start at r[off], z[off] (off = 2 a (L+1) for dof-ordered
// vectors).  The forward sweep's intermediate y is kept in z itself (V is at least as wide as F).
template <class V, class F>
__device__ __forceinline__ void colprec_apply(const Prec<F>& P, int a, const V* __restrict__ r, V* __restrict__ z,
                                              double* rz, double* rr, int64_t off) {
  const int L = P.L;
  const int64_t base = off;
  const int64_t nv = P.nv;
  F srr = F(0), p0 = F(0), p1 = F(0);
#pragma unroll 4
  for (int l = 0; l <= L; ++l) {
    F r0 = (F)r[base + 2 * l], r1 = (F)r[base + 2 * l + 1];
    srr = vfma(r1, r1, vfma(r0, r0, srr));  // chained FMAs: no separate multiply and add
    if (l > 0) {
      const F* Lp = P.Lm + (int64_t)(l - 1) * 4 * nv + a;
      r0 = vfma(-Lp[nv], p1, vfma(-Lp[0], p0, r0));
      r1 = vfma(-Lp[3 * nv], p1, vfma(-Lp[2 * nv], p0, r1));
    }
    z[base + 2 * l] = (V)r0;
    z[base + 2 * l + 1] = (V)r1;
    p0 = r0;
    p1 = r1;
  }
  F srz = F(0);
#pragma unroll 4
  for (int l = L; l >= 0; --l) {
    F t0 = (F)z[base + 2 * l], t1 = (F)z[base + 2 * l + 1];
    if (l < L) {
      const F* Fp = P.Fu + (int64_t)l * 4 * nv + a;
      t0 = vfma(-Fp[nv], p1, vfma(-Fp[0], p0, t0));
      t1 = vfma(-Fp[3 * nv], p1, vfma(-Fp[2 * nv], p0, t1));
    }
    const F* Gp = P.Ginv + (int64_t)l * 4 * nv + a;
    const F z0 = Gp[0] * t0 + Gp[nv] * t1;
    const F z1 = Gp[2 * nv] * t0 + Gp[3 * nv] * t1;
    z[base + 2 * l] = (V)z0;
    z[base + 2 * l + 1] = (V)z1;
    p0 = z0;
    p1 = z1;
    srz = vfma((F)r[base + 2 * l + 1], z1, vfma((F)r[base + 2 * l], z0, srz));
  }
  *rz = (double)srz;
  *rr = (double)srr;
}

template <class V, class F>
__global__ void __launch_bounds__(128) k_colprec_apply(const Prec<F> P, const V* __restrict__ r, V* __restrict__ z) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= P.nv) return;
  double rz, rr;
  colprec_apply(P, a, r, z, &rz, &rr, 2LL * a * (P.L + 1));
}

// ------------------------------------------------------------------ preconditioned CG (device scalars)
// scal[3k] = p_k . A p_k, scal[3k+1] = r_k . z_k, scal[3k+2] = r_k . r_k.
// CG start (FP64 vectors, and layer counts without a register-resident variant), staged like the
// update below: the block's C consecutive columns are one contiguous range of the dof-ordered
// vectors, so r = -R and x = 0 run coalesced (r.r summed by every thread), r goes to shared memory,
// each of the first C threads solves its column there, and z and p = z go back coalesced.
// Dynamic shared memory: 2 C 2(L+1) values of V.
template <class V, class F>
__global__ void __launch_bounds__(UPD_NT) k_cg_init_staged(const Prec<F> P, int C, const double* __restrict__ R,
                                                           V* __restrict__ x, V* __restrict__ r, V* __restrict__ z,
                                                           V* __restrict__ p, double* scal) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n = 2 * (P.L + 1);
  const int a0 = blockIdx.x * C;
  const int ncol = min(C, P.nv - a0);
  const int64_t base = (int64_t)a0 * n;
  const int cnt = ncol * n;
  V* sr = reinterpret_cast<V*>(smraw);
  V* sz = sr + C * n;
  V rr = V(0);
  double rz = 0.0;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const V rv = (V)(-R[base + i]);
    r[base + i] = rv;
    x[base + i] = V(0);
    sr[i] = rv;
    rr += rv * rv;
  }
  __syncthreads();
  if ((int)threadIdx.x < ncol) {
    double dummy_rr;
    colprec_apply(P, a0 + (int)threadIdx.x, sr, sz, &rz, &dummy_rr, (int64_t)threadIdx.x * n);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    z[base + i] = sz[i];
    p[base + i] = sz[i];
  }
  block_add(rz, scal + 1);
  block_add(rr, scal + 2);
}

// alpha = r.z / p.Ap;  x += alpha p;  r -= alpha q;  z = P^-1 r;  accumulate r.z, r.r of step k+1.
// Same step, staged for coalescing: the block's C consecutive columns occupy one contiguous range of
// the dof-ordered vectors, so x += alpha p and r -= alpha q run element-wise with coalesced accesses,
// r goes to shared memory, each of the first C threads solves its column there, and z is written back
// coalesced.  alpha is formed once per block.  Dynamic shared memory: 2 C 2(L+1) values of V.
template <class V, class F>
__global__ void __launch_bounds__(UPD_NT) k_cg_update_staged(const Prec<F> P, const int* kbase, int j, int C,
                                                             V* __restrict__ x, V* __restrict__ r, V* __restrict__ z,
                                                             const V* __restrict__ p, const V* __restrict__ q,
                                                             double* scal, int* stop) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ V s_alpha;
  __shared__ int s_bad;
  pdl_trigger();
  pdl_wait();
  if (*stop) return;
  const int k = *kbase + j;
  if (threadIdx.x == 0) {
    const double pq = scal[3 * k], rzk = scal[3 * k + 1];
    s_bad = !(pq > 0.0) || !isfinite(rzk);
    s_alpha = s_bad ? V(0) : (V)(rzk / pq);
    if (s_bad && blockIdx.x == 0) *stop = 2;
  }
  __syncthreads();
  if (s_bad) return;
  const V alpha = s_alpha;
  const int n = 2 * (P.L + 1);
  const int a0 = blockIdx.x * C;
  const int ncol = min(C, P.nv - a0);
  const int64_t base = (int64_t)a0 * n;
  const int cnt = ncol * n;
  V* sr = reinterpret_cast<V*>(smraw);
  V* sz = sr + C * n;
  V rr = V(0);
  double rz = 0.0;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const V xv = x[base + i] + alpha * p[base + i];
    const V rv = r[base + i] - alpha * q[base + i];
    x[base + i] = xv;
    r[base + i] = rv;
    sr[i] = rv;
    rr += rv * rv;
  }
  __syncthreads();
  if ((int)threadIdx.x < ncol) {
    double dummy_rr;
    colprec_apply(P, a0 + (int)threadIdx.x, sr, sz, &rz, &dummy_rr, (int64_t)threadIdx.x * n);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) z[base + i] = sz[i];
  block_add(rz, scal + 3 * (k + 1) + 1);
  block_add(rr, scal + 3 * (k + 1) + 2);
}

// FP32 columns with NLEV = L + 1 levels known at compile time (the CG step and its start below):
// one warp per 32 consecutive columns, every lane solves one column.  Each lane first loads its
// column's factors (NLEV - 1 lower, NLEV - 1 upper and NLEV inverse diagonal 2 x 2 blocks) into
// registers, so that the loads are all in flight together and the substitution does no global load
// (a single solving warp per block would wait on one factor load after another).  The warp's columns
// are one contiguous range of the dof-ordered vectors: the element-wise work runs coalesced, r is
// staged in shared memory (column stride padded to an odd count against bank conflicts), each lane
// solves its column in place, and z is written back coalesced.
template <int NLEV>
struct ColFactors {
  float Lf[NLEV - 1][4], Uf[NLEV - 1][4], Gf[NLEV][4];
  __device__ __forceinline__ void load(const Prec<float>& P, int a) {
    const int nv = P.nv;
#pragma unroll
    for (int l = 0; l < NLEV; ++l)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t o = ((int64_t)l * 4 + e) * nv + a;
        Gf[l][e] = P.Ginv[o];
        if (l < NLEV - 1) {
          Lf[l][e] = P.Lm[o];
          Uf[l][e] = P.Fu[o];
        }
      }
  }
  // z = P^-1 r for the column at c[0 .. 2 NLEV) (overwritten with z); returns r . z
  __device__ __forceinline__ float solve(float* c) const {
    constexpr int N = 2 * NLEV;
    float rv[N];
#pragma unroll
    for (int i = 0; i < N; ++i) rv[i] = c[i];
    // forward: y_0 = r_0, y_l = r_l - Lm_l y_{l-1}
    float y[N];
    y[0] = rv[0];
    y[1] = rv[1];
#pragma unroll
    for (int l = 1; l < NLEV; ++l) {
      const float* Lp = Lf[l - 1];
      y[2 * l] = rv[2 * l] - (Lp[0] * y[2 * l - 2] + Lp[1] * y[2 * l - 1]);
      y[2 * l + 1] = rv[2 * l + 1] - (Lp[2] * y[2 * l - 2] + Lp[3] * y[2 * l - 1]);
    }
    // backward: z_L = G_L^-1 y_L, z_l = G_l^-1 (y_l - F_l z_{l+1})
    float srz = 0.f, z0 = 0.f, z1 = 0.f;
#pragma unroll
    for (int l = NLEV - 1; l >= 0; --l) {
      float t0 = y[2 * l], t1 = y[2 * l + 1];
      if (l < NLEV - 1) {
        const float* Fp = Uf[l];
        t0 -= Fp[0] * z0 + Fp[1] * z1;
        t1 -= Fp[2] * z0 + Fp[3] * z1;
      }
      const float* Gp = Gf[l];
      z0 = Gp[0] * t0 + Gp[1] * t1;
      z1 = Gp[2] * t0 + Gp[3] * t1;
      c[2 * l] = z0;
      c[2 * l + 1] = z1;
      srz += rv[2 * l] * z0 + rv[2 * l + 1] * z1;
    }
    return srz;
  }
};

// CG step: alpha = r.z / p.Ap, x += alpha p, r -= alpha q, z = P^-1 r, and r.z, r.r of step k + 1.
// The warp's slices of x, r, p and q (32 columns: one contiguous range of each vector) arrive in
// shared memory by four bulk copies on one mbarrier, so that the element-wise step reads no global
// memory (as plain loads its 2 (L + 1) coalesced steps were one dependent round trip each); a slice
// whose length is not a multiple of 16 bytes (the last warp, odd column count) takes its last
// values by plain loads.  The factors go to registers before the wait on the previous kernel.
template <int NLEV>
__global__ void __launch_bounds__(UPD_NT) k_cg_update_cols(const Prec<float> P, const int* kbase, int j,
                                                           float* __restrict__ x, float* __restrict__ r,
                                                           float* __restrict__ z, const float* __restrict__ p,
                                                           const float* __restrict__ q, double* scal, int* stop) {
  constexpr int N = 2 * NLEV;  // values per column
  constexpr int W = 32 * N;    // values per warp slice
  __shared__ __align__(16) float sbuf[UPD_NT / 32][4][W];  // x, r (then z), p, q
  __shared__ uint64_t sbar[UPD_NT / 32];
  __shared__ float s_alpha;
  __shared__ int s_bad;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a0 = (blockIdx.x * (UPD_NT / 32) + warp) * 32;
  const bool own = a0 + lane < P.nv;
  const int ncol = min(32, P.nv - a0);  // <= 0 for a warp past the last column
  const int cnt = max(ncol, 0) * N;
  const int cnt16 = cnt & ~3;           // values moved by the bulk copies (whole 16-byte units)
  const int64_t base = (int64_t)max(a0, 0) * N;
  float* sx = sbuf[warp][0];
  float* sr = sbuf[warp][1];
  float* sp = sbuf[warp][2];
  float* sq = sbuf[warp][3];
  if (lane == 0 && cnt16 > 0) mbar_init(&sbar[warp]);
  pdl_trigger();
  ColFactors<NLEV> f;  // the factors do not depend on the previous kernels: load them before waiting
  if (own) f.load(P, a0 + lane);
  pdl_wait();
  if (*stop) return;
  const int k = *kbase + j;
  if (threadIdx.x == 0) {
    const double pq = scal[3 * k], rzk = scal[3 * k + 1];
    s_bad = !(pq > 0.0) || !isfinite(rzk);
    s_alpha = s_bad ? 0.f : (float)(rzk / pq);
    if (s_bad && blockIdx.x == 0) *stop = 2;
  }
  __syncthreads();
  if (s_bad) return;
  const float alpha = s_alpha;
  bool ok = true;
  if (cnt16 > 0) {
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)cnt16 * 4u;
      mbar_expect(&sbar[warp], 4u * bytes);
      bulk_load(sx, x + base, bytes, &sbar[warp]);
      bulk_load(sr, r + base, bytes, &sbar[warp]);
      bulk_load(sp, p + base, bytes, &sbar[warp]);
      bulk_load(sq, q + base, bytes, &sbar[warp]);
    }
    for (int i = cnt16 + lane; i < cnt; i += 32) {
      sx[i] = x[base + i];
      sr[i] = r[base + i];
      sp[i] = p[base + i];
      sq[i] = q[base + i];
    }
    ok = mbar_wait(&sbar[warp], 0);
    if (!__all_sync(0xffffffffu, ok)) {  // the copies did not complete in time: flag, drain, skip
      if (lane == 0) *stop = 5;
      mbar_wait(&sbar[warp], 0);
      ok = false;
    }
  }
  __syncwarp();
  float rr = 0.f;
  double rz = 0.0;
  if (ok) {
    for (int i = lane; i < cnt; i += 32) {
      const float xv = sx[i] + alpha * sp[i];
      const float rv = sr[i] - alpha * sq[i];
      x[base + i] = xv;
      r[base + i] = rv;
      sr[i] = rv;
      rr += rv * rv;
    }
    __syncwarp();
    if (own) rz = (double)f.solve(sr + lane * N);
    __syncwarp();
    for (int i = lane; i < cnt; i += 32) z[base + i] = sr[i];
  }
  block_add(rz, scal + 3 * (k + 1) + 1);
  block_add(rr, scal + 3 * (k + 1) + 2);
}

// CG start: x = 0, r = -R, z = P^-1 r, p = z, and r.z, r.r of step 0.  The warp's slice of R comes
// to shared memory by one bulk copy (its odd tail, if any, by plain loads), as in the update.
template <int NLEV>
__global__ void __launch_bounds__(UPD_NT) k_cg_init_cols(const Prec<float> P, const double* __restrict__ R,
                                                         float* __restrict__ x, float* __restrict__ r,
                                                         float* __restrict__ z, float* __restrict__ p,
                                                         double* scal, int* stop) {
  constexpr int N = 2 * NLEV;
  constexpr int W = 32 * N;
  __shared__ __align__(16) double sR[UPD_NT / 32][W];
  __shared__ __align__(16) float sbuf[UPD_NT / 32][W];
  __shared__ uint64_t sbar[UPD_NT / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a0 = (blockIdx.x * (UPD_NT / 32) + warp) * 32;
  const bool own = a0 + lane < P.nv;
  const int ncol = min(32, P.nv - a0);
  const int cnt = max(ncol, 0) * N;
  const int cnt16 = cnt & ~1;  // FP64 values moved by the bulk copy (whole 16-byte units)
  const int64_t base = (int64_t)max(a0, 0) * N;
  double* sd = sR[warp];
  float* sr = sbuf[warp];
  bool ok = true;
  if (cnt16 > 0) {
    if (lane == 0) {
      mbar_init(&sbar[warp]);
      mbar_expect(&sbar[warp], (uint32_t)cnt16 * 8u);
      bulk_load(sd, R + base, (uint32_t)cnt16 * 8u, &sbar[warp]);
    }
    for (int i = cnt16 + lane; i < cnt; i += 32) sd[i] = R[base + i];
  }
  ColFactors<NLEV> f;
  if (own) f.load(P, a0 + lane);
  if (cnt16 > 0) {
    __syncwarp();  // the barrier's initialisation before the other lanes poll it
    ok = mbar_wait(&sbar[warp], 0);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) *stop = 5;
      mbar_wait(&sbar[warp], 0);
      ok = false;
    }
  }
  __syncwarp();
  float rr = 0.f;
  double rz = 0.0;
  if (ok) {
    for (int i = lane; i < cnt; i += 32) {
      const float rv = -f32_of(sd[i]);
      x[base + i] = 0.f;
      r[base + i] = rv;
      sr[i] = rv;
      rr += rv * rv;
    }
    __syncwarp();
    if (own) rz = (double)f.solve(sr + lane * N);
    __syncwarp();
    for (int i = lane; i < cnt; i += 32) {
      const float zv = sr[i];
      z[base + i] = zv;
      p[base + i] = zv;
    }
  }
  block_add(rz, scal + 1);
  block_add(rr, scal + 2);
}

// beta = r_{k+1}.z_{k+1} / r_k.z_k;  p = z + beta p;  stop once r.r <= eta^2 r_0.r_0 (flag 1), the
// iteration limit is reached (flag 4) or r.r is not finite (flag 3, a breakdown that the Newton
// solve reports as BP_ENAN).  The scalars are formed once per block; the update runs on (u, v) pairs.
// Inside the device-driven loop (set_loop != 0) the first thread of block 0 also sets the loop's
// condition on every path: 1 only when no stop flag is up after this iteration, so the loop ends at
// convergence, at the iteration limit, or after a breakdown flagged by the update.
template <class V>
__global__ void __launch_bounds__(NT) k_cg_direction(const int* kbase, int j, const double* cgpar, int64_t npairs,
                                                     const V* __restrict__ z, V* __restrict__ p, const double* scal,
                                                     int* stop, cudaGraphConditionalHandle loop, int set_loop) {
  using V2 = typename Pair<V>::type;
  __shared__ V s_beta;
  __shared__ int s_done;
  pdl_trigger();
  pdl_wait();
  if (threadIdx.x == 0) {
    int done = *stop != 0;
    if (!done) {
      const int k = *kbase + j;
      const double rr = scal[3 * (k + 1) + 2];
      const bool bad = !isfinite(rr);
      const bool conv = rr <= cgpar[0] * scal[2];
      const bool limit = (double)(k + 1) >= cgpar[1];
      done = bad || conv || limit;
      s_beta = (V)(scal[3 * (k + 1) + 1] / scal[3 * k + 1]);
      if (done && blockIdx.x == 0) *stop = bad ? 3 : conv ? 1 : 4;
    }
    s_done = done;
    if (set_loop && blockIdx.x == 0) cudaGraphSetConditional(loop, done ? 0u : 1u);
  }
  __syncthreads();
  if (s_done) return;
  const V beta = s_beta;
  const V2* z2 = reinterpret_cast<const V2*>(z);
  V2* p2 = reinterpret_cast<V2*>(p);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npairs; i += (int64_t)gridDim.x * blockDim.x) {
    const V2 zz = z2[i];
    V2 pp = p2[i];
    pp.x = zz.x + beta * pp.x;
    pp.y = zz.y + beta * pp.y;
    p2[i] = pp;
  }
}

// end of a CG batch: the next batch starts BATCH iterations later
__global__ void k_cg_advance(int* kbase, int batch) {
  pdl_wait();
  *kbase += batch;
}

// ------------------------------------------------------------------ energy
// FP64 <-> arithmetic type T of the energy change; FP32 converts on the integer pipe (f32_of,
// f64_of), which leaves the FP64 pipe to the FP64 part of the kernel.
template <class T>
__device__ __forceinline__ T to_T(const double x) {
  return T(x);
}
template <>
__device__ __forceinline__ float to_T<float>(const double x) {
  return f32_of(x);
}
template <>
__device__ __forceinline__ f64x2 to_T<f64x2>(const double x) {
  return ds_of(x);
}
__device__ __forceinline__ double from_T(const double x) { return x; }
__device__ __forceinline__ double from_T(const float x) { return f64_of(x); }
__device__ __forceinline__ double from_T(const f64x2 x) { return ds_value(x); }
// a direction entry (type DT) in the arithmetic type T
template <class T, class DT>
__device__ __forceinline__ T dir_T(const DT x) {
  if constexpr (std::is_same<T, f64x2>::value) {
    return ds_of((double)x);
  } else if constexpr (std::is_same<T, float>::value && std::is_same<DT, double>::value) {
    return f32_of(x);  // on the integer pipe
  } else {
    return (T)x;
  }
}

// Hardness B = A^(-1/3) at the quadrature point (zeta level weights p0, p1 of layer l, triangle point
// tp): the nodal field interpolated like the velocity, or the uniform value cA.
__device__ __forceinline__ double hardness_at(const double* __restrict__ Bn, double cA, const int v[3], int L,
                                              int l, double p0, double p1, int tp) {
  if (!Bn) return cA;
  double lo = 0.0, hi = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double la = (a == tp) ? 2.0 / 3.0 : 1.0 / 6.0;
    lo += la * Bn[(int64_t)v[a] * (L + 1) + l];
    hi += la * Bn[(int64_t)v[a] * (L + 1) + l + 1];
  }
  return p0 * lo + p1 * hi;
}
// The same in arithmetic T (FP32 for the mixed-precision energy change: the nodal values are rounded
// once and interpolated in FP32).
template <class T>
__device__ __forceinline__ T hardness_at_t(const double* __restrict__ Bn, T cA, const int v[3], int L, int l, T p0,
                                           T p1, int tp) {
  if (!Bn) return cA;
  T lo = T(0), hi = T(0);
  for (int a = 0; a < 3; ++a) {
    const T la = T((a == tp) ? 2.0 / 3.0 : 1.0 / 6.0);
    lo += la * to_T<T>(Bn[(int64_t)v[a] * (L + 1) + l]);
    hi += la * to_T<T>(Bn[(int64_t)v[a] * (L + 1) + l + 1]);
  }
  return p0 * lo + p1 * hi;
}
// Pi_h = sum_q c_q (3/2) A^(-1/3) (eps_e^2 + delta)^(2/3) + load . U + 1/2 sum_bed U_b^T M U_b   (n = 3)
__global__ void __launch_bounds__(128) k_energy(const double2* __restrict__ xy, const double* __restrict__ bed,
                                                const double* __restrict__ thick, const double* __restrict__ sigma,
                                                const int32_t* __restrict__ tri, const double* __restrict__ basal,
                                                const double* __restrict__ load, int ntri, int L, int64_t ndof,
                                                double cA, const double* __restrict__ Bn, double delta,
                                                const double* __restrict__ U, double* out) {
  double acc = 0.0;
  // driving-stress part: load . U
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ndof; i += (int64_t)gridDim.x * blockDim.x)
    acc += load[i] * U[i];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ntri) {
    int v[3];
    double x[3], y[3], H[3], bb[3];
    for (int a = 0; a < 3; ++a) {
      v[a] = tri[3 * t + a];
      const double2 p = xy[v[a]];
      x[a] = p.x;
      y[a] = p.y;
      H[a] = thick[v[a]];
      bb[a] = bed[v[a]];
    }
    const double d = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
    const double inv_d = 1.0 / d;
    double lx[3], ly[3];
    for (int a = 0; a < 3; ++a) {
      lx[a] = (y[(a + 1) % 3] - y[(a + 2) % 3]) * inv_d;
      ly[a] = (x[(a + 2) % 3] - x[(a + 1) % 3]) * inv_d;
    }
    const double gbx = bb[0] * lx[0] + bb[1] * lx[1] + bb[2] * lx[2];
    const double gby = bb[0] * ly[0] + bb[1] * ly[1] + bb[2] * ly[2];
    const double gHx = H[0] * lx[0] + H[1] * lx[1] + H[2] * lx[2];
    const double gHy = H[0] * ly[0] + H[1] * ly[1] + H[2] * ly[2];
    const double Hs6 = (H[0] + H[1] + H[2]) * (1.0 / 6.0);
    double Hq[3];
    for (int tp = 0; tp < 3; ++tp) Hq[tp] = Hs6 + 0.5 * H[tp];
    int64_t ub[3];
    for (int a = 0; a < 3; ++a) ub[a] = 2LL * v[a] * (L + 1);
    // basal friction energy
    {
      const double* Mb = basal + 6 * (int64_t)t;
      const double M[3][3] = {{Mb[0], Mb[1], Mb[2]}, {Mb[1], Mb[3], Mb[4]}, {Mb[2], Mb[4], Mb[5]}};
      double uu[3], vv[3];
      for (int a = 0; a < 3; ++a) {
        uu[a] = U[ub[a]];
        vv[a] = U[ub[a] + 1];
      }
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) acc += 0.5 * M[a][b] * (uu[a] * uu[b] + vv[a] * vv[b]);
    }
    for (int l = 0; l < L; ++l) {
      double u0[3], v0[3], u1[3], v1[3];
      for (int a = 0; a < 3; ++a) {
        u0[a] = U[ub[a] + 2 * l];
        v0[a] = U[ub[a] + 2 * l + 1];
        u1[a] = U[ub[a] + 2 * l + 2];
        v1[a] = U[ub[a] + 2 * l + 3];
      }
      const double s_l = sigma[l], ds = sigma[l + 1] - sigma[l];
      for (int z = 0; z < 2; ++z) {
        const double p0 = z == 0 ? BP_QP_P : BP_QP_Q, p1 = z == 0 ? BP_QP_Q : BP_QP_P;
        const double sz = s_l + p1 * ds;
        const double Gzx = gbx + sz * gHx, Gzy = gby + sz * gHy;
        double GUx = 0, GUy = 0, GVx = 0, GVy = 0;
        for (int a = 0; a < 3; ++a) {
          const double ua = p0 * u0[a] + p1 * u1[a], va = p0 * v0[a] + p1 * v1[a];
          GUx += ua * lx[a];
          GUy += ua * ly[a];
          GVx += va * lx[a];
          GVy += va * ly[a];
        }
        for (int tp = 0; tp < 3; ++tp) {
          const double h = ds * Hq[tp];
          double du = 0, dv = 0;
          for (int a = 0; a < 3; ++a) {
            const double la = (a == tp) ? 2.0 / 3.0 : 1.0 / 6.0;
            du += la * (u1[a] - u0[a]);
            dv += la * (v1[a] - v0[a]);
          }
          const double uz = du / h, vz = dv / h;
          const double ux = GUx - uz * Gzx, uy = GUy - uz * Gzy, vx = GVx - vz * Gzx, vy = GVy - vz * Gzy;
          const double exy = 0.5 * (uy + vx);
          const double e2 = ux * ux + vy * vy + ux * vy + exy * exy + 0.25 * (uz * uz + vz * vz);
          const double xx = e2 + delta;
          acc += (d * h * (1.0 / 12.0)) * 1.5 * hardness_at(Bn, cA, v, L, l, p0, p1, tp) * xx * inv_cbrt(xx);
        }
      }
    }
  }
  block_add(acc, out);
}

// eps_e^2 as a quadratic form Q on velocity gradients G = (u_x, u_y, u_z, v_x, v_y, v_z), and its
// polar (symmetric bilinear) form B with B(G, G) = Q(G):
//   Q(G)    = u_x^2 + v_y^2 + u_x v_y + ((u_y + v_x)^2 + u_z^2 + v_z^2) / 4
//   B(G, H) = u_x U_x + v_y V_y + (u_x V_y + v_y U_x) / 2 + ((u_y + v_x)(U_y + V_x) + u_z U_z + v_z V_z) / 4
// written as chains of FMAs (8 and 11 operations)
__device__ __forceinline__ f64x2 vfma(const f64x2 a, const f64x2 b, const f64x2 c) { return a * b + c; }
template <class T>
__device__ __forceinline__ T eps_quad(const T* A) {
  const T s = A[1] + A[3];
  const T q = vfma(A[5], A[5], vfma(A[2], A[2], s * s));
  const T p = vfma(A[0], A[0] + A[4], A[4] * A[4]);
  return vfma(T(0.25), q, p);
}
template <class T>
__device__ __forceinline__ T eps_bilinear(const T* A, const T* B) {
  const T q = vfma(A[5], B[5], vfma(A[2], B[2], (A[1] + A[3]) * (B[1] + B[3])));
  const T m = vfma(A[0], B[4], B[0] * A[4]);
  const T p = vfma(A[4], B[4], A[0] * B[0]);
  return vfma(T(0.25), q, vfma(T(0.5), m, p));
}

// 1 / x for x > 0: an FP32 reciprocal of x rounded to FP32 as the seed (conversions on the integer
// pipe), then two Newton-Raphson steps r <- r + r (1 - x r) in FP64, each of which squares the
// relative error (2^-23 -> 2^-46 -> below FP64 rounding): four FMAs on the FP64 pipe.  x outside
// the FP32 range in which the seed is accurate takes the full division.
__device__ __forceinline__ double recip_pos(const double x) {
  const float xf = f32_of(x);
  if (!(xf > 1e-30f && xf < 1e30f)) return 1.0 / x;
  double r = f64_of(1.0f / xf);
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}
__device__ __forceinline__ float recip_pos(const float x) { return 1.0f / x; }
__device__ __forceinline__ f64x2 recip_pos(const f64x2 x) { return f64x2(1.f, 0.f) / x; }

__device__ __forceinline__ double cube_root(double x) {  // x^(1/3) = x (x^(-1/3))^2
  const double r = inv_cbrt(x);
  return x * r * r;
}
__device__ __forceinline__ float cube_root(float x) { return cbrtf(x); }
__device__ __forceinline__ f64x2 cube_root(f64x2 x) {
  const f64x2 r = ds_inv_cbrt(x);
  return x * r * r;
}

// Energy change Pi_h(U + alpha D) - Pi_h(U), formed term by term as differences so that it keeps
// its relative accuracy when it is many orders smaller than Pi_h itself (near convergence):
//   driving:  alpha load . d;   basal: alpha d^T M u + alpha^2/2 d^T M d    (both FP64);
//   stress:   x = eps_e^2 + delta is quadratic in the velocity gradient G, so
//             x1 - x0 = alpha (2 B(G0, Gd)) + alpha^2 Q(Gd) exactly, and
//             x1^(2/3) - x0^(2/3) = (a - b)(a + b), a - b = (x1 - x0) / (a^2 + a b + b^2), a, b = cube roots,
//   in arithmetic T per quadrature point (FP64, or FP32 for the mixed-precision line search: the
//   change keeps ~1e-5 relative accuracy there because it is never formed as a difference of energies).
template <class T, class DT>
__global__ void __launch_bounds__(128) k_energy_change(const double2* __restrict__ xy, const double* __restrict__ bed,
                                                       const double* __restrict__ thick,
                                                       const double* __restrict__ sigma,
                                                       const int32_t* __restrict__ tri,
                                                       const double* __restrict__ basal,
                                                       const double* __restrict__ load, int ntri, int L,
                                                       int64_t ndof, double cA, const double* __restrict__ Bn,
                                                       double delta, double alpha,
                                                       const double* __restrict__ U, const DT* __restrict__ D,
                                                       double* out, int nwhole, int nseg) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ndof; i += (int64_t)gridDim.x * blockDim.x)
    acc += alpha * load[i] * (double)D[i];
  // column t, layers [l0, l1): threads below nwhole take whole columns, the rest the last columns'
  // layer segments (the column sums are additive; only the bottom segment adds the basal term)
  int t = blockIdx.x * blockDim.x + threadIdx.x, l0 = 0, l1 = L;
  if (nseg > 1 && t >= nwhole) {
    const int nrest = ntri - nwhole, j = t - nwhole;
    const int sgm = j / nrest;
    t = sgm < nseg ? nwhole + (j - sgm * nrest) : ntri;
    l0 = sgm * L / nseg;
    l1 = (sgm + 1) * L / nseg;
  }
  if (t < ntri) {
    int v[3];
    double x[3], y[3], H[3], bb[3];
    for (int a = 0; a < 3; ++a) {
      v[a] = tri[3 * t + a];
      const double2 p = xy[v[a]];
      x[a] = p.x;
      y[a] = p.y;
      H[a] = thick[v[a]];
      bb[a] = bed[v[a]];
    }
    const double d = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
    const double inv_d = 1.0 / d;
    double lx[3], ly[3];
    for (int a = 0; a < 3; ++a) {
      lx[a] = (y[(a + 1) % 3] - y[(a + 2) % 3]) * inv_d;
      ly[a] = (x[(a + 2) % 3] - x[(a + 1) % 3]) * inv_d;
    }
    const double gbx = bb[0] * lx[0] + bb[1] * lx[1] + bb[2] * lx[2];
    const double gby = bb[0] * ly[0] + bb[1] * ly[1] + bb[2] * ly[2];
    const double gHx = H[0] * lx[0] + H[1] * lx[1] + H[2] * lx[2];
    const double gHy = H[0] * ly[0] + H[1] * ly[1] + H[2] * ly[2];
    const double Hs6 = (H[0] + H[1] + H[2]) * (1.0 / 6.0);
    int64_t ub[3];
    for (int a = 0; a < 3; ++a) ub[a] = 2LL * v[a] * (L + 1);
    if (l0 == 0) {
      const double* Mb = basal + 6 * (int64_t)t;
      const double M[3][3] = {{Mb[0], Mb[1], Mb[2]}, {Mb[1], Mb[3], Mb[4]}, {Mb[2], Mb[4], Mb[5]}};
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          const double du = (double)D[ub[a]], dv = (double)D[ub[a] + 1];
          acc += M[a][b] * (alpha * (du * U[ub[b]] + dv * U[ub[b] + 1]) +
                            0.5 * alpha * alpha * (du * (double)D[ub[b]] + dv * (double)D[ub[b] + 1]));
        }
    }
    // stress term: the column walk of the assembly kernel (level gradients carried from the wedge
    // below, one reciprocal of the thickness per triangle point), per point the exact difference
    // per column in FP64, rounded once to T; below, everything per level and point runs in T
    const T ta = to_T<T>(alpha), tdelta = to_T<T>(delta), tcA = to_T<T>(cA);
    const T tgbx = to_T<T>(gbx), tgby = to_T<T>(gby), tgHx = to_T<T>(gHx), tgHy = to_T<T>(gHy);
    T tlx[3], tly[3], invHq[3], Hq[3];
    for (int a = 0; a < 3; ++a) {
      tlx[a] = to_T<T>(lx[a]);
      tly[a] = to_T<T>(ly[a]);
      const double hq = Hs6 + 0.5 * H[a];
      Hq[a] = to_T<T>(hq);
      invHq[a] = to_T<T>(1.0 / hq);
    }
    T u0[3], v0[3], a0[3], b0[3];
    for (int a = 0; a < 3; ++a) {
      u0[a] = to_T<T>(U[ub[a] + 2 * l0]);
      v0[a] = to_T<T>(U[ub[a] + 2 * l0 + 1]);
      a0[a] = dir_T<T>(D[ub[a] + 2 * l0]);
      b0[a] = dir_T<T>(D[ub[a] + 2 * l0 + 1]);
    }
    auto grad2 = [&](const T* w, T& gx, T& gy) {
      gx = w[0] * tlx[0] + w[1] * tlx[1] + w[2] * tlx[2];
      gy = w[0] * tly[0] + w[1] * tly[1] + w[2] * tly[2];
    };
    T gU0[2], gV0[2], gA0[2], gB0[2];
    grad2(u0, gU0[0], gU0[1]);
    grad2(v0, gV0[0], gV0[1]);
    grad2(a0, gA0[0], gA0[1]);
    grad2(b0, gB0[0], gB0[1]);
    double stress = 0.0;
    for (int l = l0; l < l1; ++l) {
      T u1[3], v1[3], a1[3], b1[3];
      for (int a = 0; a < 3; ++a) {
        u1[a] = to_T<T>(U[ub[a] + 2 * l + 2]);
        v1[a] = to_T<T>(U[ub[a] + 2 * l + 3]);
        a1[a] = dir_T<T>(D[ub[a] + 2 * l + 2]);
        b1[a] = dir_T<T>(D[ub[a] + 2 * l + 3]);
      }
      T gU1[2], gV1[2], gA1[2], gB1[2];
      grad2(u1, gU1[0], gU1[1]);
      grad2(v1, gV1[0], gV1[1]);
      grad2(a1, gA1[0], gA1[1]);
      grad2(b1, gB1[0], gB1[1]);
      const T s_l = to_T<T>(sigma[l]), ds = to_T<T>(sigma[l + 1] - sigma[l]);
      const T invds = recip_pos(ds);
      const T sixth = T(1.0 / 6.0);
      const T du6 = (u1[0] - u0[0] + u1[1] - u0[1] + u1[2] - u0[2]) * sixth;
      const T dv6 = (v1[0] - v0[0] + v1[1] - v0[1] + v1[2] - v0[2]) * sixth;
      const T da6 = (a1[0] - a0[0] + a1[1] - a0[1] + a1[2] - a0[2]) * sixth;
      const T db6 = (b1[0] - b0[0] + b1[1] - b0[1] + b1[2] - b0[2]) * sixth;
      T lstress = T(0);
      for (int z = 0; z < 2; ++z) {
        const T p0 = (T)(z == 0 ? BP_QP_P : BP_QP_Q), p1 = (T)(z == 0 ? BP_QP_Q : BP_QP_P);
        const T sz = s_l + T(z == 0 ? BP_QP_Q : BP_QP_P) * ds;
        const T Gzx = tgbx + sz * tgHx, Gzy = tgby + sz * tgHy;
        const T GUx = p0 * gU0[0] + p1 * gU1[0], GUy = p0 * gU0[1] + p1 * gU1[1];
        const T GVx = p0 * gV0[0] + p1 * gV1[0], GVy = p0 * gV0[1] + p1 * gV1[1];
        const T GAx = p0 * gA0[0] + p1 * gA1[0], GAy = p0 * gA0[1] + p1 * gA1[1];
        const T GBx = p0 * gB0[0] + p1 * gB1[0], GBy = p0 * gB0[1] + p1 * gB1[1];
        for (int tp = 0; tp < 3; ++tp) {
          const T invh = invds * invHq[tp];
          const T uz = (du6 + T(0.5) * (u1[tp] - u0[tp])) * invh;
          const T vz = (dv6 + T(0.5) * (v1[tp] - v0[tp])) * invh;
          const T az = (da6 + T(0.5) * (a1[tp] - a0[tp])) * invh;
          const T bz = (db6 + T(0.5) * (b1[tp] - b0[tp])) * invh;
          const T G0[6] = {GUx - uz * Gzx, GUy - uz * Gzy, uz, GVx - vz * Gzx, GVy - vz * Gzy, vz};
          const T Gd[6] = {GAx - az * Gzx, GAy - az * Gzy, az, GBx - bz * Gzx, GBy - bz * Gzy, bz};
          const T x0 = eps_quad(G0) + tdelta;
          const T dx = ta * vfma(ta, eps_quad(Gd), T(2) * eps_bilinear(G0, Gd));
          const T x1 = x0 + dx;
          const T ca = cube_root(x1), cb = cube_root(x0);
          const T sab = ca + cb;  // a^2 + a b + b^2 = a (a + b) + b^2 > 0
          const T diff23 = dx * recip_pos(vfma(ca, sab, cb * cb)) * sab;
          lstress += Hq[tp] * hardness_at_t<T>(Bn, tcA, v, L, l, p0, p1, tp) * diff23;
        }
      }
      stress += (d * (sigma[l + 1] - sigma[l]) * (1.0 / 12.0)) * from_T(lstress);
      for (int a = 0; a < 3; ++a) {
        u0[a] = u1[a];
        v0[a] = v1[a];
        a0[a] = a1[a];
        b0[a] = b1[a];
      }
      for (int c = 0; c < 2; ++c) {
        gU0[c] = gU1[c];
        gV0[c] = gV1[c];
        gA0[c] = gA1[c];
        gB0[c] = gB1[c];
      }
    }
    acc += 1.5 * stress;
  }
  block_add(acc, out);
}

// ------------------------------------------------------------------ shallow-ice guess
__global__ void k_sia_accum(const double2* __restrict__ xy, const double* __restrict__ bed,
                            const double* __restrict__ thick, const int32_t* __restrict__ tri, int ntri,
                            double* __restrict__ acc /* [3][nv] */, int nv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntri) return;
  int v[3];
  double x[3], y[3], s[3];
  for (int a = 0; a < 3; ++a) {
    v[a] = tri[3 * t + a];
    x[a] = xy[v[a]].x;
    y[a] = xy[v[a]].y;
    s[a] = bed[v[a]] + thick[v[a]];
  }
  const double d = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
  double sx = 0, sy = 0;
  for (int a = 0; a < 3; ++a) {
    sx += s[a] * (y[(a + 1) % 3] - y[(a + 2) % 3]) / d;
    sy += s[a] * (x[(a + 2) % 3] - x[(a + 1) % 3]) / d;
  }
  const double area = 0.5 * d;
  for (int a = 0; a < 3; ++a) {
    atomicAdd(acc + v[a], area * sx);
    atomicAdd(acc + nv + v[a], area * sy);
    atomicAdd(acc + 2 * nv + v[a], area);
  }
}

__global__ void k_sia_fill(const double* __restrict__ acc, const double* __restrict__ bed,
                           const double* __restrict__ thick, const double* __restrict__ beta,
                           const double* __restrict__ sigma, int nv, int L, double A, double rho_g,
                           double* __restrict__ U) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  const double w = acc[2 * nv + a];
  const double sx = acc[a] / w, sy = acc[nv + a] / w;
  const double g2 = sx * sx + sy * sy;
  const double H = thick[a];
  const double H4 = (H * H) * (H * H);
  const double slide = beta[a] > 0.0 ? rho_g * H / beta[a] : 0.0;
  const double c = 0.5 * A * rho_g * rho_g * rho_g * g2;  // 2A/(n+1) (rho g)^n |grad s|^(n-1), n = 3
  for (int l = 0; l <= L; ++l) {
    const double dep = (1.0 - sigma[l]) * H;
    const double d4 = (dep * dep) * (dep * dep);
    const double f = c * (H4 - d4) + slide;
    U[2 * ((int64_t)a * (L + 1) + l)] = -f * sx;
    U[2 * ((int64_t)a * (L + 1) + l) + 1] = -f * sy;
  }
}

// ------------------------------------------------------------------ host helpers
int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, GRID_CAP));
}

int ensure_ws(bp_mesh* m, cudaStream_t s) {
  if (m->ws) return BP_OK;
  if (m->nl > MAXL) return BP_EUNSUP;
  bp_solver_ws tmp;
  bp_solver_ws* w = &tmp;
  int rc;
  const int64_t n = m->ndof, nv = m->nv, L = m->nl;
  // on failure the arrays already allocated stay recorded in the mesh and are freed with it
#define WS_ALLOC(ptr, cnt) \
  if ((rc = bp_alloc(m, &(ptr), (cnt))) != BP_OK) return rc
  WS_ALLOC(w->dslot, nv);
  WS_ALLOC(w->Lm, 4 * L * nv);
  WS_ALLOC(w->Ginv, 4 * (L + 1) * nv);
  WS_ALLOC(w->Fu, 4 * L * nv);
  WS_ALLOC(w->x, n);
  WS_ALLOC(w->r, n);
  WS_ALLOC(w->z, n);
  WS_ALLOC(w->p, n);
  WS_ALLOC(w->q, n);
  WS_ALLOC(w->R, n);
  WS_ALLOC(w->Ut, n);
  WS_ALLOC(w->scal, 3 * (SCAL_CAP + 2 + CG_BATCH));
  WS_ALLOC(w->stop, 1);
  WS_ALLOC(w->kbase, 1);
  WS_ALLOC(w->cgpar, 2);
  WS_ALLOC(w->red, 8);
  WS_ALLOC(w->sia, 3 * nv);
#undef WS_ALLOC
  w->scal_cap = SCAL_CAP;
  w->host_cap = 3 * (SCAL_CAP + 2) + 8;
  if (cudaMallocHost(&w->host, w->host_cap * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return BP_ENOMEM;
  }
  if (cudaMallocHost(&w->hpar, 2 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(w->host);
    return BP_ENOMEM;
  }
  k_find_dslot<<<(m->nv + 127) / 128, 128, 0, s>>>(m->nbr_ptr, m->nbr_idx, m->nv, w->dslot);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFreeHost(w->host);
    cudaFreeHost(w->hpar);
    bp_set_last_cuda_error(e, "k_find_dslot", __LINE__);
    return BP_ECUDA;
  }
  m->ws = new bp_solver_ws(tmp);
  return BP_OK;
}

int ensure_jac(bp_mesh* m) {
  if (m->ws->J) return BP_OK;
  return bp_alloc(m, &m->ws->J, m->nnz);
}

// The factor arrays are allocated as double; FP32 factors (set up from an FP32 Jacobian) use the
// first half of each.
template <class F>
Prec<F> prec_of(const bp_mesh* m) {
  return Prec<F>{reinterpret_cast<const F*>(m->ws->Lm), reinterpret_cast<const F*>(m->ws->Ginv),
                 reinterpret_cast<const F*>(m->ws->Fu), m->nv, m->nl};
}

// synchronous dot product a . b (FP64 result on the host)
template <class A, class B>
int dot_host(bp_mesh* m, const A* a, const B* b, int64_t n, cudaStream_t s, double* out) {
  bp_solver_ws* w = m->ws;
  BP_CUDA_TRY(cudaMemsetAsync(w->red, 0, sizeof(double), s));
  k_dot<<<grid_for(n, NT), NT, 0, s>>>(a, b, n, w->red);
  BP_CUDA_TRY(cudaGetLastError());
  BP_CUDA_TRY(cudaMemcpyAsync(w->host, w->red, sizeof(double), cudaMemcpyDeviceToHost, s));
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  *out = w->host[0];
  return BP_OK;
}

int energy_host(bp_mesh* m, const double* U, cudaStream_t s, double* out) {
  bp_solver_ws* w = m->ws;
  BP_CUDA_TRY(cudaMemsetAsync(w->red + 1, 0, sizeof(double), s));
  const int grid = (int)std::max<int64_t>((m->ntri + 127) / 128, std::min<int64_t>((m->ndof + 127) / 128, 148 * 16));
  k_energy<<<grid, 128, 0, s>>>(m->xy, m->bed, m->thick, m->sigma, m->tri, m->basal, m->load, m->ntri, m->nl,
                                m->ndof, m->cA, m->Bnode, m->p.delta, U, w->red + 1);
  BP_CUDA_TRY(cudaGetLastError());
  BP_CUDA_TRY(cudaMemcpyAsync(w->host, w->red + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  *out = w->host[0];
  return BP_OK;
}

// synchronous energy change Pi(U + alpha D) - Pi(U) (T: arithmetic of the per-point stress term)
template <class T, class DT>
int energy_change_host(bp_mesh* m, const double* U, const DT* D, double alpha, cudaStream_t s, double* out) {
  bp_solver_ws* w = m->ws;
  BP_CUDA_TRY(cudaMemsetAsync(w->red + 2, 0, sizeof(double), s));
  // the columns of the last partial wave of resident threads are taken in layer segments (as the
  // assembly's atomic launches do), so that the SMs finish together
  static int resident = -1;
  if (resident < 0) {
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_energy_change<T, DT>, 128, 0) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 0;
    }
    resident = nsm * per_sm * 128;
  }
  int nwhole = m->ntri, nseg = 0;
  const int segs = std::min(4, m->nl / 2);
  if (segs >= 2 && resident > 0 && m->ntri > resident && m->ntri % resident) {
    nwhole = m->ntri - m->ntri % resident;
    nseg = segs;
  }
  const int64_t threads = nwhole + (int64_t)(m->ntri - nwhole) * nseg;
  const int grid = (int)std::max<int64_t>((threads + 127) / 128, std::min<int64_t>((m->ndof + 127) / 128, 148 * 16));
  k_energy_change<T, DT><<<grid, 128, 0, s>>>(m->xy, m->bed, m->thick, m->sigma, m->tri, m->basal, m->load, m->ntri,
                                              m->nl, m->ndof, m->cA, m->Bnode, m->p.delta, alpha, U, D,
                                              w->red + 2, nwhole, nseg);
  BP_CUDA_TRY(cudaGetLastError());
  BP_CUDA_TRY(cudaMemcpyAsync(w->host, w->red + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  *out = w->host[0];
  return BP_OK;
}

// FP64 Jacobian: FP64 factors; FP32 Jacobian (mixed-precision path): FP32 factors, applied in FP32.
template <class M>
int colprec_setup_t(bp_mesh* m, const M* J, cudaStream_t s) {
  bp_solver_ws* w = m->ws;
  using F = M;
  k_colprec_setup<M, F><<<(m->nv + 127) / 128, 128, 0, s>>>(J, m->vstart, m->vdeg, w->dslot, m->nv, m->nl,
                                                            reinterpret_cast<F*>(w->Lm), reinterpret_cast<F*>(w->Ginv),
                                                            reinterpret_cast<F*>(w->Fu));
  BP_CUDA_TRY(cudaGetLastError());
  w->has_prec = true;
  w->prec_f32 = sizeof(F) == sizeof(float);
  return BP_OK;
}

// One CG batch: CG_BATCH iterations (SpMV + dot, update + preconditioner, direction), then the
// batch counter advances.  The iteration index, the tolerance and the limit are read from device
// memory, so one captured graph serves every solve on this mesh and precision.
// Launch with the programmatic-stream-serialisation attribute (captured as a programmatic edge).
// Used only while capturing the loop body; a refused launch is picked up after the capture.
template <class... Args, class... Act>
void launch_pdl(void (*kern)(Args...), int grid, int block, size_t smem, cudaStream_t s, Act... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

// y = J x (with DOT: x . y added to dot[3 (kbase + j)], or to *dot without kbase), optionally as a
// programmatic dependent launch.
template <class M, class V, bool DOT>
void spmv_launch(bp_mesh* m, const M* J, const V* x, V* y, double* dot, const int* stop, const int* kbase, int j,
                 cudaStream_t s, bool pdl = false) {
  const int npairs = (int)(m->ndof / 2);
  const int grid = grid_for((int64_t)npairs * TPR, NT);
  if (pdl)
    launch_pdl(k_spmv_pairs<M, V, DOT>, grid, NT, 0, s, (const int64_t*)m->rowptr, (const int32_t*)m->nbr_ptr,
               (const int32_t*)m->nbr_idx, m->nl, J, npairs, x, y, dot, stop, kbase, j);
  else
    k_spmv_pairs<M, V, DOT><<<grid, NT, 0, s>>>(m->rowptr, m->nbr_ptr, m->nbr_idx, m->nl, J, npairs, x, y, dot, stop,
                                                kbase, j);
}

// FP32 CG with 5 or 10 layers: the register-resident start and update; false where they do not apply.
template <class V>
bool init_cols(const Prec<V>& P, const double* R, V* x, V* r, V* z, V* p, double* scal, int* stop, int L,
               cudaStream_t s) {
  if constexpr (std::is_same<V, float>::value) {
    const int grid = (P.nv + UPD_NT - 1) / UPD_NT;
    if (L == 10) {
      k_cg_init_cols<11><<<grid, UPD_NT, 0, s>>>(P, R, x, r, z, p, scal, stop);
      return true;
    }
    if (L == 5) {
      k_cg_init_cols<6><<<grid, UPD_NT, 0, s>>>(P, R, x, r, z, p, scal, stop);
      return true;
    }
  }
  return false;
}

template <class V>
bool update_cols(const Prec<V>& P, bp_solver_ws* w, int j, V* x, V* r, V* z, const V* p, const V* q, int L,
                 cudaStream_t s, bool pdl = false) {
  if constexpr (std::is_same<V, float>::value) {
    const int grid = (P.nv + UPD_NT - 1) / UPD_NT;
    if (L == 10 || L == 5) {
      auto kern = L == 10 ? k_cg_update_cols<11> : k_cg_update_cols<6>;
      if (pdl)
        launch_pdl(kern, grid, UPD_NT, 0, s, P, (const int*)w->kbase, j, x, r, z, p, q, w->scal, w->stop);
      else
        kern<<<grid, UPD_NT, 0, s>>>(P, w->kbase, j, x, r, z, p, q, w->scal, w->stop);
      return true;
    }
  }
  return false;
}

template <class M, class V>
void launch_cg_batch(bp_mesh* m, const M* J, cudaStream_t s) {
  bp_solver_ws* w = m->ws;
  const Prec<V> P = prec_of<V>(m);
  const int64_t n = m->ndof;
  V* x = reinterpret_cast<V*>(w->x);
  V* r = reinterpret_cast<V*>(w->r);
  V* z = reinterpret_cast<V*>(w->z);
  V* p = reinterpret_cast<V*>(w->p);
  V* q = reinterpret_cast<V*>(w->q);
  const int ncolv = 2 * (m->nl + 1);
  const int C = std::max(1, std::min(32, (int)((48 << 10) / (2 * ncolv * (int)sizeof(V)))));
  const size_t smem = 2 * (size_t)C * ncolv * sizeof(V);
  const int gupd = (m->nv + C - 1) / C;
  for (int j = 0; j < CG_BATCH; ++j) {
    spmv_launch<M, V, true>(m, J, p, q, w->scal, w->stop, w->kbase, j, s);
    if (!update_cols<V>(P, w, j, x, r, z, p, q, m->nl, s))
      k_cg_update_staged<V, V><<<gupd, UPD_NT, smem, s>>>(P, w->kbase, j, C, x, r, z, p, q, w->scal, w->stop);
    k_cg_direction<V><<<grid_for(n / 2, NT), NT, 0, s>>>(w->kbase, j, w->cgpar, n / 2, z, p, w->scal, w->stop,
                                                         cudaGraphConditionalHandle{}, 0);
  }
  k_cg_advance<<<1, 1, 0, s>>>(w->kbase, CG_BATCH);
}

// LOOP_BODY CG iterations as the body of the device-driven loop: per iteration SpMV + dot, update +
// preconditioner, direction (which sets the loop condition); then the iteration counter advances.
// Launches after the stopping iteration exit at once.
template <class M, class V>
void launch_cg_iteration(bp_mesh* m, const M* J, cudaStream_t s, cudaGraphConditionalHandle loop) {
  bp_solver_ws* w = m->ws;
  const Prec<V> P = prec_of<V>(m);
  const int64_t n = m->ndof;
  V* x = reinterpret_cast<V*>(w->x);
  V* r = reinterpret_cast<V*>(w->r);
  V* z = reinterpret_cast<V*>(w->z);
  V* p = reinterpret_cast<V*>(w->p);
  V* q = reinterpret_cast<V*>(w->q);
  const int ncolv = 2 * (m->nl + 1);
  const int C = std::max(1, std::min(32, (int)((48 << 10) / (2 * ncolv * (int)sizeof(V)))));
  const size_t smem = 2 * (size_t)C * ncolv * sizeof(V);
  const int gupd = (m->nv + C - 1) / C;
  for (int j = 0; j < LOOP_BODY; ++j) {
    spmv_launch<M, V, true>(m, J, p, q, w->scal, w->stop, w->kbase, j, s, true);
    if (!update_cols<V>(P, w, j, x, r, z, p, q, m->nl, s, true))
      launch_pdl(k_cg_update_staged<V, V>, gupd, UPD_NT, smem, s, P, (const int*)w->kbase, j, C, x, r, z, (const V*)p,
                 (const V*)q, w->scal, w->stop);
    launch_pdl(k_cg_direction<V>, grid_for(n / 2, NT), NT, 0, s, (const int*)w->kbase, j, (const double*)w->cgpar,
               (int64_t)(n / 2), (const V*)z, p, (const double*)w->scal, w->stop, loop, 1);
  }
  launch_pdl(k_cg_advance, 1, 1, 0, s, w->kbase, LOOP_BODY);
}

// The whole CG iteration loop as one graph: a conditional WHILE node whose body is one iteration
// (captured once per mesh and precision).  The device decides when to stop, so a solve needs no host
// check between iterations and launches no iteration past the last.  Returns exec = NULL (and the
// caller replays batches instead) where conditional nodes are not available.
template <class M, class V>
int cg_loop_graph(bp_mesh* m, const M* J, cudaGraphExec_t* out) {
  bp_solver_ws* w = m->ws;
  const int slot = sizeof(V) == sizeof(float) ? 1 : 0;
  *out = nullptr;
  if (w->cg_loop_failed[slot]) return BP_OK;
  if (!w->cg_loop[slot]) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraphConditionalHandle h{};
    cudaGraphNodeParams cp{};
    cudaGraphNode_t node = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      launch_cg_iteration<M, V>(m, J, cs, h);
      const cudaError_t le = cudaGetLastError();  // a launch the capture refused
      cudaGraph_t body = nullptr;
      e = cudaStreamEndCapture(cs, &body);
      if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();  // not sticky: fall back to the batch graphs
      w->cg_loop_failed[slot] = true;
      return BP_OK;
    }
    w->cg_loop[slot] = exec;
  }
  *out = (cudaGraphExec_t)w->cg_loop[slot];
  return BP_OK;
}

template <class M, class V>
int cg_batch_graph(bp_mesh* m, const M* J, cudaGraphExec_t* out) {
  bp_solver_ws* w = m->ws;
  const int slot = sizeof(V) == sizeof(float) ? 1 : 0;
  if (!w->cg_exec[slot]) {
    cudaStream_t cs;
    BP_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) launch_cg_batch<M, V>(m, J, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    BP_CUDA_TRY(e);
    w->cg_exec[slot] = exec;
  }
  *out = (cudaGraphExec_t)w->cg_exec[slot];
  return BP_OK;
}

// Preconditioned CG on J delta = -R to ||r|| <= eta ||R||.  delta is left in ws->x (type V).
// The iterations run as replays of the captured batch graph; the host reads the device stop flag
// every check_every iterations (rounded up to whole batches).
// stop flag 5: a kernel's bounded wait for its bulk copies gave up (reported as a CUDA failure)
int bulk_wait_failed(int line) {
  bp_set_last_cuda_error(cudaErrorTimeout, "bulk copy wait in the CG column kernels", line);
  return BP_ECUDA;
}

template <class M, class V>
int cg_solve(bp_mesh* m, const M* J, double eta, int maxit, int check_every, bool device_loop, cudaStream_t s,
             int* iters, int* status) {
  bp_solver_ws* w = m->ws;
  const Prec<V> P = prec_of<V>(m);  // factors set up from the same-precision Jacobian
  maxit = std::min(maxit, w->scal_cap);
  V* x = reinterpret_cast<V*>(w->x);
  V* r = reinterpret_cast<V*>(w->r);
  V* z = reinterpret_cast<V*>(w->z);
  V* p = reinterpret_cast<V*>(w->p);
  cudaGraphExec_t loop = nullptr, exec = nullptr;
  int rc = device_loop ? cg_loop_graph<M, V>(m, J, &loop) : BP_OK;
  if (rc) return rc;
  if (!loop && (rc = cg_batch_graph<M, V>(m, J, &exec))) return rc;
  BP_CUDA_TRY(cudaMemsetAsync(w->scal, 0, 3 * (size_t)(maxit + 2 + CG_BATCH) * sizeof(double), s));
  BP_CUDA_TRY(cudaMemsetAsync(w->stop, 0, sizeof(int), s));
  BP_CUDA_TRY(cudaMemsetAsync(w->kbase, 0, sizeof(int), s));
  // the staging buffer is rewritten only by the next solve, after this one has synchronised
  w->hpar[0] = eta * eta;
  w->hpar[1] = (double)maxit;
  BP_CUDA_TRY(cudaMemcpyAsync(w->cgpar, w->hpar, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
  if (!init_cols<V>(P, w->R, x, r, z, p, w->scal, w->stop, m->nl, s)) {
    const int ncolv = 2 * (m->nl + 1);
    const int C = std::max(1, std::min(32, (int)((48 << 10) / (2 * ncolv * (int)sizeof(V)))));
    const size_t smem = 2 * (size_t)C * ncolv * sizeof(V);
    k_cg_init_staged<V, V><<<(m->nv + C - 1) / C, UPD_NT, smem, s>>>(P, C, w->R, x, r, z, p, w->scal);
  }
  BP_CUDA_TRY(cudaGetLastError());
  const int batches_per_check = std::max(1, (check_every + CG_BATCH - 1) / CG_BATCH);
  int k = 0, done = 0;
  *status = 0;
  if (loop) {  // one launch runs the whole solve; then read the iteration count and the history
    BP_CUDA_TRY(cudaGraphLaunch(loop, s));
    int* hk = reinterpret_cast<int*>(w->host + w->host_cap - 2);
    BP_CUDA_TRY(cudaMemcpyAsync(hk, w->kbase, sizeof(int), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaMemcpyAsync(w->host + w->host_cap - 1, w->stop, sizeof(int), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    k = std::min(std::max(*hk, 0), maxit);
    BP_CUDA_TRY(cudaMemcpyAsync(w->host, w->scal, 3 * (size_t)(k + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    int stopflag;
    std::memcpy(&stopflag, w->host + w->host_cap - 1, sizeof(int));
    if (stopflag == 2) *status = 2;
    if (stopflag == 5) return bulk_wait_failed(__LINE__);
    done = 1;
  }
  while (!done) {
    for (int b = 0; b < batches_per_check && k < maxit; ++b, k += CG_BATCH) BP_CUDA_TRY(cudaGraphLaunch(exec, s));
    const int kk = std::min(k, maxit);
    BP_CUDA_TRY(cudaMemcpyAsync(w->host, w->scal, 3 * (size_t)(kk + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaMemcpyAsync(w->host + w->host_cap - 1, w->stop, sizeof(int), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    int stopflag;
    std::memcpy(&stopflag, w->host + w->host_cap - 1, sizeof(int));
    if (stopflag || k >= maxit) done = 1;
    if (stopflag == 2) *status = 2;
    if (stopflag == 5) return bulk_wait_failed(__LINE__);
    if (done) k = kk;
  }
  // iterations actually taken: first j with r_j.r_j <= eta^2 r_0.r_0
  const double tol2 = eta * eta;
  const double rr0 = w->host[2];
  int taken = k;
  for (int j = 1; j <= k; ++j) {
    const double rr = w->host[3 * j + 2];
    if (!std::isfinite(rr)) {  // breakdown: Newton reports BP_ENAN at once
      taken = j;
      *status = 3;
      break;
    }
    if (rr <= tol2 * rr0) {
      taken = j;
      break;
    }
    if (w->host[3 * j + 2] == 0.0 && w->host[3 * j + 1] == 0.0) {  // never reached (breakdown stop)
      taken = j - 1;
      break;
    }
  }
  *iters = taken;
  if (!std::isfinite(rr0)) *status = 3;
  return BP_OK;
}

// ------------------------------------------------------------------ GMRES(m)
// Paper Sec. 3.1: the Newton step's linear system is solved by preconditioned GMRES.  The Jacobian
// here is symmetric positive definite, so CG is the default; GMRES(m) with the same column
// preconditioner is the cross-check.  Right preconditioning (J M^-1 u = -R, delta = M^-1 u), so
// the least-squares residual |g_{k+1}| is the true residual norm ||-R - J delta|| that CG's test
// also uses; Arnoldi by classical Gram-Schmidt applied twice (each pass one multi-dot and one
// multi-axpy over the basis), the small Hessenberg problem (Givens rotations) on the host.

// h[i] += basis_i . w for i = 0..k (blockIdx.y = i; one FP64 atomic per block)
template <class V>
__global__ void __launch_bounds__(NT) k_gm_multidot(const V* __restrict__ basis, int64_t n,
                                                   const V* __restrict__ w, double* h) {
  const V* v = basis + (int64_t)blockIdx.y * n;
  V sum = V(0);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    sum += v[e] * w[e];
  block_add(sum, h + blockIdx.y);
}

// w -= sum_{i <= k} c_i basis_i  (c in device memory, k + 1 values); or, with out != nullptr,
// out = sum_i c_i basis_i (w unused)
template <class V>
__global__ void __launch_bounds__(NT) k_gm_combine(const V* __restrict__ basis, int64_t n, int k1,
                                                  const double* __restrict__ c, V* __restrict__ w, V* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    V acc = V(0);
    for (int i = 0; i < k1; ++i) acc += (V)c[i] * basis[(int64_t)i * n + e];
    if (out)
      out[e] = acc;
    else
      w[e] -= acc;
  }
}

// y = a x (a from device memory: 1 / norm), or y = -R (x == nullptr)
template <class V>
__global__ void __launch_bounds__(NT) k_gm_scale(const V* __restrict__ x, const double* __restrict__ a,
                                                const double* __restrict__ R, int64_t n, V* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = x ? (V)(*a) * x[e] : (V)(-R[e]);
}

// r = -R - Jx (Jx given)
template <class V>
__global__ void __launch_bounds__(NT) k_gm_residual(const double* __restrict__ R, const V* __restrict__ Jx,
                                                   int64_t n, V* __restrict__ r) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    r[e] = (V)(-R[e]) - Jx[e];
}

template <class V>
__global__ void __launch_bounds__(NT) k_gm_add(const V* __restrict__ d, int64_t n, V* __restrict__ x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] += d[e];
}

int gmres_alloc(bp_mesh* m, int restart) {
  bp_solver_ws* w = m->ws;
  if (w->gm_basis && w->gm_cap >= restart) return BP_OK;
  int rc;
  // basis vectors (restart + 1) x ndof (double storage; FP32 vectors use the first half)
  if ((rc = bp_alloc(m, &w->gm_basis, (size_t)(restart + 1) * m->ndof))) return rc;
  if (!w->gm_h && (rc = bp_alloc(m, &w->gm_h, 2 * (size_t)(GMRES_MAX_RESTART + 2)))) return rc;
  w->gm_cap = restart;
  return BP_OK;
}

// GMRES(restart) on J delta = -R (w->R) to ||-R - J delta|| <= eta ||R||; delta in ws->x (type V).
template <class M, class V>
int gmres_solve(bp_mesh* m, const M* J, double eta, int maxit, int restart, cudaStream_t s, int* iters,
                int* status) {
  bp_solver_ws* w = m->ws;
  int rc = gmres_alloc(m, restart);
  if (rc) return rc;
  const Prec<V> P = prec_of<V>(m);
  const int64_t n = m->ndof;
  V* basis = reinterpret_cast<V*>(w->gm_basis);
  V* x = reinterpret_cast<V*>(w->x);
  V* wv = reinterpret_cast<V*>(w->r);   // Arnoldi vector
  V* z = reinterpret_cast<V*>(w->z);    // M^-1 v, and the update
  V* u = reinterpret_cast<V*>(w->p);
  double* hd = w->gm_h;                 // device: h column (first half), combination coefficients (second)
  double* hh = w->host;                 // pinned host mirror
  const int gvec = grid_for(n, NT), gcol = (m->nv + 127) / 128;
  *status = 0;
  BP_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(V), s));
  double bnorm;
  if ((rc = dot_host(m, w->R, w->R, n, s, &bnorm))) return rc;
  bnorm = std::sqrt(bnorm);
  if (!std::isfinite(bnorm)) {
    *status = 3;
    *iters = 0;
    return BP_OK;
  }
  const double target = eta * bnorm;
  std::vector<double> H((size_t)(restart + 1) * restart), cs(restart), sn(restart), g(restart + 1);
  auto Hat = [&](int i, int j) -> double& { return H[(size_t)j * (restart + 1) + i]; };
  int total = 0;
  double res = bnorm;
  // the residual of the current iterate: r = -R - J x (x = 0 at the first cycle)
  k_gm_scale<V><<<gvec, NT, 0, s>>>(nullptr, nullptr, w->R, n, wv);
  BP_CUDA_TRY(cudaGetLastError());
  while (total < maxit && res > target) {
    // v_0 = r / ||r||
    if (total > 0) {
      spmv_launch<M, V, false>(m, J, x, z, nullptr, nullptr, nullptr, 0, s);
      k_gm_residual<V><<<gvec, NT, 0, s>>>(w->R, z, n, wv);
    }
    double beta;
    if ((rc = dot_host(m, wv, wv, n, s, &beta))) return rc;
    beta = std::sqrt(beta);
    if (!std::isfinite(beta)) {
      *status = 3;
      break;
    }
    hh[0] = 1.0 / beta;
    BP_CUDA_TRY(cudaMemcpyAsync(hd, hh, sizeof(double), cudaMemcpyHostToDevice, s));
    k_gm_scale<V><<<gvec, NT, 0, s>>>(wv, hd, nullptr, n, basis);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (; k < restart && total < maxit; ++k, ++total) {
      // w = J M^-1 v_k
      k_colprec_apply<V, V><<<gcol, 128, 0, s>>>(P, basis + (int64_t)k * n, z);
      spmv_launch<M, V, false>(m, J, z, wv, nullptr, nullptr, nullptr, 0, s);
      // classical Gram-Schmidt, twice
      for (int i = 0; i <= k; ++i) Hat(i, k) = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        BP_CUDA_TRY(cudaMemsetAsync(hd, 0, (k + 1) * sizeof(double), s));
        k_gm_multidot<V><<<dim3(std::min(gvec, 64), k + 1), NT, 0, s>>>(basis, n, wv, hd);
        k_gm_combine<V><<<gvec, NT, 0, s>>>(basis, n, k + 1, hd, wv, nullptr);
        BP_CUDA_TRY(cudaMemcpyAsync(hh, hd, (k + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
        BP_CUDA_TRY(cudaStreamSynchronize(s));
        for (int i = 0; i <= k; ++i) Hat(i, k) += hh[i];
      }
      double hn;
      if ((rc = dot_host(m, wv, wv, n, s, &hn))) return rc;
      hn = std::sqrt(hn);
      Hat(k + 1, k) = hn;
      if (!std::isfinite(hn)) {
        *status = 3;
        break;
      }
      // Givens rotations of the new column, then a new rotation zeroing H(k+1, k)
      for (int i = 0; i < k; ++i) {
        const double a = Hat(i, k), b = Hat(i + 1, k);
        Hat(i, k) = cs[i] * a + sn[i] * b;
        Hat(i + 1, k) = -sn[i] * a + cs[i] * b;
      }
      const double a = Hat(k, k), b = Hat(k + 1, k), rr = std::hypot(a, b);
      cs[k] = rr > 0 ? a / rr : 1.0;
      sn[k] = rr > 0 ? b / rr : 0.0;
      Hat(k, k) = rr;
      Hat(k + 1, k) = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      res = std::fabs(g[k + 1]);
      if (res <= target || hn == 0.0) {
        ++k;
        ++total;
        break;
      }
      // v_{k+1} = w / ||w||
      hh[0] = 1.0 / hn;
      BP_CUDA_TRY(cudaMemcpyAsync(hd, hh, sizeof(double), cudaMemcpyHostToDevice, s));
      k_gm_scale<V><<<gvec, NT, 0, s>>>(wv, hd, nullptr, n, basis + (int64_t)(k + 1) * n);
    }
    if (*status == 3) break;
    // y = H^-1 g (upper triangular k x k);  x += M^-1 V y
    std::vector<double> y(k);
    for (int i = k - 1; i >= 0; --i) {
      double t = g[i];
      for (int j = i + 1; j < k; ++j) t -= Hat(i, j) * y[j];
      y[i] = t / Hat(i, i);
    }
    for (int i = 0; i < k; ++i) hh[i] = y[i];
    BP_CUDA_TRY(cudaMemcpyAsync(hd + GMRES_MAX_RESTART + 2, hh, k * sizeof(double), cudaMemcpyHostToDevice, s));
    k_gm_combine<V><<<gvec, NT, 0, s>>>(basis, n, k, hd + GMRES_MAX_RESTART + 2, nullptr, u);
    k_colprec_apply<V, V><<<gcol, 128, 0, s>>>(P, u, z);
    k_gm_add<V><<<gvec, NT, 0, s>>>(z, n, x);
    BP_CUDA_TRY(cudaGetLastError());
    BP_CUDA_TRY(cudaStreamSynchronize(s));  // the host mirror is rewritten by the next cycle
  }
  *iters = total;
  return BP_OK;
}

// ------------------------------------------------------------------ MDSC two-level preconditioner
// Paper Sec. 4.4: the multigrid preconditioner coarsens the extruded mesh vertically first, with a
// prolongation built from per-vertical-line solves, and solves the resulting plane problem by a 2D
// method.  Here, one symmetric two-level cycle:
//   P: semicoarsening to the top level; in column a, P_a(L) = I and, below, the harmonic extension
//      of the top value down the column, from the block-Thomas factors of the column part T of J:
//      P_a(L-1) = -G_{L-1}^-1 F_{L-1},  P_a(l) = -G_l^-1 F_l P_a(l+1);
//   A_c = P^T J P on the base vertices (2 x 2 blocks over the closed neighbourhoods);
//   B_c: MDSC_STEPS steps of Chebyshev acceleration of block-Jacobi on A_c over
//        [lam / MDSC_RATIO, lam], lam the Gershgorin bound of D^-1 A_c;
//   S = omega T^-1 (the column solve, damped);
//   z1 = S r;  z2 = z1 + P B_c P^T (r - J z1);  z = z2 + S (r - J z2).
// Symmetric (S and B_c are), positive definite for omega < 2 / lambda_max(T^-1 J).
constexpr double MDSC_OMEGA = 0.7;
constexpr int MDSC_STEPS = 8;
constexpr double MDSC_RATIO = 30.0;

template <class F>
__device__ __forceinline__ void load2x2(const F* base, int64_t stride, F* out) {
#pragma unroll
  for (int e = 0; e < 4; ++e) out[e] = base[e * stride];
}

// Prolongation blocks of levels L-1 .. 0, one thread per column.
template <class F>
__global__ void __launch_bounds__(128) k_mdsc_prolong(const Prec<F> Pr, F* __restrict__ P) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= Pr.nv) return;
  const int64_t nv = Pr.nv;
  F cur[4] = {F(1), F(0), F(0), F(1)};  // P(L) = I
  for (int l = Pr.L - 1; l >= 0; --l) {
    F G[4], Fl[4], t[4];
    load2x2(Pr.Ginv + (int64_t)l * 4 * nv + a, nv, G);
    load2x2(Pr.Fu + (int64_t)l * 4 * nv + a, nv, Fl);
    // t = F_l P(l+1), P(l) = -G_l^-1 t
    t[0] = Fl[0] * cur[0] + Fl[1] * cur[2];
    t[1] = Fl[0] * cur[1] + Fl[1] * cur[3];
    t[2] = Fl[2] * cur[0] + Fl[3] * cur[2];
    t[3] = Fl[2] * cur[1] + Fl[3] * cur[3];
    cur[0] = -(G[0] * t[0] + G[1] * t[2]);
    cur[1] = -(G[0] * t[1] + G[1] * t[3]);
    cur[2] = -(G[2] * t[0] + G[3] * t[2]);
    cur[3] = -(G[2] * t[1] + G[3] * t[3]);
#pragma unroll
    for (int e = 0; e < 4; ++e) P[((int64_t)l * 4 + e) * nv + a] = cur[e];
  }
}

// Plane operator A_c = P^T J P (one thread per base vertex: its row of 2 x 2 blocks), the inverses
// of its diagonal blocks, and the Gershgorin bound of D^-1 A_c (atomic maximum over the rows).
template <class M, class F>
__global__ void __launch_bounds__(128) k_mdsc_plane(const M* __restrict__ J, const int64_t* __restrict__ vstart,
                                                    const int32_t* __restrict__ vdeg,
                                                    const int32_t* __restrict__ dslot,
                                                    const int32_t* __restrict__ nbr_ptr,
                                                    const int32_t* __restrict__ nbr_idx, const F* __restrict__ P,
                                                    int nv, int L, F* __restrict__ Ac, F* __restrict__ Dinv,
                                                    double* lam) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  const int64_t vs = vstart[a];
  const int dg = vdeg[a], p0 = nbr_ptr[a];
  auto pblk = [&](int l, int v, F* out) {
    if (l == L) {
      out[0] = F(1), out[1] = F(0), out[2] = F(0), out[3] = F(1);
    } else {
      load2x2(P + (int64_t)l * 4 * nv + v, nv, out);
    }
  };
  for (int s = 0; s < dg; ++s) {
    const int b = nbr_idx[p0 + s];
    F acc[4] = {F(0), F(0), F(0), F(0)};
    for (int l = 0; l <= L; ++l) {
      F Pa[4];
      pblk(l, a, Pa);
      const int nl = bp_nlev(l, L), lmin = l > 0 ? l - 1 : 0;
      for (int d = 0; d < nl; ++d) {
        const int lp = lmin + d;
        F A[4], Pb[4], t[4];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int cp = 0; cp < 2; ++cp) A[2 * c + cp] = (F)J[col_entry(vs, dg, s, l, c, lp, cp, L)];
        pblk(lp, b, Pb);
        // t = A Pb;  acc += Pa^T t
        t[0] = A[0] * Pb[0] + A[1] * Pb[2];
        t[1] = A[0] * Pb[1] + A[1] * Pb[3];
        t[2] = A[2] * Pb[0] + A[3] * Pb[2];
        t[3] = A[2] * Pb[1] + A[3] * Pb[3];
        acc[0] += Pa[0] * t[0] + Pa[2] * t[2];
        acc[1] += Pa[0] * t[1] + Pa[2] * t[3];
        acc[2] += Pa[1] * t[0] + Pa[3] * t[2];
        acc[3] += Pa[1] * t[1] + Pa[3] * t[3];
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) Ac[(int64_t)(p0 + s) * 4 + e] = acc[e];
  }
  F D[4], Di[4];
  load2x2(Ac + (int64_t)(p0 + dslot[a]) * 4, 1, D);
  const F idet = F(1) / (D[0] * D[3] - D[1] * D[2]);
  Di[0] = D[3] * idet, Di[1] = -D[1] * idet, Di[2] = -D[2] * idet, Di[3] = D[0] * idet;
#pragma unroll
  for (int e = 0; e < 4; ++e) Dinv[(int64_t)a * 4 + e] = Di[e];
  F s0 = F(0), s1 = F(0);
  for (int s = 0; s < dg; ++s) {
    F B[4];
    load2x2(Ac + (int64_t)(p0 + s) * 4, 1, B);
    s0 += fabs(Di[0] * B[0] + Di[1] * B[2]) + fabs(Di[0] * B[1] + Di[1] * B[3]);
    s1 += fabs(Di[2] * B[0] + Di[3] * B[2]) + fabs(Di[2] * B[1] + Di[3] * B[3]);
  }
  const double g = (double)(s0 > s1 ? s0 : s1);
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(lam), (unsigned long long)__double_as_longlong(g));
}

// out = (base ? base : 0) + omega T^-1 r, one thread per column (sb: scratch for T^-1 r).
template <class V, class F>
__global__ void __launch_bounds__(128) k_mdsc_smooth(const Prec<F> Pr, const V* __restrict__ r, V* __restrict__ sb,
                                                     const V* base, V* out, F omega) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= Pr.nv) return;
  const int64_t off = 2LL * a * (Pr.L + 1);
  double rz, rr;
  colprec_apply(Pr, a, r, sb, &rz, &rr, off);
  for (int i = 0; i < 2 * (Pr.L + 1); ++i) {
    const V v = (V)(omega * (F)sb[off + i]);
    out[off + i] = base ? base[off + i] + v : v;
  }
}

// The same for FP32 columns of NLEV levels: one warp per 32 columns, factors in registers, r staged
// in shared memory (as in the CG update).
template <int NLEV>
__global__ void __launch_bounds__(UPD_NT) k_mdsc_smooth_cols(const Prec<float> Pr, const float* __restrict__ r,
                                                             const float* base, float* out, float omega) {
  constexpr int N = 2 * NLEV;
  constexpr int SN = N | 1;
  __shared__ float sbuf[UPD_NT / 32][32 * SN];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a0 = (blockIdx.x * (UPD_NT / 32) + warp) * 32;
  const bool own = a0 + lane < Pr.nv;
  ColFactors<NLEV> f;
  if (own) f.load(Pr, a0 + lane);
  float* sr = sbuf[warp];
  const int ncol = min(32, Pr.nv - a0);
  const int64_t b0 = (int64_t)a0 * N;
  for (int i = lane; i < ncol * N; i += 32) sr[(i / N) * SN + i % N] = r[b0 + i];
  __syncwarp();
  if (own) f.solve(sr + lane * SN);
  __syncwarp();
  for (int i = lane; i < ncol * N; i += 32) {
    const float v = omega * sr[(i / N) * SN + i % N];
    out[b0 + i] = base ? base[b0 + i] + v : v;
  }
}

// out = base + omega T^-1 r with the fastest applicable kernel
template <class V, class F>
void mdsc_smooth(const Prec<F>& Pr, const V* r, V* sb, const V* base, V* out, F omega, cudaStream_t s) {
  if constexpr (std::is_same<V, float>::value && std::is_same<F, float>::value) {
    const int grid = (Pr.nv + UPD_NT - 1) / UPD_NT;
    if (Pr.L == 10) {
      k_mdsc_smooth_cols<11><<<grid, UPD_NT, 0, s>>>(Pr, r, base, out, omega);
      return;
    }
    if (Pr.L == 5) {
      k_mdsc_smooth_cols<6><<<grid, UPD_NT, 0, s>>>(Pr, r, base, out, omega);
      return;
    }
  }
  k_mdsc_smooth<V, F><<<(Pr.nv + 127) / 128, 128, 0, s>>>(Pr, r, sb, base, out, omega);
}

// t = r - t (element-wise)
template <class V>
__global__ void __launch_bounds__(NT) k_mdsc_sub(const V* __restrict__ r, V* __restrict__ t, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    t[i] = r[i] - t[i];
}

// rc = P^T t, one thread per column
template <class V, class F>
__global__ void __launch_bounds__(128) k_mdsc_restrict(const F* __restrict__ P, const V* __restrict__ t,
                                                       F* __restrict__ rc, int nv, int L) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  const int64_t base = 2LL * a * (L + 1);
  F r0 = (F)t[base + 2 * L], r1 = (F)t[base + 2 * L + 1];
  for (int l = 0; l < L; ++l) {
    F Pl[4];
    load2x2(P + (int64_t)l * 4 * nv + a, nv, Pl);
    const F v0 = (F)t[base + 2 * l], v1 = (F)t[base + 2 * l + 1];
    r0 += Pl[0] * v0 + Pl[2] * v1;
    r1 += Pl[1] * v0 + Pl[3] * v1;
  }
  rc[2 * a] = r0;
  rc[2 * a + 1] = r1;
}

// z += P ec, one thread per column
template <class V, class F>
__global__ void __launch_bounds__(128) k_mdsc_prolong_add(const F* __restrict__ P, const F* __restrict__ ec,
                                                          V* __restrict__ z, int nv, int L) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  const int64_t base = 2LL * a * (L + 1);
  const F e0 = ec[2 * a], e1 = ec[2 * a + 1];
  for (int l = 0; l < L; ++l) {
    F Pl[4];
    load2x2(P + (int64_t)l * 4 * nv + a, nv, Pl);
    z[base + 2 * l] += (V)(Pl[0] * e0 + Pl[1] * e1);
    z[base + 2 * l + 1] += (V)(Pl[2] * e0 + Pl[3] * e1);
  }
  z[base + 2 * L] += (V)e0;
  z[base + 2 * L + 1] += (V)e1;
}

// Chebyshev acceleration (Saad, Sec. 12.3) of block-Jacobi on A_c from x = 0:
//   start  x = 0, r = b, d = D^-1 r / theta;
//   step   x += d, r -= A_c d, d = rho' rho d + (2 rho' / delta) D^-1 r   (coefficients in cheb).
template <class F>
__global__ void __launch_bounds__(NT) k_mdsc_cheb_init(const F* __restrict__ Dinv, const double* __restrict__ cheb,
                                                       const F* __restrict__ b, F* __restrict__ x, F* __restrict__ r,
                                                       F* __restrict__ d, int nv) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  const F it = (F)cheb[0];
  const F b0 = b[2 * a], b1 = b[2 * a + 1];
  F Di[4];
  load2x2(Dinv + (int64_t)a * 4, 1, Di);
  x[2 * a] = F(0);
  x[2 * a + 1] = F(0);
  r[2 * a] = b0;
  r[2 * a + 1] = b1;
  d[2 * a] = it * (Di[0] * b0 + Di[1] * b1);
  d[2 * a + 1] = it * (Di[2] * b0 + Di[3] * b1);
}

template <class F>
__global__ void __launch_bounds__(NT) k_mdsc_cheb_step(const F* __restrict__ Ac, const F* __restrict__ Dinv,
                                                       const int32_t* __restrict__ nbr_ptr,
                                                       const int32_t* __restrict__ nbr_idx,
                                                       const double* __restrict__ cheb, int k,
                                                       const F* __restrict__ d, F* __restrict__ dn,
                                                       F* __restrict__ x, F* __restrict__ r, int nv) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  F q0 = F(0), q1 = F(0);
  for (int i = nbr_ptr[a]; i < nbr_ptr[a + 1]; ++i) {
    const int b = nbr_idx[i];
    F B[4];
    load2x2(Ac + (int64_t)i * 4, 1, B);
    const F d0 = d[2 * b], d1 = d[2 * b + 1];
    q0 += B[0] * d0 + B[1] * d1;
    q1 += B[2] * d0 + B[3] * d1;
  }
  const F da0 = d[2 * a], da1 = d[2 * a + 1];
  x[2 * a] += da0;
  x[2 * a + 1] += da1;
  const F r0 = r[2 * a] - q0, r1 = r[2 * a + 1] - q1;
  r[2 * a] = r0;
  r[2 * a + 1] = r1;
  F Di[4];
  load2x2(Dinv + (int64_t)a * 4, 1, Di);
  const F c1 = (F)cheb[1 + 2 * k], c2 = (F)cheb[2 + 2 * k];
  dn[2 * a] = c1 * da0 + c2 * (Di[0] * r0 + Di[1] * r1);
  dn[2 * a + 1] = c1 * da1 + c2 * (Di[2] * r0 + Di[3] * r1);
}

template <class F>
int mdsc_alloc(bp_mesh* m) {
  bp_solver_ws* w = m->ws;
  if (w->mP) return BP_OK;
  int rc;
  const int64_t n = m->ndof, nv = m->nv, L = m->nl;
  w->nbr_total = m->nnz / (4 * (3 * L + 1));  // nv + 2 E: the closed-neighbourhood entries
#define MD_ALLOC(ptr, cnt) \
  if ((rc = bp_alloc(m, &(ptr), (cnt))) != BP_OK) return rc
  MD_ALLOC(w->mP, 4 * std::max<int64_t>(L, 1) * nv);
  MD_ALLOC(w->mAc, 4 * w->nbr_total);
  MD_ALLOC(w->mDinv, 4 * nv);
  MD_ALLOC(w->mcheb, 2 * MDSC_STEPS + 2);
  MD_ALLOC(w->mlam, 1);
  MD_ALLOC(w->mz1, n);
  MD_ALLOC(w->mt, n);
  MD_ALLOC(w->ms, n);
  MD_ALLOC(w->mrc, 2 * nv);
  MD_ALLOC(w->mec, 2 * nv);
  MD_ALLOC(w->mrr, 2 * nv);
  MD_ALLOC(w->md0, 2 * nv);
  MD_ALLOC(w->md1, 2 * nv);
#undef MD_ALLOC
  return BP_OK;
}

// Setup from the same-precision Jacobian (the column factors are set up first): P, A_c, D^-1, the
// Gershgorin bound (read back once) and the Chebyshev coefficients.  F: factor / plane type.
template <class M>
int mdsc_setup_t(bp_mesh* m, const M* J, cudaStream_t s) {
  using F = M;
  int rc = colprec_setup_t(m, J, s);
  if (rc) return rc;
  if ((rc = mdsc_alloc<F>(m))) return rc;
  bp_solver_ws* w = m->ws;
  const int gcol = (m->nv + 127) / 128;
  F* P = reinterpret_cast<F*>(w->mP);
  k_mdsc_prolong<F><<<gcol, 128, 0, s>>>(prec_of<F>(m), P);
  BP_CUDA_TRY(cudaMemsetAsync(w->mlam, 0, sizeof(double), s));
  k_mdsc_plane<M, F><<<gcol, 128, 0, s>>>(J, m->vstart, m->vdeg, w->dslot, m->nbr_ptr, m->nbr_idx, P, m->nv, m->nl,
                                          reinterpret_cast<F*>(w->mAc), reinterpret_cast<F*>(w->mDinv), w->mlam);
  BP_CUDA_TRY(cudaGetLastError());
  BP_CUDA_TRY(cudaMemcpyAsync(w->host, w->mlam, sizeof(double), cudaMemcpyDeviceToHost, s));
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  const double lam_hi = w->host[0];
  if (!(lam_hi > 0) || !std::isfinite(lam_hi)) return BP_ENAN;
  const double lam_lo = lam_hi / MDSC_RATIO;
  const double theta = 0.5 * (lam_hi + lam_lo), delta = 0.5 * (lam_hi - lam_lo), sigma = theta / delta;
  double* c = w->host;  // staged in the pinned mirror (synchronised below)
  c[0] = 1.0 / theta;
  double rho = 1.0 / sigma;
  for (int k = 0; k < MDSC_STEPS; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    c[1 + 2 * k] = rn * rho;
    c[2 + 2 * k] = 2.0 * rn / delta;
    rho = rn;
  }
  BP_CUDA_TRY(cudaMemcpyAsync(w->mcheb, c, (2 * MDSC_STEPS + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  w->has_mdsc = true;
  w->mdsc_f32 = sizeof(F) == sizeof(float);
  return BP_OK;
}

// ------------------------------------------------------------------ SA-AMG plane solve of the MDSC cycle
// Paper Sec. 4.4 / Sec. 3.1: after the vertical semicoarsening to one layer, the plane problem A_c is
// solved by smoothed-aggregation algebraic multigrid with a Chebyshev smoother.  Statement (on 2 x 2
// blocks, u and v per vertex):
//   aggregation of the level's block graph (pattern of A_k, a vertex adjacent to itself): pass 1 in
//     vertex order, a vertex whose whole neighbourhood is free starts an aggregate of that
//     neighbourhood; pass 2, a vertex still free joins the pass-1 aggregate of its lowest-numbered
//     neighbour that pass 1 aggregated;
//   P_k = (I - omega D^-1 A_k) Pt, Pt(i, agg(i)) = I, omega = 4 / (3 lam_k), lam_k the Gershgorin
//     bound of D^-1 A_k;  A_{k+1} = P_k^T A_k P_k;
//   coarsening stops at <= AMG_COARSE vertices, when a level shrinks by less than AMG_MIN_RATIO, or
//     after AMG_MAX_LEVELS levels; the coarsest level is solved with its dense inverse;
//   V-cycle: AMG_SMOOTH Chebyshev steps (block Jacobi over [lam / MDSC_RATIO, lam], from zero),
//     coarse correction, the same polynomial on the new residual (symmetric positive definite).
// The aggregates and every sparsity pattern depend on the mesh only: they are built once per mesh on
// the host, with the index lists that the numeric products need (P values: the A entries summed per
// entry; T = A P: (A, P) entry pairs; A_{k+1} = P^T T: (P, T) entry pairs); each Newton step then
// forms P, T, A_{k+1}, D^-1, lam and the dense coarse inverse on the device.
constexpr int AMG_COARSE = 64;
constexpr double AMG_MIN_RATIO = 0.8;
constexpr int AMG_MAX_LEVELS = 8;
constexpr int AMG_SMOOTH = 3;
constexpr int AMG_DENSE_MAX = 512;  // largest coarsest level (vertices) the dense inverse takes

struct AmgLevel {
  int n = 0, nnz = 0;
  const int32_t* ptr = nullptr;  // CSR of A_k over the level's vertices (level 0: the mesh's neighbourhoods)
  const int32_t* col = nullptr;
  int32_t* diag = nullptr;       // [n] entry of the diagonal block
  double *A = nullptr, *Dinv = nullptr, *lam = nullptr, *cheb = nullptr;  // (F storage)
  double *b = nullptr, *x = nullptr, *r = nullptr, *y = nullptr, *rr = nullptr, *d0 = nullptr, *d1 = nullptr;
  // to the next level
  int pnnz = 0, tnnz = 0;
  int32_t *pptr = nullptr, *pcol = nullptr, *prow = nullptr, *ptptr = nullptr, *ptsrc = nullptr;
  int32_t *pvptr = nullptr, *pvsrc = nullptr, *pdiag = nullptr, *tvptr = nullptr, *tvsrc = nullptr;
  int32_t *cvptr = nullptr, *cvsrc = nullptr;
  double *P = nullptr, *T = nullptr;
};

struct AmgHier {
  std::vector<AmgLevel> lv;
  std::vector<std::vector<int32_t>> agg;  // host copies of the aggregates of levels 0 .. L-2
  double* W = nullptr;                    // dense Gauss-Jordan scratch [N][2N], N = 2 n_coarsest
  double* Cinv = nullptr;                 // dense inverse of the coarsest operator [N][N]
};

// ---- host construction (once per mesh)
std::vector<int32_t> amg_aggregate(const std::vector<int32_t>& ptr, const std::vector<int32_t>& col) {
  const int n = (int)ptr.size() - 1;
  std::vector<int32_t> agg(n, -1);
  int count = 0;
  for (int a = 0; a < n; ++a) {
    bool free_nbhd = true;
    for (int e = ptr[a]; e < ptr[a + 1] && free_nbhd; ++e) free_nbhd = agg[col[e]] < 0;
    if (!free_nbhd) continue;
    for (int e = ptr[a]; e < ptr[a + 1]; ++e) agg[col[e]] = count;
    ++count;
  }
  const std::vector<int32_t> first = agg;
  for (int a = 0; a < n; ++a) {
    if (agg[a] >= 0) continue;
    for (int e = ptr[a]; e < ptr[a + 1]; ++e)  // columns sorted: the lowest-numbered such neighbour
      if (first[col[e]] >= 0) {
        agg[a] = first[col[e]];
        break;
      }
  }
  return agg;
}

template <class T>
int amg_upload(bp_mesh* m, const std::vector<T>& v, T** out) {
  int rc = bp_alloc(m, out, v.size());
  if (rc) return rc;
  if (!v.empty()) BP_CUDA_TRY(cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return BP_OK;
}

int amg_level_vectors(bp_mesh* m, AmgLevel& L, bool level0) {
  int rc;
  const size_t n2 = 2 * (size_t)L.n;
  bp_solver_ws* w = m->ws;
  if (level0) {  // borrow the MDSC plane vectors (the one-level Chebyshev plane solve's scratch)
    L.b = w->mrc, L.x = w->mec, L.rr = w->mrr, L.d0 = w->md0, L.d1 = w->md1;
  } else {
    if ((rc = bp_alloc(m, &L.b, n2)) || (rc = bp_alloc(m, &L.x, n2)) || (rc = bp_alloc(m, &L.rr, n2)) ||
        (rc = bp_alloc(m, &L.d0, n2)) || (rc = bp_alloc(m, &L.d1, n2)))
      return rc;
  }
  if ((rc = bp_alloc(m, &L.r, n2)) || (rc = bp_alloc(m, &L.y, n2)) || (rc = bp_alloc(m, &L.cheb, 2 * AMG_SMOOTH + 2)))
    return rc;
  return BP_OK;
}

int amg_build(bp_mesh* m) {
  bp_solver_ws* w = m->ws;
  if (w->amg) return BP_OK;
  std::unique_ptr<AmgHier> owner(new AmgHier());
  AmgHier* H = owner.get();
  int rc = BP_OK;
  // level 0: the plane operator on the base vertices' closed neighbourhoods
  std::vector<int32_t> gptr(m->nv + 1), gcol;
  BP_CUDA_TRY(cudaMemcpy(gptr.data(), m->nbr_ptr, (m->nv + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
  gcol.resize(gptr[m->nv]);
  BP_CUDA_TRY(cudaMemcpy(gcol.data(), m->nbr_idx, gcol.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
  {
    AmgLevel L0;
    L0.n = m->nv;
    L0.nnz = gptr[m->nv];
    L0.ptr = m->nbr_ptr;
    L0.col = m->nbr_idx;
    L0.diag = w->dslot;  // absolute entry = ptr[a] + dslot[a]: see k_amg_diag (level 0 keeps dslot)
    L0.A = w->mAc, L0.Dinv = w->mDinv, L0.lam = w->mlam;
    if ((rc = amg_level_vectors(m, L0, true))) return rc;
    H->lv.push_back(L0);
  }
  for (;;) {
    AmgLevel& L = H->lv.back();
    const int n = L.n;
    if (n <= AMG_COARSE || (int)H->lv.size() >= AMG_MAX_LEVELS) break;
    std::vector<int32_t> agg = amg_aggregate(gptr, gcol);
    int nc = 0;
    for (int32_t a : agg) nc = std::max(nc, a + 1);
    if (nc > AMG_MIN_RATIO * n) break;
    // P: row i holds the aggregates of i's neighbourhood
    std::vector<int32_t> pptr(n + 1, 0), pcol, prow, pvptr(1, 0), pvsrc, pdiag;
    for (int i = 0; i < n; ++i) {
      std::vector<int32_t> js;
      for (int e = gptr[i]; e < gptr[i + 1]; ++e) js.push_back(agg[gcol[e]]);
      std::sort(js.begin(), js.end());
      js.erase(std::unique(js.begin(), js.end()), js.end());
      for (int32_t J : js) {
        pcol.push_back(J);
        prow.push_back(i);
        pdiag.push_back(J == agg[i] ? 1 : 0);
        for (int e = gptr[i]; e < gptr[i + 1]; ++e)
          if (agg[gcol[e]] == J) pvsrc.push_back(e);
        pvptr.push_back((int32_t)pvsrc.size());
      }
      pptr[i + 1] = (int32_t)pcol.size();
    }
    const int pnnz = (int)pcol.size();
    // P^T: per coarse row, its P entries in fine-row order
    std::vector<int32_t> ptptr(nc + 1, 0), ptsrc(pnnz);
    for (int f = 0; f < pnnz; ++f) ++ptptr[pcol[f] + 1];
    for (int I = 0; I < nc; ++I) ptptr[I + 1] += ptptr[I];
    {
      std::vector<int32_t> fill(ptptr.begin(), ptptr.end() - 1);
      for (int f = 0; f < pnnz; ++f) ptsrc[fill[pcol[f]]++] = f;
    }
    // T = A P: row i, columns the P columns of i's neighbours; terms (A entry, P entry)
    std::vector<int32_t> tptr(n + 1, 0), tcol, tvptr(1, 0), tvsrc;
    for (int i = 0; i < n; ++i) {
      std::vector<std::pair<int32_t, std::pair<int32_t, int32_t>>> terms;  // (J, (A entry, P entry))
      for (int e = gptr[i]; e < gptr[i + 1]; ++e) {
        const int j = gcol[e];
        for (int f = pptr[j]; f < pptr[j + 1]; ++f) terms.push_back({pcol[f], {e, f}});
      }
      std::sort(terms.begin(), terms.end());
      for (size_t q = 0; q < terms.size();) {
        const int32_t J = terms[q].first;
        tcol.push_back(J);
        for (; q < terms.size() && terms[q].first == J; ++q) {
          tvsrc.push_back(terms[q].second.first);
          tvsrc.push_back(terms[q].second.second);
        }
        tvptr.push_back((int32_t)(tvsrc.size() / 2));
      }
      tptr[i + 1] = (int32_t)tcol.size();
    }
    // A_{k+1} = P^T T: row I, columns the T columns of the fine rows in aggregate support; terms (P, T)
    std::vector<int32_t> cptr(nc + 1, 0), ccol, cvptr(1, 0), cvsrc, cdiag(nc, -1);
    for (int I = 0; I < nc; ++I) {
      std::vector<std::pair<int32_t, std::pair<int32_t, int32_t>>> terms;
      for (int q = ptptr[I]; q < ptptr[I + 1]; ++q) {
        const int f = ptsrc[q], i = prow[f];
        for (int t = tptr[i]; t < tptr[i + 1]; ++t) terms.push_back({tcol[t], {f, t}});
      }
      std::sort(terms.begin(), terms.end());
      for (size_t q = 0; q < terms.size();) {
        const int32_t J = terms[q].first;
        if (J == I) cdiag[I] = (int32_t)ccol.size() - cptr[I];
        ccol.push_back(J);
        for (; q < terms.size() && terms[q].first == J; ++q) {
          cvsrc.push_back(terms[q].second.first);
          cvsrc.push_back(terms[q].second.second);
        }
        cvptr.push_back((int32_t)(cvsrc.size() / 2));
      }
      cptr[I + 1] = (int32_t)ccol.size();
    }
    // device copies of this level's prolongation data and of the next level
    AmgLevel N;
    N.n = nc;
    N.nnz = (int)ccol.size();
    int32_t *dptr = nullptr, *dcol = nullptr;
    if ((rc = amg_upload(m, pptr, &L.pptr)) || (rc = amg_upload(m, pcol, &L.pcol)) ||
        (rc = amg_upload(m, prow, &L.prow)) || (rc = amg_upload(m, ptptr, &L.ptptr)) ||
        (rc = amg_upload(m, ptsrc, &L.ptsrc)) || (rc = amg_upload(m, pvptr, &L.pvptr)) ||
        (rc = amg_upload(m, pvsrc, &L.pvsrc)) || (rc = amg_upload(m, pdiag, &L.pdiag)) ||
        (rc = amg_upload(m, tvptr, &L.tvptr)) || (rc = amg_upload(m, tvsrc, &L.tvsrc)) ||
        (rc = amg_upload(m, cvptr, &L.cvptr)) || (rc = amg_upload(m, cvsrc, &L.cvsrc)) ||
        (rc = amg_upload(m, cptr, &dptr)) || (rc = amg_upload(m, ccol, &dcol)) ||
        (rc = amg_upload(m, cdiag, &N.diag)) || (rc = bp_alloc(m, &L.P, 4 * (size_t)pnnz)) ||
        (rc = bp_alloc(m, &L.T, 4 * tcol.size())) || (rc = bp_alloc(m, &N.A, 4 * ccol.size())) ||
        (rc = bp_alloc(m, &N.Dinv, 4 * (size_t)nc)) || (rc = bp_alloc(m, &N.lam, 1)))
      return rc;
    L.pnnz = pnnz;
    L.tnnz = (int)tcol.size();
    N.ptr = dptr;
    N.col = dcol;
    if ((rc = amg_level_vectors(m, N, false))) return rc;
    H->agg.push_back(std::move(agg));
    H->lv.push_back(N);
    gptr = std::move(cptr);
    gcol = std::move(ccol);
  }
  const int nco = H->lv.back().n;
  if (nco > AMG_DENSE_MAX) return BP_EUNSUP;
  const size_t N2 = 2 * (size_t)nco;
  if ((rc = bp_alloc(m, &H->W, 2 * N2 * N2)) || (rc = bp_alloc(m, &H->Cinv, N2 * N2))) return rc;
  w->amg = owner.release();
  return BP_OK;
}

// ---- device kernels (F: double or float; blocks row-major uu, uv, vu, vv)
template <class F>
__global__ void __launch_bounds__(128) k_amg_pvals(int pnnz, const int32_t* __restrict__ prow,
                                                   const int32_t* __restrict__ pvptr, const int32_t* __restrict__ pvsrc,
                                                   const int32_t* __restrict__ pdiag, const F* __restrict__ A,
                                                   const F* __restrict__ Dinv, const double* __restrict__ lam,
                                                   F* __restrict__ P) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= pnnz) return;
  const int i = prow[e];
  F S[4] = {F(0), F(0), F(0), F(0)};
  for (int t = pvptr[e]; t < pvptr[e + 1]; ++t)
#pragma unroll
    for (int k = 0; k < 4; ++k) S[k] += A[4 * (int64_t)pvsrc[t] + k];
  F Di[4];
  load2x2(Dinv + 4 * (int64_t)i, 1, Di);
  const F om = (F)(4.0 / (3.0 * *lam));
  const F one = pdiag[e] ? F(1) : F(0);
  P[4 * (int64_t)e + 0] = one - om * (Di[0] * S[0] + Di[1] * S[2]);
  P[4 * (int64_t)e + 1] = -om * (Di[0] * S[1] + Di[1] * S[3]);
  P[4 * (int64_t)e + 2] = -om * (Di[2] * S[0] + Di[3] * S[2]);
  P[4 * (int64_t)e + 3] = one - om * (Di[2] * S[1] + Di[3] * S[3]);
}

// out[e] = sum over the entry's pairs (a, b) of X[a]^(T if TX) Y[b]
template <class F, bool TX>
__global__ void __launch_bounds__(128) k_amg_pairs(int nnz, const int32_t* __restrict__ vptr,
                                                   const int32_t* __restrict__ vsrc, const F* __restrict__ X,
                                                   const F* __restrict__ Y, F* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  F o[4] = {F(0), F(0), F(0), F(0)};
  for (int t = vptr[e]; t < vptr[e + 1]; ++t) {
    F a[4], b[4];
    load2x2(X + 4 * (int64_t)vsrc[2 * t], 1, a);
    load2x2(Y + 4 * (int64_t)vsrc[2 * t + 1], 1, b);
    if (TX) {
      const F t1 = a[1];
      a[1] = a[2];
      a[2] = t1;
    }
    o[0] += a[0] * b[0] + a[1] * b[2];
    o[1] += a[0] * b[1] + a[1] * b[3];
    o[2] += a[2] * b[0] + a[3] * b[2];
    o[3] += a[2] * b[1] + a[3] * b[3];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) out[4 * (int64_t)e + k] = o[k];
}

// D^-1 of the diagonal blocks and the Gershgorin bound of D^-1 A (atomic maximum; lam zeroed before)
template <class F>
__global__ void __launch_bounds__(128) k_amg_diag(int n, const int32_t* __restrict__ ptr,
                                                  const int32_t* __restrict__ diag, const F* __restrict__ A,
                                                  F* __restrict__ Dinv, double* lam) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  F D[4], Di[4];
  load2x2(A + 4 * (int64_t)(ptr[a] + diag[a]), 1, D);
  const F idet = F(1) / (D[0] * D[3] - D[1] * D[2]);
  Di[0] = D[3] * idet, Di[1] = -D[1] * idet, Di[2] = -D[2] * idet, Di[3] = D[0] * idet;
#pragma unroll
  for (int e = 0; e < 4; ++e) Dinv[(int64_t)a * 4 + e] = Di[e];
  F s0 = F(0), s1 = F(0);
  for (int e = ptr[a]; e < ptr[a + 1]; ++e) {
    F B[4];
    load2x2(A + 4 * (int64_t)e, 1, B);
    s0 += fabs(Di[0] * B[0] + Di[1] * B[2]) + fabs(Di[0] * B[1] + Di[1] * B[3]);
    s1 += fabs(Di[2] * B[0] + Di[3] * B[2]) + fabs(Di[2] * B[1] + Di[3] * B[3]);
  }
  const double g = (double)(s0 > s1 ? s0 : s1);
  atomicMax(reinterpret_cast<unsigned long long*>(lam), (unsigned long long)__double_as_longlong(g));
}

// Chebyshev coefficients over [lam / ratio, lam] (the recurrence of the MDSC plane iteration)
__global__ void k_amg_cheb(const double* lam, double ratio, int steps, double* c) {
  const double hi = *lam, lo = hi / ratio;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  c[0] = 1.0 / theta;
  double rho = 1.0 / sigma;
  for (int k = 0; k < steps; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    c[1 + 2 * k] = rn * rho;
    c[2 + 2 * k] = 2.0 * rn / delta;
    rho = rn;
  }
}

// Dense inverse of the coarsest operator by Gauss-Jordan elimination without pivoting (SPD), one block.
template <class F>
__global__ void __launch_bounds__(256) k_amg_dense_inverse(int n, const int32_t* __restrict__ ptr,
                                                           const int32_t* __restrict__ col, const F* __restrict__ A,
                                                           F* __restrict__ W, F* __restrict__ Cinv) {
  const int N = 2 * n, N2 = 2 * N;
  __shared__ F fcol[2 * AMG_DENSE_MAX];
  for (int idx = threadIdx.x; idx < N * N2; idx += blockDim.x) {
    const int i = idx / N2, j = idx % N2;
    W[idx] = (j == N + i) ? F(1) : F(0);
  }
  __syncthreads();
  for (int a = threadIdx.x; a < n; a += blockDim.x)
    for (int e = ptr[a]; e < ptr[a + 1]; ++e)
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) W[(2 * a + r) * N2 + 2 * col[e] + c] = A[4 * (int64_t)e + 2 * r + c];
  __syncthreads();
  for (int p = 0; p < N; ++p) {
    const F ip = F(1) / W[p * N2 + p];
    __syncthreads();
    for (int j = threadIdx.x; j < N2; j += blockDim.x) W[p * N2 + j] *= ip;
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) fcol[i] = (i == p) ? F(0) : W[i * N2 + p];
    __syncthreads();
    for (int idx = threadIdx.x; idx < N * N2; idx += blockDim.x) {
      const int i = idx / N2, j = idx % N2;
      if (i != p) W[idx] -= fcol[i] * W[p * N2 + j];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int i = idx / N, j = idx % N;
    Cinv[idx] = W[i * N2 + N + j];
  }
}

template <class F>
__global__ void __launch_bounds__(256) k_amg_dense_apply(int N, const F* __restrict__ Cinv, const F* __restrict__ b,
                                                         F* __restrict__ x) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    F s = F(0);
    for (int j = 0; j < N; ++j) s += Cinv[(int64_t)i * N + j] * b[j];
    x[i] = s;
  }
}

// r = b - A x
template <class F>
__global__ void __launch_bounds__(128) k_amg_residual(int n, const int32_t* __restrict__ ptr,
                                                      const int32_t* __restrict__ col, const F* __restrict__ A,
                                                      const F* __restrict__ x, const F* __restrict__ b,
                                                      F* __restrict__ r) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  F q0 = F(0), q1 = F(0);
  for (int e = ptr[a]; e < ptr[a + 1]; ++e) {
    F B[4];
    load2x2(A + 4 * (int64_t)e, 1, B);
    const int c = col[e];
    q0 += B[0] * x[2 * c] + B[1] * x[2 * c + 1];
    q1 += B[2] * x[2 * c] + B[3] * x[2 * c + 1];
  }
  r[2 * a] = b[2 * a] - q0;
  r[2 * a + 1] = b[2 * a + 1] - q1;
}

// bc = P^T r (one thread per coarse vertex)
template <class F>
__global__ void __launch_bounds__(128) k_amg_restrict(int nc, const int32_t* __restrict__ ptptr,
                                                      const int32_t* __restrict__ ptsrc,
                                                      const int32_t* __restrict__ prow, const F* __restrict__ P,
                                                      const F* __restrict__ r, F* __restrict__ bc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  F s0 = F(0), s1 = F(0);
  for (int q = ptptr[I]; q < ptptr[I + 1]; ++q) {
    const int f = ptsrc[q], i = prow[f];
    F B[4];
    load2x2(P + 4 * (int64_t)f, 1, B);
    s0 += B[0] * r[2 * i] + B[2] * r[2 * i + 1];
    s1 += B[1] * r[2 * i] + B[3] * r[2 * i + 1];
  }
  bc[2 * I] = s0;
  bc[2 * I + 1] = s1;
}

// x += P xc (one thread per fine vertex)
template <class F>
__global__ void __launch_bounds__(128) k_amg_prolong_add(int n, const int32_t* __restrict__ pptr,
                                                         const int32_t* __restrict__ pcol, const F* __restrict__ P,
                                                         const F* __restrict__ xc, F* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  F s0 = F(0), s1 = F(0);
  for (int f = pptr[i]; f < pptr[i + 1]; ++f) {
    F B[4];
    load2x2(P + 4 * (int64_t)f, 1, B);
    const int J = pcol[f];
    s0 += B[0] * xc[2 * J] + B[1] * xc[2 * J + 1];
    s1 += B[2] * xc[2 * J] + B[3] * xc[2 * J + 1];
  }
  x[2 * i] += s0;
  x[2 * i + 1] += s1;
}

template <class F>
__global__ void __launch_bounds__(NT) k_amg_add(int n2, const F* __restrict__ y, F* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n2) x[i] += y[i];
}

template <class F>
F* fp(double* p) {
  return reinterpret_cast<F*>(p);
}

// Numeric setup of the hierarchy from level 0 (A_c, D^-1, lam already formed by mdsc_setup_t).
template <class F>
int amg_numeric(bp_mesh* m, cudaStream_t s) {
  AmgHier* H = static_cast<AmgHier*>(m->ws->amg);
  const int nl = (int)H->lv.size();
  for (int k = 0; k < nl; ++k) {
    AmgLevel& L = H->lv[k];
    if (k > 0) {
      BP_CUDA_TRY(cudaMemsetAsync(L.lam, 0, sizeof(double), s));
      k_amg_diag<F><<<(L.n + 127) / 128, 128, 0, s>>>(L.n, L.ptr, L.diag, fp<F>(L.A), fp<F>(L.Dinv), L.lam);
    }
    if (k == nl - 1) break;
    k_amg_cheb<<<1, 1, 0, s>>>(L.lam, MDSC_RATIO, AMG_SMOOTH, L.cheb);
    AmgLevel& N = H->lv[k + 1];
    k_amg_pvals<F><<<(L.pnnz + 127) / 128, 128, 0, s>>>(L.pnnz, L.prow, L.pvptr, L.pvsrc, L.pdiag, fp<F>(L.A),
                                                        fp<F>(L.Dinv), L.lam, fp<F>(L.P));
    k_amg_pairs<F, false><<<(L.tnnz + 127) / 128, 128, 0, s>>>(L.tnnz, L.tvptr, L.tvsrc, fp<F>(L.A), fp<F>(L.P),
                                                               fp<F>(L.T));
    k_amg_pairs<F, true><<<(N.nnz + 127) / 128, 128, 0, s>>>(N.nnz, L.cvptr, L.cvsrc, fp<F>(L.P), fp<F>(L.T),
                                                             fp<F>(N.A));
  }
  const AmgLevel& C = H->lv.back();
  k_amg_dense_inverse<F><<<1, 256, 0, s>>>(C.n, C.ptr, C.col, fp<F>(C.A), fp<F>(H->W), fp<F>(H->Cinv));
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

// x_k = V-cycle(b_k) on level k
template <class F>
void amg_vcycle(const AmgHier* H, int k, cudaStream_t s) {
  const AmgLevel& L = H->lv[k];
  const int g = (L.n + 127) / 128, gv = (L.n + NT - 1) / NT;
  if (k == (int)H->lv.size() - 1) {
    k_amg_dense_apply<F><<<1, 256, 0, s>>>(2 * L.n, fp<F>(H->Cinv), fp<F>(L.b), fp<F>(L.x));
    return;
  }
  F* d[2] = {fp<F>(L.d0), fp<F>(L.d1)};
  // pre-smoothing: x = Cheb(b) from zero
  k_mdsc_cheb_init<F><<<gv, NT, 0, s>>>(fp<F>(L.Dinv), L.cheb, fp<F>(L.b), fp<F>(L.x), fp<F>(L.rr), d[0], L.n);
  for (int q = 0; q < AMG_SMOOTH; ++q)
    k_mdsc_cheb_step<F><<<gv, NT, 0, s>>>(fp<F>(L.A), fp<F>(L.Dinv), L.ptr, L.col, L.cheb, q, d[q & 1],
                                          d[(q + 1) & 1], fp<F>(L.x), fp<F>(L.rr), L.n);
  // coarse correction
  const AmgLevel& N = H->lv[k + 1];
  k_amg_residual<F><<<g, 128, 0, s>>>(L.n, L.ptr, L.col, fp<F>(L.A), fp<F>(L.x), fp<F>(L.b), fp<F>(L.r));
  k_amg_restrict<F><<<(N.n + 127) / 128, 128, 0, s>>>(N.n, L.ptptr, L.ptsrc, L.prow, fp<F>(L.P), fp<F>(L.r),
                                                      fp<F>(N.b));
  amg_vcycle<F>(H, k + 1, s);
  k_amg_prolong_add<F><<<g, 128, 0, s>>>(L.n, L.pptr, L.pcol, fp<F>(L.P), fp<F>(N.x), fp<F>(L.x));
  // post-smoothing: x += Cheb(b - A x)
  k_amg_residual<F><<<g, 128, 0, s>>>(L.n, L.ptr, L.col, fp<F>(L.A), fp<F>(L.x), fp<F>(L.b), fp<F>(L.r));
  k_mdsc_cheb_init<F><<<gv, NT, 0, s>>>(fp<F>(L.Dinv), L.cheb, fp<F>(L.r), fp<F>(L.y), fp<F>(L.rr), d[0], L.n);
  for (int q = 0; q < AMG_SMOOTH; ++q)
    k_mdsc_cheb_step<F><<<gv, NT, 0, s>>>(fp<F>(L.A), fp<F>(L.Dinv), L.ptr, L.col, L.cheb, q, d[q & 1],
                                          d[(q + 1) & 1], fp<F>(L.y), fp<F>(L.rr), L.n);
  k_amg_add<F><<<(2 * L.n + NT - 1) / NT, NT, 0, s>>>(2 * L.n, fp<F>(L.y), fp<F>(L.x));
}

// MDSC setup with the SA-AMG plane solve: the two-level setup (column factors, P, A_c, D^-1, lam),
// the hierarchy's patterns (first call on the mesh) and its numeric setup.
template <class M>
int mdsc_amg_setup_t(bp_mesh* m, const M* J, cudaStream_t s) {
  int rc = mdsc_setup_t(m, J, s);
  if (rc) return rc;
  if ((rc = amg_build(m))) return rc;
  return amg_numeric<M>(m, s);
}

// z = M^-1 r (the cycle above) for vectors V, Jacobian values M, factors and plane data F.
template <class M, class V, class F, bool AMG = false>
void mdsc_apply_launch(bp_mesh* m, const M* J, const V* r, V* z, cudaStream_t s) {
  bp_solver_ws* w = m->ws;
  const Prec<F> Pr = prec_of<F>(m);
  const F* P = reinterpret_cast<const F*>(w->mP);
  const F* Ac = reinterpret_cast<const F*>(w->mAc);
  const F* Dinv = reinterpret_cast<const F*>(w->mDinv);
  F* rc = reinterpret_cast<F*>(w->mrc);
  F* ec = reinterpret_cast<F*>(w->mec);
  F* rr = reinterpret_cast<F*>(w->mrr);
  F* d[2] = {reinterpret_cast<F*>(w->md0), reinterpret_cast<F*>(w->md1)};
  V* z1 = reinterpret_cast<V*>(w->mz1);
  V* t = reinterpret_cast<V*>(w->mt);
  V* sb = reinterpret_cast<V*>(w->ms);
  const int64_t n = m->ndof;
  const int gcol = (m->nv + 127) / 128, gv = (m->nv + NT - 1) / NT;
  const int gvec = grid_for(n, NT);
  const F omega = (F)MDSC_OMEGA;
  // z1 = S r
  mdsc_smooth<V, F>(Pr, r, sb, nullptr, z1, omega, s);
  // rc = P^T (r - J z1)
  spmv_launch<M, V, false>(m, J, z1, t, nullptr, nullptr, nullptr, 0, s);
  k_mdsc_sub<V><<<gvec, NT, 0, s>>>(r, t, n);
  k_mdsc_restrict<V, F><<<gcol, 128, 0, s>>>(P, t, rc, m->nv, m->nl);
  // ec = B_c rc: the Chebyshev plane iteration, or one SA-AMG V-cycle (level 0 reads rc, writes ec)
  if constexpr (AMG) {
    amg_vcycle<F>(static_cast<const AmgHier*>(w->amg), 0, s);
  } else {
    k_mdsc_cheb_init<F><<<gv, NT, 0, s>>>(Dinv, w->mcheb, rc, ec, rr, d[0], m->nv);
    for (int k = 0; k < MDSC_STEPS; ++k)
      k_mdsc_cheb_step<F><<<gv, NT, 0, s>>>(Ac, Dinv, m->nbr_ptr, m->nbr_idx, w->mcheb, k, d[k & 1],
                                            d[(k + 1) & 1], ec, rr, m->nv);
  }
  // z2 = z1 + P ec (in z1);  z = z2 + S (r - J z2)
  k_mdsc_prolong_add<V, F><<<gcol, 128, 0, s>>>(P, ec, z1, m->nv, m->nl);
  spmv_launch<M, V, false>(m, J, z1, t, nullptr, nullptr, nullptr, 0, s);
  k_mdsc_sub<V><<<gvec, NT, 0, s>>>(r, t, n);
  mdsc_smooth<V, F>(Pr, t, sb, z1, z, omega, s);
}

// ---- preconditioned CG with the MDSC cycle (device scalars as in cg_solve)
// x = 0, r = -R, and r.r of step 0
template <class V>
__global__ void __launch_bounds__(NT) k_pcg_init(const double* __restrict__ R, V* __restrict__ x, V* __restrict__ r,
                                                 int64_t n, double* scal) {
  V rr = V(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const V v = (V)(-R[i]);
    x[i] = V(0);
    r[i] = v;
    rr += v * v;
  }
  block_add(rr, scal + 2);
}

// alpha = r.z / p.Ap, x += alpha p, r -= alpha q, and r.r of step k + 1
template <class V>
__global__ void __launch_bounds__(NT) k_pcg_update(const int* kbase, int j, V* __restrict__ x, V* __restrict__ r,
                                                   const V* __restrict__ p, const V* __restrict__ q, int64_t n,
                                                   double* scal, int* stop) {
  __shared__ V s_alpha;
  __shared__ int s_bad;
  if (*stop) return;
  const int k = *kbase + j;
  if (threadIdx.x == 0) {
    const double pq = scal[3 * k], rzk = scal[3 * k + 1];
    s_bad = !(pq > 0.0) || !isfinite(rzk);
    s_alpha = s_bad ? V(0) : (V)(rzk / pq);
    if (s_bad && blockIdx.x == 0) *stop = 2;
  }
  __syncthreads();
  if (s_bad) return;
  const V alpha = s_alpha;
  V rr = V(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const V v = r[i] - alpha * q[i];
    r[i] = v;
    rr += v * v;
  }
  block_add(rr, scal + 3 * (k + 1) + 2);
}

// r.z into scal[3 (kbase + j + shift) + 1]
template <class V>
__global__ void __launch_bounds__(NT) k_pcg_rz(const int* kbase, int j, int shift, const V* __restrict__ r,
                                               const V* __restrict__ z, int64_t n, double* scal, const int* stop) {
  if (*stop) return;
  V acc = V(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += r[i] * z[i];
  block_add(acc, scal + 3 * (*kbase + j + shift) + 1);
}

// One MDSC-preconditioned CG iteration (the loop body when `loop` is set).
template <class M, class V, bool AMG = false>
void launch_mdsc_iteration(bp_mesh* m, const M* J, cudaStream_t s, cudaGraphConditionalHandle loop, int set_loop) {
  bp_solver_ws* w = m->ws;
  const int64_t n = m->ndof;
  V* x = reinterpret_cast<V*>(w->x);
  V* r = reinterpret_cast<V*>(w->r);
  V* z = reinterpret_cast<V*>(w->z);
  V* p = reinterpret_cast<V*>(w->p);
  V* q = reinterpret_cast<V*>(w->q);
  const int gvec = grid_for(n, NT);
  spmv_launch<M, V, true>(m, J, p, q, w->scal, w->stop, w->kbase, 0, s);
  k_pcg_update<V><<<gvec, NT, 0, s>>>(w->kbase, 0, x, r, p, q, n, w->scal, w->stop);
  mdsc_apply_launch<M, V, V, AMG>(m, J, r, z, s);
  k_pcg_rz<V><<<gvec, NT, 0, s>>>(w->kbase, 0, 1, r, z, n, w->scal, w->stop);
  k_cg_direction<V><<<grid_for(n / 2, NT), NT, 0, s>>>(w->kbase, 0, w->cgpar, n / 2, z, p, w->scal, w->stop, loop,
                                                       set_loop);
  k_cg_advance<<<1, 1, 0, s>>>(w->kbase, 1);
}

template <class M, class V, bool AMG = false>
int mdsc_loop_graph(bp_mesh* m, const M* J, cudaGraphExec_t* out) {
  bp_solver_ws* w = m->ws;
  const int slot = sizeof(V) == sizeof(float) ? 1 : 0;
  void** loops = AMG ? w->amg_loop : w->mdsc_loop;
  *out = nullptr;
  if (w->cg_loop_failed[slot]) return BP_OK;
  if (!loops[slot]) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraphConditionalHandle h{};
    cudaGraphNodeParams cp{};
    cudaGraphNode_t node = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      launch_mdsc_iteration<M, V, AMG>(m, J, cs, h, 1);
      const cudaError_t le = cudaGetLastError();  // a launch the capture refused
      cudaGraph_t body = nullptr;
      e = cudaStreamEndCapture(cs, &body);
      if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return BP_OK;  // the caller iterates from the host
    }
    loops[slot] = exec;
  }
  *out = (cudaGraphExec_t)loops[slot];
  return BP_OK;
}

// MDSC-preconditioned CG on J delta = -R to ||r|| <= eta ||R||; delta in ws->x (type V).  The
// Jacobian J must be the one mdsc_setup_t saw (captured in the loop graph by address).
template <class M, class V, bool AMG = false>
int mdsc_cg_solve(bp_mesh* m, const M* J, double eta, int maxit, bool device_loop, cudaStream_t s, int* iters,
                  int* status) {
  bp_solver_ws* w = m->ws;
  maxit = std::min(maxit, w->scal_cap);
  const int64_t n = m->ndof;
  V* r = reinterpret_cast<V*>(w->r);
  V* z = reinterpret_cast<V*>(w->z);
  V* p = reinterpret_cast<V*>(w->p);
  cudaGraphExec_t loop = nullptr;
  int rc = device_loop ? mdsc_loop_graph<M, V, AMG>(m, J, &loop) : BP_OK;
  if (rc) return rc;
  BP_CUDA_TRY(cudaMemsetAsync(w->scal, 0, 3 * (size_t)(maxit + 2 + CG_BATCH) * sizeof(double), s));
  BP_CUDA_TRY(cudaMemsetAsync(w->stop, 0, sizeof(int), s));
  BP_CUDA_TRY(cudaMemsetAsync(w->kbase, 0, sizeof(int), s));
  w->hpar[0] = eta * eta;
  w->hpar[1] = (double)maxit;
  BP_CUDA_TRY(cudaMemcpyAsync(w->cgpar, w->hpar, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
  const int gvec = grid_for(n, NT);
  k_pcg_init<V><<<gvec, NT, 0, s>>>(w->R, reinterpret_cast<V*>(w->x), r, n, w->scal);
  mdsc_apply_launch<M, V, V, AMG>(m, J, r, z, s);
  k_pcg_rz<V><<<gvec, NT, 0, s>>>(w->kbase, 0, 0, r, z, n, w->scal, w->stop);
  BP_CUDA_TRY(cudaMemcpyAsync(p, z, n * sizeof(V), cudaMemcpyDeviceToDevice, s));
  BP_CUDA_TRY(cudaGetLastError());
  int k = 0;
  *status = 0;
  int* hk = reinterpret_cast<int*>(w->host + w->host_cap - 2);
  int stopflag = 0;
  if (loop) {
    BP_CUDA_TRY(cudaGraphLaunch(loop, s));
    BP_CUDA_TRY(cudaMemcpyAsync(hk, w->kbase, sizeof(int), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaMemcpyAsync(w->host + w->host_cap - 1, w->stop, sizeof(int), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    k = std::min(std::max(*hk, 0), maxit);
    std::memcpy(&stopflag, w->host + w->host_cap - 1, sizeof(int));
  } else {  // no conditional nodes: one iteration per host check
    while (!stopflag && k < maxit) {
      launch_mdsc_iteration<M, V, AMG>(m, J, s, cudaGraphConditionalHandle{}, 0);
      BP_CUDA_TRY(cudaGetLastError());
      BP_CUDA_TRY(cudaMemcpyAsync(w->host + w->host_cap - 1, w->stop, sizeof(int), cudaMemcpyDeviceToHost, s));
      BP_CUDA_TRY(cudaStreamSynchronize(s));
      std::memcpy(&stopflag, w->host + w->host_cap - 1, sizeof(int));
      ++k;
    }
  }
  BP_CUDA_TRY(cudaMemcpyAsync(w->host, w->scal, 3 * (size_t)(k + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  if (stopflag == 2) *status = 2;
  const double tol2 = eta * eta, rr0 = w->host[2];
  int taken = k;
  for (int j = 1; j <= k; ++j) {
    const double rr = w->host[3 * j + 2];
    if (!std::isfinite(rr)) {  // breakdown: Newton reports BP_ENAN at once
      taken = j;
      *status = 3;
      break;
    }
    if (rr <= tol2 * rr0) {
      taken = j;
      break;
    }
    if (w->host[3 * j + 2] == 0.0 && w->host[3 * j + 1] == 0.0) {
      taken = j - 1;
      break;
    }
  }
  *iters = taken;
  if (!std::isfinite(rr0)) *status = 3;
  return BP_OK;
}

double elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return 1e-3 * ms;
}

}  // namespace

void bp_solver_ws_free(bp_mesh* m) {
  if (!m->ws) return;
  if (m->ws->host) cudaFreeHost(m->ws->host);
  if (m->ws->hpar) cudaFreeHost(m->ws->hpar);
  for (void* g : m->ws->cg_exec)
    if (g) cudaGraphExecDestroy((cudaGraphExec_t)g);
  for (void* g : m->ws->cg_loop)
    if (g) cudaGraphExecDestroy((cudaGraphExec_t)g);
  for (void* g : m->ws->mdsc_loop)
    if (g) cudaGraphExecDestroy((cudaGraphExec_t)g);
  for (void* g : m->ws->amg_loop)
    if (g) cudaGraphExecDestroy((cudaGraphExec_t)g);
  delete static_cast<AmgHier*>(m->ws->amg);
  delete m->ws;  // device arrays are in m->allocations
  m->ws = nullptr;
}

int bp_nodal_surface_gradient(bp_mesh* m, double** acc, cudaStream_t s) {
  int rc = ensure_ws(m, s);
  if (rc) return rc;
  bp_solver_ws* w = m->ws;
  BP_CUDA_TRY(cudaMemsetAsync(w->sia, 0, 3 * (size_t)m->nv * sizeof(double), s));
  k_sia_accum<<<(m->ntri + 127) / 128, 128, 0, s>>>(m->xy, m->bed, m->thick, m->tri, m->ntri, w->sia, m->nv);
  BP_CUDA_TRY(cudaGetLastError());
  *acc = w->sia;
  return BP_OK;
}

int bp_norm2_host(bp_mesh* m, const double* v, cudaStream_t s, double* out) {
  int rc = ensure_ws(m, s);
  if (rc) return rc;
  double d;
  if ((rc = dot_host(m, v, v, m->ndof, s, &d))) return rc;
  *out = std::sqrt(d);
  return BP_OK;
}

int bp_learned_scratch(bp_mesh* m, uint16_t** X, float** Y, double** Usia, double** R, double** red) {
  int rc = ensure_ws(m, nullptr);
  if (rc) return rc;
  if (!m->mlp_X) {
    if ((rc = bp_alloc(m, &m->mlp_X, 16 * (size_t)m->nv))) return rc;
    if ((rc = bp_alloc(m, &m->mlp_Y, 32 * (size_t)m->nv))) return rc;
  }
  *X = m->mlp_X;
  *Y = m->mlp_Y;
  *Usia = m->ws->Ut;
  *R = m->ws->R;
  *red = m->ws->red;
  return BP_OK;
}

extern "C" int bp_spmv(bp_mesh* m, const void* J, int precision, const double* x, double* y, void* stream) {
  if (!m || !J || !x || !y || !bp_aligned16(x) || !bp_aligned16(y) || !bp_aligned16(J)) return BP_EINVAL;
  if (precision < BP_F64 || precision > BP_F64X2_DS) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = grid_for(m->ndof / 2 * TPR, NT);
  const int npairs = (int)(m->ndof / 2);
  if (!bp_values_f32(precision))
    k_spmv_pairs<double, double, true><<<grid, NT, 0, s>>>(m->rowptr, m->nbr_ptr, m->nbr_idx, m->nl,
                                                           (const double*)J, npairs, x, y, nullptr, nullptr,
                                                           nullptr, 0);
  else
    k_spmv_pairs<float, double, false><<<grid, NT, 0, s>>>(m->rowptr, m->nbr_ptr, m->nbr_idx, m->nl,
                                                           (const float*)J, npairs, x, y, nullptr, nullptr,
                                                           nullptr, 0);
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

extern "C" int bp_spmv_f32(bp_mesh* m, const float* J, const float* x, float* y, void* stream) {
  if (!m || !J || !x || !y || !bp_aligned16(x) || !bp_aligned16(y) || !bp_aligned16(J)) return BP_EINVAL;
  if (m->nl > MAXL) return BP_EUNSUP;
  bp_device_guard g(m->device);
  spmv_launch<float, float, false>(m, J, x, y, nullptr, nullptr, nullptr, 0, (cudaStream_t)stream);
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

extern "C" int bp_colprec_setup(bp_mesh* m, const void* J, int precision, void* stream) {
  if (!m || !J) return BP_EINVAL;
  if (precision < BP_F64 || precision > BP_F64X2_DS) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_ws(m, s);
  if (rc) return rc;
  return !bp_values_f32(precision) ? colprec_setup_t(m, (const double*)J, s)
                                    : colprec_setup_t(m, (const float*)J, s);
}

extern "C" int bp_colprec_apply(bp_mesh* m, const double* r, double* z, void* stream) {
  if (!m || !r || !z) return BP_EINVAL;
  if (!m->ws || !m->ws->has_prec) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (m->ws->prec_f32)
    k_colprec_apply<double, float><<<(m->nv + 127) / 128, 128, 0, s>>>(prec_of<float>(m), r, z);
  else
    k_colprec_apply<double, double><<<(m->nv + 127) / 128, 128, 0, s>>>(prec_of<double>(m), r, z);
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

extern "C" int bp_mdsc_setup(bp_mesh* m, const void* J, int precision, void* stream) {
  if (!m || !J) return BP_EINVAL;
  if (precision < BP_F64 || precision > BP_F64X2_DS) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_ws(m, s);
  if (rc) return rc;
  return !bp_values_f32(precision) ? mdsc_setup_t(m, (const double*)J, s) : mdsc_setup_t(m, (const float*)J, s);
}

extern "C" int bp_mdsc_apply(bp_mesh* m, const void* J, const double* r, double* z, void* stream) {
  if (!m || !J || !r || !z || !bp_aligned16(r) || !bp_aligned16(z) || !bp_aligned16(J)) return BP_EINVAL;
  if (!m->ws || !m->ws->has_mdsc) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (m->ws->mdsc_f32)
    mdsc_apply_launch<float, double, float>(m, (const float*)J, r, z, s);
  else
    mdsc_apply_launch<double, double, double>(m, (const double*)J, r, z, s);
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

extern "C" int bp_mdsc_amg_setup(bp_mesh* m, const void* J, int precision, void* stream) {
  if (!m || !J) return BP_EINVAL;
  if (precision < BP_F64 || precision > BP_F64X2_DS) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_ws(m, s);
  if (rc) return rc;
  rc = !bp_values_f32(precision) ? mdsc_amg_setup_t(m, (const double*)J, s)
                                  : mdsc_amg_setup_t(m, (const float*)J, s);
  if (rc) return rc;
  m->ws->has_amg = true;
  return BP_OK;
}

extern "C" int bp_mdsc_amg_apply(bp_mesh* m, const void* J, const double* r, double* z, void* stream) {
  if (!m || !J || !r || !z || !bp_aligned16(r) || !bp_aligned16(z) || !bp_aligned16(J)) return BP_EINVAL;
  if (!m->ws || !m->ws->has_mdsc || !m->ws->amg) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (m->ws->mdsc_f32)
    mdsc_apply_launch<float, double, float, true>(m, (const float*)J, r, z, s);
  else
    mdsc_apply_launch<double, double, double, true>(m, (const double*)J, r, z, s);
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

extern "C" int bp_mdsc_amg_levels(const bp_mesh* m, int32_t* sizes, int max_levels, int* nlevels) {
  if (!m || !nlevels || !m->ws || !m->ws->amg) return BP_EINVAL;
  const AmgHier* H = static_cast<const AmgHier*>(m->ws->amg);
  *nlevels = (int)H->lv.size();
  if (sizes)
    for (int k = 0; k < std::min(max_levels, (int)H->lv.size()); ++k) sizes[k] = H->lv[k].n;
  return BP_OK;
}

extern "C" int bp_mdsc_amg_aggregates(const bp_mesh* m, int level, int32_t* agg) {
  if (!m || !agg || !m->ws || !m->ws->amg) return BP_EINVAL;
  const AmgHier* H = static_cast<const AmgHier*>(m->ws->amg);
  if (level < 0 || level >= (int)H->agg.size()) return BP_EINVAL;
  std::copy(H->agg[level].begin(), H->agg[level].end(), agg);
  return BP_OK;
}

extern "C" int bp_energy(bp_mesh* m, const double* U, double* out, void* stream) {
  if (!m || !U || !out) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_ws(m, s);
  if (rc) return rc;
  return energy_host(m, U, s, out);
}

extern "C" int bp_energy_change(bp_mesh* m, const double* U, const double* D, double alpha, double* out,
                                void* stream) {
  if (!m || !U || !D || !out) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_ws(m, s);
  if (rc) return rc;
  return energy_change_host<double, double>(m, U, D, alpha, s, out);
}

extern "C" int bp_energy_change_ex(bp_mesh* m, const double* U, const double* D, double alpha, int precision,
                                   double* out, void* stream) {
  if (!m || !U || !D || !out) return BP_EINVAL;
  if (precision != BP_F64 && precision != BP_F64X2_DS && precision != BP_F32) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_ws(m, s);
  if (rc) return rc;
  if (precision == BP_F64X2_DS) return energy_change_host<f64x2, double>(m, U, D, alpha, s, out);
  if (precision == BP_F32) return energy_change_host<float, double>(m, U, D, alpha, s, out);
  return energy_change_host<double, double>(m, U, D, alpha, s, out);
}

extern "C" int bp_initial_guess(bp_mesh* m, int kind, double* U, void* stream) {
  if (!m || !U) return BP_EINVAL;
  if (kind != BP_GUESS_ZERO && kind != BP_GUESS_SIA) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (kind == BP_GUESS_ZERO) {
    BP_CUDA_TRY(cudaMemsetAsync(U, 0, m->ndof * sizeof(double), s));
    return BP_OK;
  }
  int rc = ensure_ws(m, s);
  if (rc) return rc;
  bp_solver_ws* w = m->ws;
  BP_CUDA_TRY(cudaMemsetAsync(w->sia, 0, 3 * (size_t)m->nv * sizeof(double), s));
  k_sia_accum<<<(m->ntri + 127) / 128, 128, 0, s>>>(m->xy, m->bed, m->thick, m->tri, m->ntri, w->sia, m->nv);
  k_sia_fill<<<(m->nv + 127) / 128, 128, 0, s>>>(w->sia, m->bed, m->thick, m->beta, m->sigma, m->nv, m->nl, m->p.A,
                                                 m->p.rho * m->p.g, U);
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

extern "C" void bp_solve_opts_default(bp_solve_opts* o) {
  if (!o) return;
  o->rtol = 1e-8;
  o->max_newton = 50;
  o->max_krylov = 1000;
  o->eta_max = 0.1;
  o->precision = BP_F64;
  o->krylov = BP_KRYLOV_CG;
  o->line_search = 1;
  o->check_every = 8;
  o->picard_rtol = 0.0;
  o->value32_rtol = 0.0;
  o->device_loop = 1;
  o->preconditioner = BP_PREC_COLUMN;
  o->gmres_restart = 50;
}

extern "C" int bp_newton_solve(bp_mesh* m, double* U, const bp_solve_opts* opts, bp_solve_report* rep,
                               void* stream) {
  if (!m || !U || !opts || !rep || !bp_aligned16(U)) return BP_EINVAL;
  const bp_solve_opts o = *opts;
  if (o.line_search < 0 || o.line_search > BP_LS_QUADRATIC) return BP_EINVAL;
  if (!(o.picard_rtol >= 0) || !(o.value32_rtol >= 0)) return BP_EINVAL;
  if (o.value32_rtol > 0 && o.value32_rtol < o.rtol) return BP_EINVAL;  // an FP32 residual could pass the test
  if (o.picard_rtol > 0 && o.precision == BP_F64X2_DS) return BP_EUNSUP;   // no paired-lane Picard matrix
  if ((o.device_loop != 0 && o.device_loop != 1) ||
      (o.preconditioner != BP_PREC_COLUMN && o.preconditioner != BP_PREC_MDSC &&
       o.preconditioner != BP_PREC_MDSC_AMG))
    return BP_EINVAL;
  if (!(o.rtol > 0) || o.max_newton < 0 || o.max_newton > 64 || o.max_krylov < 1 || o.check_every < 1 ||
      (o.precision != BP_F64 && o.precision != BP_F32 && o.precision != BP_F32_DS && o.precision != BP_F64X2_DS) ||
      (o.krylov != BP_KRYLOV_CG && o.krylov != BP_KRYLOV_GMRES) || !(o.eta_max > 0))
    return BP_EINVAL;
  if (o.krylov == BP_KRYLOV_GMRES &&
      (o.gmres_restart < 1 || o.gmres_restart > GMRES_MAX_RESTART || o.preconditioner != BP_PREC_COLUMN))
    return o.preconditioner != BP_PREC_COLUMN ? BP_EUNSUP : BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_ws(m, s);
  if (rc) return rc;
  if ((rc = ensure_jac(m))) return rc;
  bp_solver_ws* w = m->ws;
  std::memset(rep, 0, sizeof(*rep));
  cudaEvent_t ev[10];
  for (auto& e : ev) BP_CUDA_TRY(cudaEventCreate(&e));
  struct EvFree {
    cudaEvent_t* e;
    ~EvFree() {
      for (int i = 0; i < 10; ++i) cudaEventDestroy(e[i]);
    }
  } evfree{ev};
  BP_CUDA_TRY(cudaEventRecord(ev[0], s));
  double fref;
  if ((rc = dot_host(m, m->load, m->load, m->ndof, s, &fref))) return rc;
  fref = std::sqrt(fref);  // ||F(0)||: at U = 0 the residual is the driving-stress load
  rep->fnorm_ref = fref;
  const bool f32 = bp_values_f32(o.precision);  // FP32 Jacobian values and Krylov vectors
  const double eta_floor = f32 ? 1e-5 : 1e-10;
  double eta = o.eta_max, fprev = 0.0;
  int status = BP_ENOCONV;
  bool residual_first = false;  // the previous step is expected to have reached the tolerance
  for (int k = 0;; ++k) {
    // assemble J and F at U
    BP_CUDA_TRY(cudaEventRecord(ev[1], s));
    // Picard (fixed-viscosity) matrix while far from the solution, if asked for: the residual of the
    // previous step decides (the first step uses the initial residual, unknown yet: Picard if on)
    const bool picard = o.picard_rtol > 0 && (k == 0 || rep->history[k - 1] > o.picard_rtol);
    // FP32 value path (inexact residual) while the previous residual was above value32_rtol; a
    // residual that comes out below it is assembled again with the FP64 value path before it is
    // tested or used, so that convergence is always judged on the FP64 residual (value32_rtol is
    // 0 or at least rtol: every residual that can pass the test is an FP64 one)
    bool v32 = f32 && o.value32_rtol > 0 && (k == 0 || rep->history[k - 1] > o.value32_rtol);
    const double v32_exit = o.value32_rtol * fref;
    double fn;
    bool need_j = true;
    if (residual_first) {
      // test the FP64 residual alone first (about a fifth of the cost of the FP64 or paired-lane
      // Jacobian with it); J and R are assembled together only if the test fails
      if ((rc = bp_assemble_residual(m, U, w->R, s))) return rc;
      if ((rc = dot_host(m, w->R, w->R, m->ndof, s, &fn))) return rc;
      fn = std::sqrt(fn);
      need_j = !(std::isfinite(fn) && fn <= o.rtol * fref);
    }
    while (need_j) {
      if ((rc = bp_assemble_jacobian_ex(m, U, w->R, w->J, v32 ? BP_F32_ALL : o.precision, BP_SCATTER_ATOMIC,
                                        BP_JAC_FACTORED, picard ? 1 : 0, s)))
        return rc;
      if ((rc = dot_host(m, w->R, w->R, m->ndof, s, &fn))) return rc;
      fn = std::sqrt(fn);
      if (v32 && std::isfinite(fn) && fn <= v32_exit) {
        v32 = false;
        continue;
      }
      break;
    }
    if (v32) ++rep->value32_steps;
    BP_CUDA_TRY(cudaEventRecord(ev[2], s));
    BP_CUDA_TRY(cudaEventSynchronize(ev[2]));
    rep->t_assemble += elapsed(ev[1], ev[2]);
    if (!std::isfinite(fn)) {
      status = BP_ENAN;
      break;
    }
    if (k == 0) rep->fnorm_initial = fn;
    rep->history[k] = fn / fref;
    rep->fnorm_final = fn;
    rep->newton_iters = k;
    if (fn <= o.rtol * fref) {
      status = BP_OK;
      rep->converged = 1;
      break;
    }
    if (k >= o.max_newton) break;
    // forcing term (Eisenstat-Walker choice 2), not below what the final tolerance needs
    if (k > 0) {
      double e = 0.9 * (fn / fprev) * (fn / fprev);
      const double safe = 0.9 * eta * eta;
      if (safe > 0.1) e = std::max(e, safe);
      eta = std::min(e, o.eta_max);
    }
    eta = std::max(eta, 0.5 * o.rtol * fref / fn);
    eta = std::max(eta, eta_floor);
    fprev = fn;
    // preconditioner + Krylov
    const bool amg = o.preconditioner == BP_PREC_MDSC_AMG;
    const bool mdsc = o.preconditioner == BP_PREC_MDSC;
    BP_CUDA_TRY(cudaEventRecord(ev[3], s));
    if (amg)
      rc = f32 ? mdsc_amg_setup_t(m, reinterpret_cast<const float*>(w->J), s) : mdsc_amg_setup_t(m, w->J, s);
    else if (mdsc)
      rc = f32 ? mdsc_setup_t(m, reinterpret_cast<const float*>(w->J), s) : mdsc_setup_t(m, w->J, s);
    else
      rc = f32 ? colprec_setup_t(m, reinterpret_cast<const float*>(w->J), s) : colprec_setup_t(m, w->J, s);
    if (rc) return rc;
    BP_CUDA_TRY(cudaEventRecord(ev[4], s));
    int its = 0, kst = 0;
    const bool gmres = o.krylov == BP_KRYLOV_GMRES;
    if (gmres && f32)
      rc = gmres_solve<float, float>(m, reinterpret_cast<const float*>(w->J), eta, o.max_krylov, o.gmres_restart, s,
                                     &its, &kst);
    else if (gmres)
      rc = gmres_solve<double, double>(m, w->J, eta, o.max_krylov, o.gmres_restart, s, &its, &kst);
    else if (amg && f32)
      rc = mdsc_cg_solve<float, float, true>(m, reinterpret_cast<const float*>(w->J), eta, o.max_krylov,
                                             o.device_loop != 0, s, &its, &kst);
    else if (amg)
      rc = mdsc_cg_solve<double, double, true>(m, w->J, eta, o.max_krylov, o.device_loop != 0, s, &its, &kst);
    else if (mdsc && f32)
      rc = mdsc_cg_solve<float, float>(m, reinterpret_cast<const float*>(w->J), eta, o.max_krylov,
                                       o.device_loop != 0, s, &its, &kst);
    else if (mdsc)
      rc = mdsc_cg_solve<double, double>(m, w->J, eta, o.max_krylov, o.device_loop != 0, s, &its, &kst);
    else if (f32)
      rc = cg_solve<float, float>(m, reinterpret_cast<const float*>(w->J), eta, o.max_krylov, o.check_every,
                                  o.device_loop != 0, s, &its, &kst);
    else
      rc = cg_solve<double, double>(m, w->J, eta, o.max_krylov, o.check_every, o.device_loop != 0, s, &its, &kst);
    if (rc) return rc;
    BP_CUDA_TRY(cudaEventRecord(ev[5], s));
    BP_CUDA_TRY(cudaEventSynchronize(ev[5]));
    rep->t_precond += elapsed(ev[3], ev[4]);
    rep->t_krylov += elapsed(ev[4], ev[5]);
    rep->krylov_per_newton[k] = its;
    rep->krylov_iters += its;
    if (kst == 3) {
      status = BP_ENAN;
      break;
    }
    // line search on the energy
    BP_CUDA_TRY(cudaEventRecord(ev[6], s));
    double slope;
    if (f32)
      rc = dot_host(m, w->R, reinterpret_cast<const float*>(w->x), m->ndof, s, &slope);
    else
      rc = dot_host(m, w->R, w->x, m->ndof, s, &slope);
    if (rc) return rc;
    double alpha = 1.0;
    // Once the residual falls by 10x per full step Newton is in its quadratic regime: take the full
    // step without evaluating the energy (the Armijo test is then always met).
    const bool quadratic = k > 0 && rep->alpha[k - 1] == 1.0 && fn <= 0.1 * rep->history[k - 1] * fref;
    if (o.line_search && slope < 0.0 && !quadratic) {
      // Armijo on the energy: Pi(U + alpha delta) - Pi(U) <= c alpha F . delta.  Trial steps:
      // BP_LS_HALVING alpha = 1, 1/2, ..., 2^-10; BP_LS_QUADRATIC the minimiser of the quadratic
      // through the energy change at 0 (value 0, slope F . delta) and at the rejected alpha,
      // kept within [0.1, 0.9] of that alpha (backtracking by interpolation).
      const double c = 1e-4;
      for (int h = 0; h <= 10; ++h) {
        double dE;
        if (f32)
          rc = energy_change_host<float, float>(m, U, reinterpret_cast<const float*>(w->x), alpha, s, &dE);
        else  // FP64-accurate: the per-point work in pairs on the FP32 pipe (2.5x faster than FP64)
          rc = energy_change_host<f64x2, double>(m, U, w->x, alpha, s, &dE);
        if (rc) return rc;
        if (dE <= c * alpha * slope || h == 10) break;
        if (o.line_search == BP_LS_QUADRATIC) {
          const double curv = dE - slope * alpha;  // > 0 here (Armijo failed)
          double an = -slope * alpha * alpha / (2.0 * curv);
          if (!std::isfinite(an)) an = 0.5 * alpha;
          alpha = std::min(std::max(an, 0.1 * alpha), 0.9 * alpha);
        } else {
          alpha *= 0.5;
        }
      }
    }
    if (f32)
      k_axpy_to<float><<<grid_for(m->ndof, NT), NT, 0, s>>>(U, reinterpret_cast<const float*>(w->x), alpha, m->ndof,
                                                           U);
    else
      k_axpy_to<double><<<grid_for(m->ndof, NT), NT, 0, s>>>(U, w->x, alpha, m->ndof, U);
    BP_CUDA_TRY(cudaGetLastError());
    BP_CUDA_TRY(cudaEventRecord(ev[7], s));
    BP_CUDA_TRY(cudaEventSynchronize(ev[7]));
    rep->t_linesearch += elapsed(ev[6], ev[7]);
    rep->alpha[k] = alpha;
    // A full step whose linear residual eta ||F|| is within the tolerance is expected to reach it:
    // the next residual is then tested before any Jacobian is assembled (the FP32 kinds assemble J
    // with R at about the cost of R alone and keep assembling both).
    residual_first = !f32 && alpha == 1.0 && eta * fn <= o.rtol * fref;
  }
  BP_CUDA_TRY(cudaEventRecord(ev[8], s));
  BP_CUDA_TRY(cudaEventSynchronize(ev[8]));
  rep->t_total = elapsed(ev[0], ev[8]);
  return status;
}
