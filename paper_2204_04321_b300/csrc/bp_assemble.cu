// Entry points of the fused residual / Jacobian assembly (the kernel body is in bp_column.cuh).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "bp_column.cuh"

namespace {

#ifndef BP_ASM_MIN_BLOCKS
#define BP_ASM_MIN_BLOCKS 1  // minimum resident blocks of 128 threads per SM asked of the register allocator
#endif

#ifndef BP_ASM_MIN_BLOCKS_F32
#define BP_ASM_MIN_BLOCKS_F32 1
#endif
#ifndef BP_ASM_MIN_BLOCKS_F32ALL
#define BP_ASM_MIN_BLOCKS_F32ALL 1
#endif
template <class TL, class TV>
constexpr int min_blocks() {
  return std::is_same<TV, float>::value ? BP_ASM_MIN_BLOCKS_F32ALL
                                        : (std::is_same<TL, float>::value ? BP_ASM_MIN_BLOCKS_F32 : BP_ASM_MIN_BLOCKS);
}

template <int MODE, class TL, bool ATOMIC, bool PICARD = false, class TV = double>
__global__ void __launch_bounds__(128, min_blocks<TL, TV>()) k_assemble(const AsmArgs A) {
  int c, l0, l1;
  if (!column_segment(A, blockIdx.x * blockDim.x + threadIdx.x, c, l0, l1)) return;
  const int t = A.tri_list ? A.tri_list[c] : c;
  if constexpr (MODE == MODE_FACT) {  // in-plane coefficients (24 lanes) and carried block (21)
    __shared__ __align__(16) unsigned char sraw[45 * 128 * sizeof(TL)];
    assemble_column<MODE, TL, ATOMIC, PICARD, TV, true>(A, t, reinterpret_cast<TL*>(sraw) + threadIdx.x, l0, l1);
  } else {
    assemble_column<MODE, TL, ATOMIC, PICARD, TV>(A, t, nullptr, l0, l1);
  }
}

// Paired-FP32 lanes with the staged rank-one part (blocks of 64: 81 lanes per thread in shared memory,
// the in-plane table, the carried block and the 6 points' rank-one factors).
constexpr int STAGED_TPB = 64;
template <bool ATOMIC, class TV = double>
__global__ void __launch_bounds__(STAGED_TPB) k_assemble_staged(const AsmArgs A) {
  int c, l0, l1;
  if (!column_segment(A, blockIdx.x * blockDim.x + threadIdx.x, c, l0, l1)) return;
  const int t = A.tri_list ? A.tri_list[c] : c;
  __shared__ __align__(16) unsigned char sraw[81 * STAGED_TPB * sizeof(f64x2)];
  assemble_column<MODE_FACT, f64x2, ATOMIC, false, TV, true, true>(A, t, reinterpret_cast<f64x2*>(sraw) + threadIdx.x,
                                                                  l0, l1);
}

// Tail split of an atomic launch of `count` columns: when the columns fill more than one wave of
// resident threads but not a whole number of waves, the columns of the last partial wave are taken
// in layer segments (at least 2 layers each, at most 4 per column), so that the last wave is made
// of short units and the SMs finish together.  Threads to launch are returned.
int tail_split(AsmArgs& a, int resident_threads) {
  a.nwhole = a.count;
  a.nseg = 0;
  const int nseg = std::min(4, a.L / 2);
  if (nseg < 2 || resident_threads <= 0 || a.count <= resident_threads) return a.count;
  const int rem = a.count % resident_threads;
  if (rem == 0) return a.count;
  a.nwhole = a.count - rem;
  a.nseg = nseg;
  return a.nwhole + rem * nseg;
}

// resident threads per device of a kernel launched with `tpb` threads per block
template <class K>
int resident_threads(K kernel, int tpb) {
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, tpb, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nsm * per_sm * tpb;
}

AsmArgs make_args(const bp_mesh* m, const double* U, double* R, void* J) {
  AsmArgs a{};
  a.xy = m->xy;
  a.bed = m->bed;
  a.thick = m->thick;
  a.sigma = m->sigma;
  a.tri = m->tri;
  a.slots = m->slots;
  a.basal = m->basal;
  a.vstart = m->vstart;
  a.vdeg = m->vdeg;
  a.tri_list = nullptr;
  a.count = m->ntri;
  a.L = m->nl;
  a.cA = m->cA;
  a.Bn = m->Bnode;
  a.delta = m->p.delta;
  a.U = U;
  a.R = R;
  a.J = J;
  return a;
}

template <int MODE, class TL, bool PICARD = false, class TV = double>
int launch(const bp_mesh* m, AsmArgs a, int scatter, cudaStream_t s) {
  constexpr int TPB = 128;
  if (scatter == BP_SCATTER_COLOR) {
    for (int c = 0; c < m->ncolors; ++c) {
      a.tri_list = m->color_tris + m->color_off[c];
      a.count = m->color_off[c + 1] - m->color_off[c];
      k_assemble<MODE, TL, false, PICARD, TV><<<(a.count + TPB - 1) / TPB, TPB, 0, s>>>(a);
    }
  } else {
    static const int resident = resident_threads(k_assemble<MODE, TL, true, PICARD, TV>, TPB);
    const int threads = tail_split(a, resident);
    k_assemble<MODE, TL, true, PICARD, TV><<<(threads + TPB - 1) / TPB, TPB, 0, s>>>(a);
  }
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

template <class TV = double>
int launch_staged(const bp_mesh* m, AsmArgs a, int scatter, cudaStream_t s) {
  if (scatter == BP_SCATTER_COLOR) {
    for (int c = 0; c < m->ncolors; ++c) {
      a.tri_list = m->color_tris + m->color_off[c];
      a.count = m->color_off[c + 1] - m->color_off[c];
      k_assemble_staged<false, TV><<<(a.count + STAGED_TPB - 1) / STAGED_TPB, STAGED_TPB, 0, s>>>(a);
    }
  } else {
    static const int resident = resident_threads(k_assemble_staged<true, TV>, STAGED_TPB);
    const int threads = tail_split(a, resident);
    k_assemble_staged<true, TV><<<(threads + STAGED_TPB - 1) / STAGED_TPB, STAGED_TPB, 0, s>>>(a);
  }
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

// Argument checks shared by the Jacobian entry points.
int check_jacobian_args(int precision, int scatter, int method) {
  if (precision < BP_F64 || precision > BP_F64X2_DS) return BP_EINVAL;
  if (scatter < BP_SCATTER_AUTO || scatter > BP_SCATTER_COLOR) return BP_EINVAL;
  if (method < BP_JAC_AUTO || method > BP_JAC_FACTORED) return BP_EINVAL;
  if (precision != BP_F64 && precision != BP_F32 && method == BP_JAC_DUAL) return BP_EUNSUP;
  return BP_OK;
}

size_t jacobian_value_bytes(int precision) {
  return (precision == BP_F32 || precision == BP_F32_ALL || precision == BP_F32_DS) ? sizeof(float) : sizeof(double);
}

// Launch of the Jacobian kernel for checked arguments (scatter and method resolved).
int launch_jacobian(const bp_mesh* m, const AsmArgs& a, int precision, int scatter, int method, cudaStream_t s) {
  switch (precision) {
    case BP_F64X2:
      return launch_staged(m, a, scatter, s);
    case BP_F64X2_DS:
      return launch_staged<f64x2>(m, a, scatter, s);
    case BP_F32_DS:
      return launch<MODE_FACT, float, false, f64x2>(m, a, scatter, s);
    case BP_F32_ALL:
      return launch<MODE_FACT, float, false, float>(m, a, scatter, s);
    case BP_F64:
      return method == BP_JAC_DUAL ? launch<MODE_DUAL, double>(m, a, scatter, s)
                                   : launch<MODE_FACT, double>(m, a, scatter, s);
    default:
      return method == BP_JAC_DUAL ? launch<MODE_DUAL, float>(m, a, scatter, s)
                                   : launch<MODE_FACT, float>(m, a, scatter, s);
  }
}

}  // namespace

extern "C" int bp_assemble_residual(bp_mesh* m, const double* U, double* R, void* stream) {
  if (!m || !U || !R || !bp_aligned16(U)) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  BP_CUDA_TRY(cudaMemcpyAsync(R, m->load, m->ndof * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return launch<MODE_RES, double>(m, make_args(m, U, R, nullptr), BP_SCATTER_ATOMIC, s);
}

int bp_assemble_jacobian_ex(bp_mesh* m, const double* U, double* R, void* J, int precision, int scatter, int method,
                            int picard, void* stream) {
  if (!m || !U || !J || !bp_aligned16(U) || !bp_aligned8(J)) return BP_EINVAL;
  int rc0 = check_jacobian_args(precision, scatter, method);
  if (rc0) return rc0;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (scatter == BP_SCATTER_AUTO) scatter = BP_SCATTER_ATOMIC;
  if (method == BP_JAC_AUTO) method = BP_JAC_FACTORED;
  double* Rw = R;
  if (!Rw) {  // residual not wanted: assemble it into mesh-owned scratch (allocated once)
    if (!m->rscratch) {
      int rc = bp_alloc(m, &m->rscratch, m->ndof);
      if (rc) return rc;
    }
    Rw = m->rscratch;
  }
  BP_CUDA_TRY(cudaMemcpyAsync(Rw, m->load, m->ndof * sizeof(double), cudaMemcpyDeviceToDevice, s));
  BP_CUDA_TRY(cudaMemsetAsync(J, 0, m->nnz * jacobian_value_bytes(precision), s));
  const AsmArgs a = make_args(m, U, Rw, J);
  if (picard) {  // fixed-viscosity matrix (Newton solver's Picard steps): factored method, FP64 or FP32
    if (method != BP_JAC_FACTORED || precision == BP_F64X2 || precision == BP_F64X2_DS) return BP_EUNSUP;
    switch (precision) {
      case BP_F64:
        return launch<MODE_FACT, double, true>(m, a, scatter, s);
      case BP_F32_ALL:
        return launch<MODE_FACT, float, true, float>(m, a, scatter, s);
      case BP_F32_DS:
        return launch<MODE_FACT, float, true, f64x2>(m, a, scatter, s);
      default:
        return launch<MODE_FACT, float, true>(m, a, scatter, s);
    }
  }
  return launch_jacobian(m, a, precision, scatter, method, s);
}

extern "C" int bp_assemble_jacobian(bp_mesh* m, const double* U, double* R, void* J, int precision,
                                    int scatter, int method, void* stream) {
  return bp_assemble_jacobian_ex(m, U, R, J, precision, scatter, method, 0, stream);
}

// ---------------------------------------------------------------------------------------------
// Allocation-free Jacobian assembly.
//
// bp_assemble_jacobian with R == NULL allocates a residual scratch (ndof doubles) in the mesh
// object on its first call.  Callers that may not allocate device memory once they are running
// -- code under a fixed device-memory budget, or inside a framework whose allocator owns all
// device memory and forbids direct cudaMalloc -- use bp_assemble_jacobian_noalloc instead: its
// residual scratch is this file-scope device array, so the call itself never allocates.
//
// The array is part of the library's module image: every GPU on which the library's module is
// loaded holds BP_NOALLOC_MAX_NDOF doubles (8 MiB) of it until the process exits.  In host code
// the name g_noalloc_residual is only a host-side stand-in; the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the entry point's first
// call there, and kept for the life of the process (a cudaDeviceReset, which may reload the
// module at another address, ends the entry point's use on that device).
static __device__ __align__(256) double g_noalloc_residual[BP_NOALLOC_MAX_NDOF];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_residual on `device` (current); looked up once per device.
int noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return BP_EUNSUP;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    BP_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_residual));
    g_noalloc_ptr[device] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[device];
  return BP_OK;
}
}  // namespace

extern "C" int bp_assemble_jacobian_noalloc(bp_mesh* m, const double* U, void* J, int precision,
                                            int scatter, int method, void* stream) {
  if (!m || !U || !J || !bp_aligned16(U) || !bp_aligned8(J)) return BP_EINVAL;
  int rc0 = check_jacobian_args(precision, scatter, method);
  if (rc0) return rc0;
  if (m->ndof > BP_NOALLOC_MAX_NDOF) return BP_ESIZE;
  bp_device_guard g(m->device);
  double* Rw = nullptr;
  int rc = noalloc_scratch(m->device, &Rw);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (scatter == BP_SCATTER_AUTO) scatter = BP_SCATTER_ATOMIC;
  if (method == BP_JAC_AUTO) method = BP_JAC_FACTORED;
  // the scratch keeps the previous call's residual: start it again from the memoised load
  BP_CUDA_TRY(cudaMemcpyAsync(Rw, m->load, m->ndof * sizeof(double), cudaMemcpyDeviceToDevice, s));
  BP_CUDA_TRY(cudaMemsetAsync(J, 0, m->nnz * jacobian_value_bytes(precision), s));
  return launch_jacobian(m, make_args(m, U, Rw, J), precision, scatter, method, s);
}
