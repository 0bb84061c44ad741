// Ensemble assembly: the residuals and Jacobians of many uneven meshes in one persistent launch.
//
// The work is a list of tiles (member, first column, column count).  A grid sized to be fully
// resident pulls tiles from an atomic counter -- dynamic scheduling absorbs the members' different
// layer counts (a column's cost grows with L) -- and every thread assembles one column with the
// same per-column body as the single-mesh kernel.  There is no waiting on other blocks: the queue
// is an atomic counter only.  The coloured variant runs one such launch per colour, each over all
// members' triangles of that colour, with plain read-modify-write scatter.  A project-written
// autotuner times columns-per-block x scatter candidates and the winner is captured in a CUDA graph.
#include <algorithm>
#include <cstring>
#include <vector>

#include "bp_column.cuh"

namespace {

struct Tile {
  int member, first, count, pad;
};

struct InitItem {
  double* R;
  const double* load;
  int64_t ndof;
  void* J;
  int64_t jbytes;
};

constexpr int kMaxCounters = 128;

__global__ void k_ens_init(const InitItem* __restrict__ items, int count, int* __restrict__ counters) {
  if (blockIdx.x == 0 && threadIdx.x < kMaxCounters) counters[threadIdx.x] = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int m = 0; m < count; ++m) {
    const InitItem it = items[m];
    for (int64_t i = t0; i < it.ndof; i += stride) it.R[i] = it.load[i];
    const int64_t n16 = bp_aligned16(it.J) ? it.jbytes / 16 : 0;
    uint4* J16 = reinterpret_cast<uint4*>(it.J);
    for (int64_t i = t0; i < n16; i += stride) J16[i] = make_uint4(0, 0, 0, 0);
    const int64_t n4 = it.jbytes / 4;
    for (int64_t i = 4 * n16 + t0; i < n4; i += stride) reinterpret_cast<uint32_t*>(it.J)[i] = 0u;
  }
}

// dynamic shared memory of a block: the per-column in-plane coefficients and the carried element
// block, 45 lanes per thread
template <class TL>
size_t ens_smem(int cpb) {
  return 45 * (size_t)cpb * sizeof(TL);
}

template <class TL, bool ATOMIC>
__global__ void __launch_bounds__(256) k_ensemble(const AsmArgs* __restrict__ args, const Tile* __restrict__ tiles,
                                                  int ntiles, int* counter) {
  extern __shared__ __align__(16) unsigned char ens_sbl[];
  __shared__ int s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int k = s_tile;
    __syncthreads();
    if (k >= ntiles) return;
    const Tile T = tiles[k];
    if ((int)threadIdx.x < T.count) {
      const AsmArgs a = args[T.member];
      const int idx = T.first + threadIdx.x;
      assemble_column<MODE_FACT, TL, ATOMIC, false, double, true>(a, a.tri_list ? a.tri_list[idx] : idx,
                                                                  reinterpret_cast<TL*>(ens_sbl) + threadIdx.x);
    }
  }
}

struct Candidate {
  int cpb = 128, colored = 0;
  Tile* tiles = nullptr;                // device
  std::vector<int> color_off;           // colored: tiles of colour c are [color_off[c], color_off[c+1])
  int ntiles = 0, grid = 0;
};

}  // namespace

struct bp_ensemble {
  int device = 0, count = 0, precision = BP_F64;
  std::vector<bp_mesh*> members;
  AsmArgs* args_atomic = nullptr;  // device [count], tri_list = NULL
  AsmArgs* args_color = nullptr;   // device [count], tri_list = the member's colour-grouped triangles
  InitItem* init = nullptr;        // device [count]
  int* counters = nullptr;         // device [kMaxCounters]
  std::vector<Candidate> cands;
  int chosen = -1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> allocs;
};

namespace {

template <class T>
int ens_alloc(bp_ensemble* e, T** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return BP_ENOMEM;
  }
  e->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return BP_OK;
}

int build_candidate(bp_ensemble* e, int cpb, int colored, cudaStream_t s, Candidate* c) {
  c->cpb = cpb;
  c->colored = colored;
  std::vector<Tile> tiles;
  // members with more layers first: their columns cost more (longest-processing-time order)
  std::vector<int> order(e->count);
  for (int i = 0; i < e->count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return e->members[a]->nl > e->members[b]->nl; });
  if (!colored) {
    for (int m : order) {
      const int n = e->members[m]->ntri;
      for (int f = 0; f < n; f += cpb) tiles.push_back(Tile{m, f, std::min(cpb, n - f), 0});
    }
    c->color_off = {0, (int)tiles.size()};
  } else {
    int maxc = 0;
    for (auto* mm : e->members) maxc = std::max(maxc, mm->ncolors);
    if (maxc + 1 > kMaxCounters) return BP_EUNSUP;
    c->color_off.assign(1, 0);
    for (int col = 0; col < maxc; ++col) {
      for (int m : order) {
        const bp_mesh* mm = e->members[m];
        if (col >= mm->ncolors) continue;
        const int b = mm->color_off[col], en = mm->color_off[col + 1];
        for (int f = b; f < en; f += cpb) tiles.push_back(Tile{m, f, std::min(cpb, en - f), 0});
      }
      c->color_off.push_back((int)tiles.size());
    }
  }
  c->ntiles = (int)tiles.size();
  int rc = ens_alloc(e, &c->tiles, tiles.size());
  if (rc) return rc;
  BP_CUDA_TRY(cudaMemcpyAsync(c->tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, s));
  int per_sm = 0, nsm = 0;
  if (e->precision == BP_F64)
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm,
                                                              colored ? k_ensemble<double, false> : k_ensemble<double, true>,
                                                              cpb, ens_smem<double>(cpb)));
  else
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm,
                                                              colored ? k_ensemble<float, false> : k_ensemble<float, true>,
                                                              cpb, ens_smem<float>(cpb)));
  BP_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, e->device));
  c->grid = std::max(1, per_sm) * nsm;
  return BP_OK;
}

int launch_candidate(bp_ensemble* e, const Candidate& c, cudaStream_t s) {
  k_ens_init<<<148 * 4, 256, 0, s>>>(e->init, e->count, e->counters);
  const int ncol = (int)c.color_off.size() - 1;
  for (int k = 0; k < ncol; ++k) {
    const Tile* tl = c.tiles + c.color_off[k];
    const int nt = c.color_off[k + 1] - c.color_off[k];
    if (nt == 0) continue;
    const int grid = std::min(c.grid, nt);
    int* ctr = e->counters + 1 + k;
    if (e->precision == BP_F64) {
      const size_t sm = ens_smem<double>(c.cpb);
      if (c.colored)
        k_ensemble<double, false><<<grid, c.cpb, sm, s>>>(e->args_color, tl, nt, ctr);
      else
        k_ensemble<double, true><<<grid, c.cpb, sm, s>>>(e->args_atomic, tl, nt, ctr);
    } else {
      const size_t sm = ens_smem<float>(c.cpb);
      if (c.colored)
        k_ensemble<float, false><<<grid, c.cpb, sm, s>>>(e->args_color, tl, nt, ctr);
      else
        k_ensemble<float, true><<<grid, c.cpb, sm, s>>>(e->args_atomic, tl, nt, ctr);
    }
  }
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

}  // namespace

extern "C" void bp_ensemble_free(bp_ensemble* e) {
  if (!e) return;
  bp_device_guard g(e->device);
  cudaDeviceSynchronize();
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  for (void* p : e->allocs) cudaFree(p);
  delete e;
}

extern "C" int bp_ensemble_create(bp_mesh* const* members, int count, const double* const* U, double* const* R,
                                  void* const* J, int precision, void* stream, bp_ensemble** out) {
  if (!out) return BP_EINVAL;
  *out = nullptr;
  if (!members || !U || !R || !J || count < 1) return BP_EINVAL;
  if (precision != BP_F64 && precision != BP_F32) return BP_EINVAL;
  int dev = 0;
  BP_CUDA_TRY(cudaGetDevice(&dev));
  for (int i = 0; i < count; ++i)
    if (!members[i] || !U[i] || !R[i] || !J[i] || members[i]->device != dev || !bp_aligned16(U[i]) ||
        !bp_aligned8(J[i]))
      return BP_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  auto* e = new bp_ensemble();
  e->device = dev;
  e->count = count;
  e->precision = precision;
  e->members.assign(members, members + count);
  std::vector<AsmArgs> aa(count), ac(count);
  std::vector<InitItem> it(count);
  for (int i = 0; i < count; ++i) {
    const bp_mesh* m = members[i];
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
    a.U = U[i];
    a.R = R[i];
    a.J = J[i];
    aa[i] = a;
    a.tri_list = m->color_tris;
    ac[i] = a;
    it[i] = InitItem{R[i], m->load, m->ndof, J[i],
                     m->nnz * (int64_t)(precision == BP_F64 ? sizeof(double) : sizeof(float))};
  }
  int rc;
  auto fail = [&](int code) {
    bp_ensemble_free(e);
    return code;
  };
  if ((rc = ens_alloc(e, &e->args_atomic, count)) || (rc = ens_alloc(e, &e->args_color, count)) ||
      (rc = ens_alloc(e, &e->init, count)) || (rc = ens_alloc(e, &e->counters, kMaxCounters)))
    return fail(rc);
  if (cudaMemcpyAsync(e->args_atomic, aa.data(), count * sizeof(AsmArgs), cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(e->args_color, ac.data(), count * sizeof(AsmArgs), cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(e->init, it.data(), count * sizeof(InitItem), cudaMemcpyHostToDevice, s))
    return fail(BP_ECUDA);
  // 256 columns per block need 90 KiB of dynamic shared memory: opt in
  if (cudaFuncSetAttribute(k_ensemble<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ens_smem<double>(256)) ||
      cudaFuncSetAttribute(k_ensemble<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ens_smem<double>(256)) ||
      cudaFuncSetAttribute(k_ensemble<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ens_smem<float>(256)) ||
      cudaFuncSetAttribute(k_ensemble<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ens_smem<float>(256)))
    return fail(BP_ECUDA);
  for (int cpb : {32, 64, 128, 256})
    for (int colored : {0, 1}) {
      Candidate c;
      if ((rc = build_candidate(e, cpb, colored, s, &c))) return fail(rc);
      e->cands.push_back(c);
    }
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(BP_ECUDA);
  *out = e;
  return BP_OK;
}

namespace {
int capture(bp_ensemble* e, int i, cudaStream_t s) {
  if (e->exec) {
    cudaGraphExecDestroy(e->exec);
    e->exec = nullptr;
  }
  if (e->graph) {
    cudaGraphDestroy(e->graph);
    e->graph = nullptr;
  }
  e->chosen = i;
  cudaStream_t cs;
  BP_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  BP_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  int rc = launch_candidate(e, e->cands[i], cs);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (rc) return rc;
  BP_CUDA_TRY(ce);
  e->graph = graph;
  BP_CUDA_TRY(cudaGraphInstantiate(&e->exec, e->graph, 0));
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  return BP_OK;
}
}  // namespace

extern "C" int bp_ensemble_select(bp_ensemble* e, int cpb, int scatter, void* stream) {
  if (!e) return BP_EINVAL;
  bp_device_guard g(e->device);
  for (size_t i = 0; i < e->cands.size(); ++i)
    if (e->cands[i].cpb == cpb && e->cands[i].colored == (scatter == BP_SCATTER_COLOR))
      return capture(e, (int)i, (cudaStream_t)stream);
  return BP_EINVAL;
}

extern "C" int bp_ensemble_tune(bp_ensemble* e, int reps, void* stream, double* times_ms, int* chosen) {
  if (!e || reps < 1) return BP_EINVAL;
  bp_device_guard g(e->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t a = nullptr, b = nullptr;
  struct EvFree {  // the events are released on every return path
    cudaEvent_t *a, *b;
    ~EvFree() {
      if (*a) cudaEventDestroy(*a);
      if (*b) cudaEventDestroy(*b);
    }
  } evfree{&a, &b};
  BP_CUDA_TRY(cudaEventCreate(&a));
  BP_CUDA_TRY(cudaEventCreate(&b));
  double best = 1e300;
  int best_i = 0;
  for (size_t i = 0; i < e->cands.size(); ++i) {
    int rc = launch_candidate(e, e->cands[i], s);  // warm-up
    if (rc) return rc;
    std::vector<float> t(reps);
    for (int r = 0; r < reps; ++r) {
      BP_CUDA_TRY(cudaEventRecord(a, s));
      if ((rc = launch_candidate(e, e->cands[i], s))) return rc;
      BP_CUDA_TRY(cudaEventRecord(b, s));
      BP_CUDA_TRY(cudaEventSynchronize(b));
      BP_CUDA_TRY(cudaEventElapsedTime(&t[r], a, b));
    }
    std::sort(t.begin(), t.end());
    const double med = t[reps / 2];
    if (times_ms) times_ms[i] = med;
    if (med < best) {
      best = med;
      best_i = (int)i;
    }
  }
  if (chosen) {
    chosen[0] = e->cands[best_i].cpb;
    chosen[1] = e->cands[best_i].colored ? BP_SCATTER_COLOR : BP_SCATTER_ATOMIC;
  }
  return capture(e, best_i, s);
}

extern "C" int bp_ensemble_assemble(bp_ensemble* e, void* stream) {
  if (!e) return BP_EINVAL;
  bp_device_guard g(e->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (e->exec) {
    BP_CUDA_TRY(cudaGraphLaunch(e->exec, s));
    return BP_OK;
  }
  for (auto& c : e->cands)
    if (c.cpb == 128 && !c.colored) return launch_candidate(e, c, s);
  return BP_EINVAL;
}
