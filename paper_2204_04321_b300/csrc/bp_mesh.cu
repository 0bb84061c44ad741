// Mesh upload: validation, extruded CSR pattern, scatter slots, triangle colouring and the
// solution-independent data of the assembly (paper Sec. 4.1 memoisation: the surface
// gradient, the driving-stress load and the basal friction matrices do not change between
// Newton iterations, so they are formed once here).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "bp_internal.cuh"

namespace {
thread_local char g_last_error[256] = "";
}

void bp_set_last_cuda_error(cudaError_t err, const char* what, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s (%s, line %d)", cudaGetErrorString(err), what, line);
}

extern "C" const char* bp_version(void) { return "libbp 0.1 (sm_103a)"; }

extern "C" const char* bp_strerror(int status) {
  switch (status) {
    case BP_OK: return "success";
    case BP_EINVAL: return "invalid argument";
    case BP_EMESH: return "invalid mesh";
    case BP_ENOMEM: return "out of device memory";
    case BP_ECUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case BP_ENAN: return "non-finite value";
    case BP_ENOCONV: return "iteration limit reached before the tolerance";
    case BP_EUNSUP: return "unsupported parameters (the kernels implement Glen exponent n = 3)";
    case BP_ESIZE: return "problem exceeds the fixed capacity of this call (BP_NOALLOC_MAX_NDOF dofs)";
    case BP_EIO: return "file could not be read or written, or is not in the expected format";
    default: return "unknown status";
  }
}

namespace {

// row pointer of every dof from the per-vertex block start and closed-neighbourhood size
__global__ void k_rowptr(const int64_t* __restrict__ vstart, const int32_t* __restrict__ vdeg, int nv,
                         int L, int64_t nnz, int64_t* __restrict__ rowptr) {
  const int64_t ndof = 2LL * nv * (L + 1);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= ndof;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (r == ndof) {
      rowptr[r] = nnz;
      continue;
    }
    const int64_t a = r / (2 * (L + 1));
    const int rem = (int)(r - a * 2 * (L + 1));
    const int l = rem >> 1, c = rem & 1;
    rowptr[r] = vstart[a] + (int64_t)vdeg[a] * (4 * bp_levels_before(l) + 2 * c * bp_nlev(l, L));
  }
}

// column indices: row (a, l, c) holds (b, l', c') for b in the sorted closed neighbourhood,
// l' = max(0, l-1) .. min(L, l+1), c' = 0, 1 -- already in increasing dof order.
__global__ void k_colidx(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ nbr_ptr,
                         const int32_t* __restrict__ nbr_idx, int nv, int L, int32_t* __restrict__ colidx) {
  const int64_t ndof = 2LL * nv * (L + 1);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < ndof;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = r / (2 * (L + 1));
    const int l = (int)((r - a * 2 * (L + 1)) >> 1);
    const int lmin = l > 0 ? l - 1 : 0, lmax = l < L ? l + 1 : L;
    int64_t pos = rowptr[r];
    for (int s = nbr_ptr[a]; s < nbr_ptr[a + 1]; ++s) {
      const int b = nbr_idx[s];
      for (int lp = lmin; lp <= lmax; ++lp) {
        colidx[pos++] = (int32_t)bp_dof(b, lp, 0, L);
        colidx[pos++] = (int32_t)bp_dof(b, lp, 1, L);
      }
    }
  }
}

// Driving-stress load rho g grad s . int N_{a,k} and the basal friction matrices.
// Over a wedge with vertical edges int lambda_a psi_k dV = area/24 (h_a + h_0 + h_1 + h_2), which the
// 6-point rule integrates exactly.  The basal matrix uses the 3-point triangle rule on the true face area
// (the integrand beta lambda_a lambda_b is cubic, so the rule -- not the exact integral -- defines it).
// Ocean margin load (Sec. 2, lateral condition 2 mu eps_c . n = (rho g (s - z) - rho_w g max(-z, 0)) n_c):
// the vertical face over boundary edge a -> b and layer l adds -int f n_c N_i dGamma to the load of its
// four nodes.  Along the edge t in [0, 1], across the layer zeta in [-1, 1]: N = lambda(t) psi(zeta),
// n_c dGamma = e_c (dz/dzeta) dt dzeta with e = (dy, -dx) the outward edge normal times the edge length
// (triangles counter-clockwise).  2 x 2 Gauss points, weights 1/2 (t) x 1 (zeta).  One thread per
// (edge, layer); atomics because neighbouring faces share nodes.
__global__ void k_margin_load(const double2* __restrict__ xy, const double* __restrict__ bed,
                              const double* __restrict__ thick, const double* __restrict__ sigma,
                              const int2* __restrict__ edges, int nedges, int L, double rg, double rwg,
                              double* __restrict__ load) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)nedges * L) return;
  const int e = (int)(i / L), l = (int)(i - (int64_t)e * L);
  const int v[2] = {edges[e].x, edges[e].y};
  const double2 pa = xy[v[0]], pb = xy[v[1]];
  const double en[2] = {pb.y - pa.y, pa.x - pb.x};
  double zlo[2], zhi[2], sv[2];
  for (int j = 0; j < 2; ++j) {
    zlo[j] = bed[v[j]] + sigma[l] * thick[v[j]];
    zhi[j] = bed[v[j]] + sigma[l + 1] * thick[v[j]];
    sv[j] = bed[v[j]] + thick[v[j]];
  }
  const double gp = 0.5 / sqrt(3.0);
  double acc[2][2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};  // [vertex][level k][component]
  for (int it = 0; it < 2; ++it)
    for (int iz = 0; iz < 2; ++iz) {
      const double t = it == 0 ? 0.5 - gp : 0.5 + gp;
      const double zeta = iz == 0 ? -2.0 * gp : 2.0 * gp;
      const double lam[2] = {1.0 - t, t}, psi[2] = {0.5 * (1.0 - zeta), 0.5 * (1.0 + zeta)};
      double z = 0.0, s = 0.0, dz = 0.0;
      for (int j = 0; j < 2; ++j) {
        z += lam[j] * (psi[0] * zlo[j] + psi[1] * zhi[j]);
        s += lam[j] * sv[j];
        dz += lam[j] * 0.5 * (zhi[j] - zlo[j]);
      }
      const double f = rg * (s - z) - rwg * fmax(-z, 0.0);
      const double wf = 0.5 * f * dz;
      for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k)
          for (int c = 0; c < 2; ++c) acc[j][k][c] += wf * en[c] * lam[j] * psi[k];
    }
  for (int j = 0; j < 2; ++j)
    for (int k = 0; k < 2; ++k)
      for (int c = 0; c < 2; ++c) atomicAdd(load + bp_dof(v[j], l + k, c, L), -acc[j][k][c]);
}

__global__ void k_memo(const double2* __restrict__ xy, const double* __restrict__ bed,
                       const double* __restrict__ thick, const double* __restrict__ beta,
                       const double* __restrict__ sigma, const int32_t* __restrict__ tri, int ntri, int L,
                       double rho_g, double* __restrict__ load, double* __restrict__ basal, int do_load) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntri) return;
  int v[3];
  double x[3], y[3], s[3], H[3], b[3], be[3];
  for (int a = 0; a < 3; ++a) {
    v[a] = tri[3 * t + a];
    const double2 p = xy[v[a]];
    x[a] = p.x;
    y[a] = p.y;
    H[a] = thick[v[a]];
    b[a] = bed[v[a]];
    s[a] = b[a] + H[a];
    be[a] = beta[v[a]];
  }
  const double d = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
  const double inv_d = 1.0 / d;
  // grad lambda_a = (y_{a+1} - y_{a+2}, x_{a+2} - x_{a+1}) / d
  double sx = 0.0, sy = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    sx += s[a] * (y[a1] - y[a2]) * inv_d;
    sy += s[a] * (x[a2] - x[a1]) * inv_d;
  }
  const double area = 0.5 * d;
  for (int l = 0; do_load && l < L; ++l) {
    const double ds = sigma[l + 1] - sigma[l];
    const double hsum = ds * (H[0] + H[1] + H[2]);
    for (int a = 0; a < 3; ++a) {
      const double intN = area / 24.0 * (ds * H[a] + hsum);
      for (int k = 0; k < 2; ++k) {
        atomicAdd(load + bp_dof(v[a], l + k, 0, L), rho_g * sx * intN);
        atomicAdd(load + bp_dof(v[a], l + k, 1, L), rho_g * sy * intN);
      }
    }
  }
  // basal face: true area of the triangle (x_a, y_a, b_a)
  const double e1x = x[1] - x[0], e1y = y[1] - y[0], e1z = b[1] - b[0];
  const double e2x = x[2] - x[0], e2y = y[2] - y[0], e2z = b[2] - b[0];
  const double cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
  const double area2 = sqrt(cx * cx + cy * cy + cz * cz);
  double M[6] = {0, 0, 0, 0, 0, 0};
  for (int q = 0; q < 3; ++q) {
    double lam[3];
    for (int a = 0; a < 3; ++a) lam[a] = (a == q) ? 2.0 / 3.0 : 1.0 / 6.0;
    const double bq = lam[0] * be[0] + lam[1] * be[1] + lam[2] * be[2];
    const double w = area2 / 6.0 * bq;
    M[0] += w * lam[0] * lam[0];
    M[1] += w * lam[0] * lam[1];
    M[2] += w * lam[0] * lam[2];
    M[3] += w * lam[1] * lam[1];
    M[4] += w * lam[1] * lam[2];
    M[5] += w * lam[2] * lam[2];
  }
  for (int i = 0; i < 6; ++i) basal[6 * (int64_t)t + i] = M[i];
}

int validate(const bp_mesh_desc* d) {
  if (!d || !d->xy || !d->tri || !d->bed || !d->thick || !d->beta || !d->sigma) return BP_EINVAL;
  if (d->nv < 3 || d->ntri < 1 || d->nlayers < 1) return BP_EINVAL;
  if (d->params.n != 3.0) return BP_EUNSUP;
  if (!(d->params.A > 0) || !(d->params.rho > 0) || !(d->params.g > 0) || !(d->params.delta >= 0))
    return BP_EINVAL;
  if (d->params.margin != BP_MARGIN_FREE && d->params.margin != BP_MARGIN_OCEAN) return BP_EINVAL;
  if (d->params.margin == BP_MARGIN_OCEAN && !(d->params.rho_w >= 0 && std::isfinite(d->params.rho_w)))
    return BP_EINVAL;
  const int L = d->nlayers;
  // ndof must fit the int32 column indices
  if (2.0 * d->nv * (L + 1) >= 2147483647.0) return BP_EINVAL;
  if (d->sigma[0] != 0.0 || d->sigma[L] != 1.0) return BP_EMESH;
  for (int l = 0; l < L; ++l)
    if (!(d->sigma[l + 1] > d->sigma[l])) return BP_EMESH;
  for (int a = 0; a < d->nv; ++a) {
    if (!(d->thick[a] > 0) || !(d->beta[a] >= 0) || !std::isfinite(d->bed[a]) ||
        !std::isfinite(d->xy[2 * a]) || !std::isfinite(d->xy[2 * a + 1]) || !std::isfinite(d->beta[a]) ||
        !std::isfinite(d->thick[a]))
      return BP_EMESH;
  }
  for (int t = 0; t < d->ntri; ++t) {
    int v[3];
    for (int a = 0; a < 3; ++a) {
      v[a] = d->tri[3 * t + a];
      if (v[a] < 0 || v[a] >= d->nv) return BP_EMESH;
    }
    if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) return BP_EMESH;
    const double* P = d->xy;
    const double det = (P[2 * v[1]] - P[2 * v[0]]) * (P[2 * v[2] + 1] - P[2 * v[0] + 1]) -
                       (P[2 * v[2]] - P[2 * v[0]]) * (P[2 * v[1] + 1] - P[2 * v[0] + 1]);
    if (!(det > 0)) return BP_EMESH;
  }
  return BP_OK;
}

}  // namespace

extern "C" void bp_mesh_free(bp_mesh* m) {
  if (!m) return;
  bp_device_guard g(m->device);
  cudaDeviceSynchronize();
  bp_solver_ws_free(m);
  for (void* p : m->allocations) cudaFree(p);
  delete m;
}

extern "C" int bp_mesh_upload(const bp_mesh_desc* d, void* stream_, bp_mesh** out) {
  if (!out) return BP_EINVAL;
  *out = nullptr;
  int rc = validate(d);
  if (rc) return rc;
  cudaStream_t stream = (cudaStream_t)stream_;
  const int nv = d->nv, ntri = d->ntri, L = d->nlayers;
  int device = 0;
  BP_CUDA_TRY(cudaGetDevice(&device));

  // closed neighbourhoods from the triangle list (sorted, unique)
  std::vector<int64_t> pairs;
  pairs.reserve((size_t)ntri * 9);
  for (int t = 0; t < ntri; ++t)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) pairs.push_back((int64_t)d->tri[3 * t + a] * nv + d->tri[3 * t + b]);
  std::sort(pairs.begin(), pairs.end());
  pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
  std::vector<int32_t> nbr_ptr(nv + 1, 0), nbr_idx(pairs.size());
  for (size_t i = 0; i < pairs.size(); ++i) {
    nbr_ptr[pairs[i] / nv + 1]++;
    nbr_idx[i] = (int32_t)(pairs[i] % nv);
  }
  for (int a = 0; a < nv; ++a) nbr_ptr[a + 1] += nbr_ptr[a];
  std::vector<int32_t> vdeg(nv);
  std::vector<int64_t> vstart(nv);
  int64_t acc = 0;
  for (int a = 0; a < nv; ++a) {
    vdeg[a] = nbr_ptr[a + 1] - nbr_ptr[a];
    if (vdeg[a] < 2) return BP_EMESH;  // vertex used by no triangle
    vstart[a] = acc;
    acc += 4LL * vdeg[a] * (3 * L + 1);
  }
  const int64_t nnz = acc;
  std::vector<int32_t> slots((size_t)ntri * 9);
  for (int t = 0; t < ntri; ++t)
    for (int a = 0; a < 3; ++a) {
      const int va = d->tri[3 * t + a];
      const int32_t* b0 = nbr_idx.data() + nbr_ptr[va];
      const int32_t* b1 = nbr_idx.data() + nbr_ptr[va + 1];
      for (int b = 0; b < 3; ++b) {
        const int vb = d->tri[3 * t + b];
        slots[9 * (size_t)t + 3 * a + b] = (int32_t)(std::lower_bound(b0, b1, vb) - b0);
      }
    }
  // greedy colouring: triangles sharing a vertex get different colours
  std::vector<uint64_t> used(nv, 0);
  std::vector<int32_t> color(ntri);
  int ncolors = 0;
  for (int t = 0; t < ntri; ++t) {
    uint64_t u = 0;
    for (int a = 0; a < 3; ++a) u |= used[d->tri[3 * t + a]];
    if (~u == 0) return BP_EMESH;  // more than 64 colours needed (pathological vertex degree)
    int c = 0;
    while (u & (1ULL << c)) ++c;
    color[t] = c;
    ncolors = std::max(ncolors, c + 1);
    for (int a = 0; a < 3; ++a) used[d->tri[3 * t + a]] |= (1ULL << c);
  }
  std::vector<int32_t> color_off(ncolors + 1, 0), color_tris(ntri);
  for (int t = 0; t < ntri; ++t) color_off[color[t] + 1]++;
  for (int c = 0; c < ncolors; ++c) color_off[c + 1] += color_off[c];
  {
    std::vector<int32_t> fill(color_off.begin(), color_off.end() - 1);
    for (int t = 0; t < ntri; ++t) color_tris[fill[color[t]]++] = t;
  }

  bp_mesh* m = new bp_mesh();
  m->device = device;
  m->nv = nv;
  m->ntri = ntri;
  m->nl = L;
  m->ndof = 2LL * nv * (L + 1);
  m->nnz = nnz;
  m->p = d->params;
  m->cA = std::pow(d->params.A, -1.0 / 3.0);
  m->ncolors = ncolors;
  m->color_off = color_off;

  auto fail = [&](int code) {
    bp_mesh_free(m);
    return code;
  };
#define BP_ALLOC(ptr, n) \
  if ((rc = bp_alloc(m, &(ptr), (n))) != BP_OK) return fail(rc)
  BP_ALLOC(m->xy, nv);
  BP_ALLOC(m->bed, nv);
  BP_ALLOC(m->thick, nv);
  BP_ALLOC(m->beta, nv);
  BP_ALLOC(m->vstart, nv);
  BP_ALLOC(m->vdeg, nv);
  BP_ALLOC(m->nbr_ptr, nv + 1);
  BP_ALLOC(m->nbr_idx, nbr_idx.size());
  BP_ALLOC(m->sigma, 2 * L + 1);
  BP_ALLOC(m->tri, 3 * (size_t)ntri);
  BP_ALLOC(m->slots, 9 * (size_t)ntri);
  BP_ALLOC(m->basal, 6 * (size_t)ntri);
  BP_ALLOC(m->color_tris, ntri);
  BP_ALLOC(m->rowptr, m->ndof + 1);
  BP_ALLOC(m->colidx, nnz);
  BP_ALLOC(m->load, m->ndof);
#undef BP_ALLOC

#define BP_H2D(dst, src, n)                                                                       \
  do {                                                                                           \
    cudaError_t e_ = cudaMemcpyAsync((dst), (src), (n) * sizeof(*(dst)), cudaMemcpyHostToDevice, \
                                     stream);                                                    \
    if (e_ != cudaSuccess) {                                                                     \
      bp_set_last_cuda_error(e_, "upload", __LINE__);                                            \
      return fail(BP_ECUDA);                                                                     \
    }                                                                                            \
  } while (0)
  BP_H2D(m->xy, reinterpret_cast<const double2*>(d->xy), nv);
  BP_H2D(m->bed, d->bed, nv);
  BP_H2D(m->thick, d->thick, nv);
  BP_H2D(m->beta, d->beta, nv);
  BP_H2D(m->vstart, vstart.data(), nv);
  BP_H2D(m->vdeg, vdeg.data(), nv);
  BP_H2D(m->nbr_ptr, nbr_ptr.data(), nv + 1);
  BP_H2D(m->nbr_idx, nbr_idx.data(), nbr_idx.size());
  // the levels, then the inverse layer thicknesses 1 / (sigma_{l+1} - sigma_l) (IEEE division here,
  // bitwise what the kernels would form)
  std::vector<double> sig(2 * (size_t)L + 1);
  for (int l = 0; l <= L; ++l) sig[l] = d->sigma[l];
  for (int l = 0; l < L; ++l) sig[L + 1 + l] = 1.0 / (d->sigma[l + 1] - d->sigma[l]);
  BP_H2D(m->sigma, sig.data(), 2 * (size_t)L + 1);
  BP_H2D(m->tri, d->tri, 3 * (size_t)ntri);
  BP_H2D(m->slots, slots.data(), 9 * (size_t)ntri);
  BP_H2D(m->color_tris, color_tris.data(), ntri);
#undef BP_H2D
  if (cudaMemsetAsync(m->load, 0, m->ndof * sizeof(double), stream) != cudaSuccess) return fail(BP_ECUDA);
  const int threads = 256;
  const int grid_rows = (int)std::min<int64_t>((m->ndof + threads) / threads, 148 * 64);
  k_rowptr<<<grid_rows, threads, 0, stream>>>(m->vstart, m->vdeg, nv, L, nnz, m->rowptr);
  k_colidx<<<grid_rows, threads, 0, stream>>>(m->rowptr, m->nbr_ptr, m->nbr_idx, nv, L, m->colidx);
  k_memo<<<(ntri + 127) / 128, 128, 0, stream>>>(m->xy, m->bed, m->thick, m->beta, m->sigma, m->tri, ntri, L,
                                                 d->params.rho * d->params.g, m->load, m->basal, 1);
  if (d->params.margin == BP_MARGIN_OCEAN) {
    // boundary edges: directed edges a -> b of the (counter-clockwise) triangles whose reverse is absent
    std::vector<int64_t> dir;
    dir.reserve(3 * (size_t)ntri);
    for (int t = 0; t < ntri; ++t)
      for (int k = 0; k < 3; ++k) dir.push_back((int64_t)d->tri[3 * t + k] * nv + d->tri[3 * t + (k + 1) % 3]);
    std::sort(dir.begin(), dir.end());
    std::vector<int2> bedges;
    for (int64_t key : dir) {
      const int a = (int)(key / nv), b = (int)(key % nv);
      if (!std::binary_search(dir.begin(), dir.end(), (int64_t)b * nv + a)) bedges.push_back(make_int2(a, b));
    }
    m->nbedges = (int)bedges.size();
    if (m->nbedges > 0) {
      if ((rc = bp_alloc(m, &m->bedges, bedges.size())) != BP_OK) return fail(rc);
      if (cudaMemcpyAsync(m->bedges, bedges.data(), bedges.size() * sizeof(int2), cudaMemcpyHostToDevice,
                          stream) != cudaSuccess)
        return fail(BP_ECUDA);
      const int64_t work = (int64_t)m->nbedges * L;
      k_margin_load<<<(int)((work + 127) / 128), 128, 0, stream>>>(
          m->xy, m->bed, m->thick, m->sigma, m->bedges, m->nbedges, L, d->params.rho * d->params.g,
          d->params.rho_w * d->params.g, m->load);
      // the upload returns only after the stream is synchronised below, so `bedges` outlives the copy
      cudaError_t ce = cudaStreamSynchronize(stream);
      if (ce != cudaSuccess) {
        bp_set_last_cuda_error(ce, "margin load", __LINE__);
        return fail(BP_ECUDA);
      }
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    bp_set_last_cuda_error(e, "mesh upload kernels", __LINE__);
    return fail(BP_ECUDA);
  }
  *out = m;
  return BP_OK;
}

extern "C" int bp_mesh_info(const bp_mesh* m, bp_mesh_info_t* info) {
  if (!m || !info) return BP_EINVAL;
  info->ndof = m->ndof;
  info->nnz = m->nnz;
  info->nwedges = (int64_t)m->ntri * m->nl;
  info->nv = m->nv;
  info->ntri = m->ntri;
  info->nlayers = m->nl;
  info->ncolors = m->ncolors;
  info->device_bytes = m->device_bytes;
  return BP_OK;
}

extern "C" int bp_csr_pattern(const bp_mesh* m, const int64_t** rowptr, const int32_t** colidx) {
  if (!m || !rowptr || !colidx) return BP_EINVAL;
  *rowptr = m->rowptr;
  *colidx = m->colidx;
  return BP_OK;
}

extern "C" int bp_mesh_set_rate_factor(bp_mesh* m, const double* A, void* stream) {
  if (!m) return BP_EINVAL;
  if (!A) {  // back to the uniform rate factor of the upload parameters
    m->Bnode = nullptr;
    return BP_OK;
  }
  const int64_t n = (int64_t)m->nv * (m->nl + 1);
  std::vector<double> B(n);
  for (int64_t i = 0; i < n; ++i) {
    if (!(A[i] > 0) || !std::isfinite(A[i])) return BP_EINVAL;
    B[i] = std::pow(A[i], -1.0 / 3.0);  // hardness, interpolated at the quadrature points
  }
  bp_device_guard g(m->device);
  if (!m->Bnode_buf) {
    int rc = bp_alloc(m, &m->Bnode_buf, (size_t)n);
    if (rc) return rc;
  }
  cudaStream_t s = (cudaStream_t)stream;
  BP_CUDA_TRY(cudaMemcpyAsync(m->Bnode_buf, B.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  m->Bnode = m->Bnode_buf;
  return BP_OK;
}

extern "C" int bp_mesh_set_beta(bp_mesh* m, const double* beta, void* stream) {
  if (!m || !beta) return BP_EINVAL;
  for (int a = 0; a < m->nv; ++a)
    if (!(beta[a] >= 0) || !std::isfinite(beta[a])) return BP_EMESH;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  BP_CUDA_TRY(cudaMemcpyAsync(m->beta, beta, m->nv * sizeof(double), cudaMemcpyHostToDevice, s));
  k_memo<<<(m->ntri + 127) / 128, 128, 0, s>>>(m->xy, m->bed, m->thick, m->beta, m->sigma, m->tri, m->ntri, m->nl,
                                               m->p.rho * m->p.g, m->load, m->basal, 0);
  BP_CUDA_TRY(cudaGetLastError());
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  return BP_OK;
}
