// CPU oracle for the first-order (Blatter-Pattyn) Stokes velocity residual and Jacobian.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct FP64 statement
// of what the CUDA path computes.  Only the test-suite, the smoke check and the CPU-baseline
// leg of the benchmark may load it.  It shares no code, header, table or helper with the
// CUDA library: both sides read the same seeded inputs and nothing else.
//
// What it computes (paper section / equation in brackets):
//  * the momentum equations -div(2 mu eps_1) + rho g ds/dx = 0 (and eps_2, ds/dy)   [Sec. 2, Eq. FOStokes]
//  * strain-rate vectors eps_1 = [2 exx + eyy, exy, exz], eps_2 = [exy, exx + 2 eyy, eyz]
//    with exx = u_x, eyy = v_y, exy = (u_y + v_x)/2, exz = u_z/2, eyz = v_z/2     [Sec. 2]
//  * Glen viscosity mu = 1/2 A^(-1/n) (eps_e^2 + delta)^((1-n)/(2n))             [Sec. 2, Eq. effvisc,
//    with the effective strain rate eps_e^2 = exx^2 + eyy^2 + exx eyy + exy^2 + exz^2 + eyz^2   Eq. effeps]
//    (delta regularises U = 0; the paper's form is the delta = 0 limit)
//  * stress-free upper surface (natural, contributes nothing), linear sliding law
//    2 mu eps . n + beta u = 0 at the bed (Robin), and on the vertical margins either
//    stress-free (margin = 0) or the ocean condition (margin = 1)                      [Sec. 2 BCs]
//    2 mu eps_c . n = (rho g (s - z) - rho_w g max(-z, 0)) n_c  (z = 0 at sea level; the
//    paper prints max(z, 0), read as the submerged part), whose weak form adds
//    -int_face (rho g (s - z) - rho_w g max(-z, 0)) n_c N_i to R_i on every vertical face
//    over a boundary edge of the base triangulation (2 x 2 Gauss rule per face);
//  * discretised with low-order nodal prismatic (6-node wedge) elements on the mesh
//    extruded from the base triangulation, residual F(U; {phi_i}, {grad phi_i}, H, beta)  [Sec. 3.1, Eq. residual]
//  * the Jacobian dF/dU by forward-mode automatic differentiation with a compile-time
//    number of derivative lanes (12 = 6 nodes x 2 components), the SFad choice of   [Sec. 3.2]
//
// Readings where the paper is silent (stated once here, used throughout):
//  * weak form: test with phi_i, integrate the stress term by parts; bed term
//    integrated over the true (3D) basal face area;
//  * reference wedge: lambda = (1 - xi - eta, xi, eta), N = lambda_a (1 -/+ zeta)/2,
//    bottom nodes 0..2 then top nodes 3..5, local dof j = 2 * node + component;
//  * volume quadrature: 3-point triangle rule (points (1/6,1/6), (2/3,1/6), (1/6,2/3),
//    weights 1/6) x 2-point Gauss-Legendre in zeta (+-1/sqrt 3, weights 1); basal face:
//    the same triangle rule at zeta = -1;
//  * s, beta, z nodal; z = b + sigma_l H; s = b + H;
//  * a temperature-dependent rate factor (Arrhenius, Sec. 2) enters as nodal A; its hardness
//    A^(-1/n) is interpolated with the wedge basis at each quadrature point.
//
// Nothing here is blocked, fused or reordered for speed.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <thread>
#include <utility>
#include <vector>

namespace {

struct Mesh {
  int32_t nv, ntri, nlayers;
  const double* xy;     // [nv][2]
  const int32_t* tri;   // [ntri][3]
  const double* bed;    // [nv]
  const double* thick;  // [nv]
  const double* beta;   // [nv]
  const double* sigma;  // [nlayers + 1]
  double n, A, rho, g, delta;
  double rho_w;         // sea-water density (margin = 1)
  int32_t margin;       // 0: stress-free vertical margins; 1: ocean condition
  const double* Anode;  // nullable [nv][L + 1] rate factor per node (else the constant A)
};

// A^(-1/n) at a point with wedge basis values N (nodes: bottom a = 0..2 at level l, top at l + 1):
// the nodal values of A^(-1/n) interpolated with the basis (reading of the Arrhenius field's
// per-point evaluation), or the constant A^(-1/n).
inline double hardness(const Mesh& m, const int64_t vert[3], int l, const double N[6]) {
  if (!m.Anode) return std::pow(m.A, -1.0 / m.n);
  double B = 0.0;
  for (int k = 0; k < 2; ++k)
    for (int a = 0; a < 3; ++a)
      B += N[3 * k + a] * std::pow(m.Anode[vert[a] * (m.nlayers + 1) + l + k], -1.0 / m.n);
  return B;
}

// ---------------------------------------------------------------- dual numbers
constexpr int NL = 12;
struct Dual {
  double v;
  double d[NL];
};
inline Dual dconst(double a) {
  Dual r;
  r.v = a;
  for (int k = 0; k < NL; ++k) r.d[k] = 0.0;
  return r;
}
inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v + b.v;
  for (int k = 0; k < NL; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v - b.v;
  for (int k = 0; k < NL; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v * b.v;
  for (int k = 0; k < NL; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
inline Dual operator*(double s, const Dual& a) {
  Dual r;
  r.v = s * a.v;
  for (int k = 0; k < NL; ++k) r.d[k] = s * a.d[k];
  return r;
}
inline Dual operator*(const Dual& a, double s) { return s * a; }
inline Dual operator+(const Dual& a, double s) {
  Dual r = a;
  r.v += s;
  return r;
}
// x^p for a dual: value x^p, derivative p x^(p-1) x'
inline Dual dpow(const Dual& x, double p) {
  Dual r;
  r.v = std::pow(x.v, p);
  const double dv = p * std::pow(x.v, p - 1.0);
  for (int k = 0; k < NL; ++k) r.d[k] = dv * x.d[k];
  return r;
}
inline double dpow(double x, double p) { return std::pow(x, p); }
// helpers so the template can build zeros of the right type
inline double dconst_like(double, double a) { return a; }
inline Dual dconst_like(const Dual&, double a) { return dconst(a); }
inline double value_of(double a) { return a; }
inline double value_of(const Dual& a) { return a.v; }

// ---------------------------------------------------------------- reference wedge
const double kTriQp[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
const double kTriW = 1.0 / 6.0;

inline void ref_shape(double xi, double eta, double zeta, double N[6], double dN[6][3]) {
  const double lam[3] = {1.0 - xi - eta, xi, eta};
  const double dlam[3][2] = {{-1.0, -1.0}, {1.0, 0.0}, {0.0, 1.0}};
  const double psi[2] = {0.5 * (1.0 - zeta), 0.5 * (1.0 + zeta)};
  const double dpsi[2] = {-0.5, 0.5};
  for (int k = 0; k < 2; ++k)
    for (int a = 0; a < 3; ++a) {
      const int i = 3 * k + a;
      N[i] = lam[a] * psi[k];
      dN[i][0] = dlam[a][0] * psi[k];
      dN[i][1] = dlam[a][1] * psi[k];
      dN[i][2] = lam[a] * dpsi[k];
    }
}

// Physical basis at reference point: N, grad N (physical), det of the reference->physical map.
inline void phys_basis(const double X[6][3], double xi, double eta, double zeta, double N[6],
                       double gN[6][3], double* detJ) {
  double dN[6][3];
  ref_shape(xi, eta, zeta, N, dN);
  double J[3][3] = {{0}};  // J[r][s] = d x_r / d ref_s
  for (int i = 0; i < 6; ++i)
    for (int r = 0; r < 3; ++r)
      for (int s = 0; s < 3; ++s) J[r][s] += X[i][r] * dN[i][s];
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  // inverse: Jinv[s][r] = d ref_s / d x_r
  double Jinv[3][3];
  Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  for (int i = 0; i < 6; ++i)
    for (int r = 0; r < 3; ++r) {
      double acc = 0.0;
      for (int s = 0; s < 3; ++s) acc += dN[i][s] * Jinv[s][r];
      gN[i][r] = acc;
    }
  *detJ = det;
}

inline void qp_ref(int q, double* xi, double* eta, double* zeta, double* w) {
  const double gz = 1.0 / std::sqrt(3.0);
  const int t = q % 3, k = q / 3;
  *xi = kTriQp[t][0];
  *eta = kTriQp[t][1];
  *zeta = (k == 0) ? -gz : gz;
  *w = kTriW * 1.0;
}

inline int64_t dof_index(const Mesh& m, int64_t a, int64_t l, int c) {
  return 2 * (a * (m.nlayers + 1) + l) + c;
}

inline void wedge_nodes(const Mesh& m, int t, int l, int64_t vert[3], double X[6][3]) {
  for (int a = 0; a < 3; ++a) vert[a] = m.tri[3 * (int64_t)t + a];
  for (int k = 0; k < 2; ++k)
    for (int a = 0; a < 3; ++a) {
      const int64_t v = vert[a];
      X[3 * k + a][0] = m.xy[2 * v];
      X[3 * k + a][1] = m.xy[2 * v + 1];
      X[3 * k + a][2] = m.bed[v] + m.sigma[l + k] * m.thick[v];
    }
}

inline void node_dofs(const Mesh& m, int l, const int64_t vert[3], int64_t dofs[12]) {
  for (int k = 0; k < 2; ++k)
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 2; ++c) dofs[2 * (3 * k + a) + c] = dof_index(m, vert[a], l + k, c);
}

// Effective strain rate squared (Eq. effeps) from the velocity gradients grad u, grad v.
template <class S>
S effective_strain2(const S gu[3], const S gv[3]) {
  const S exx = gu[0];
  const S eyy = gv[1];
  const S exy = 0.5 * (gu[1] + gv[0]);
  const S exz = 0.5 * gu[2];
  const S eyz = 0.5 * gv[2];
  return exx * exx + eyy * eyy + exx * eyy + exy * exy + exz * exz + eyz * eyz;
}

// Strain-rate vectors eps_1, eps_2 of the x and y momentum equations (Sec. 2).
template <class S>
void strain_vectors(const S gu[3], const S gv[3], S eps1[3], S eps2[3]) {
  const S exx = gu[0];
  const S eyy = gv[1];
  const S exy = 0.5 * (gu[1] + gv[0]);
  eps1[0] = 2.0 * exx + eyy;
  eps1[1] = exy;
  eps1[2] = 0.5 * gu[2];
  eps2[0] = exy;
  eps2[1] = exx + 2.0 * eyy;
  eps2[2] = 0.5 * gv[2];
}

// Element residual of wedge (t, l) for scalar type S (double -> residual, Dual -> residual + Jacobian).
template <class S>
void element_residual(const Mesh& m, int t, int l, const S Ue[12], S Re[12]) {
  int64_t vert[3];
  double X[6][3];
  wedge_nodes(m, t, l, vert, X);
  double s_nodal[6];
  for (int k = 0; k < 2; ++k)
    for (int a = 0; a < 3; ++a) s_nodal[3 * k + a] = m.bed[vert[a]] + m.thick[vert[a]];
  for (int j = 0; j < 12; ++j) Re[j] = S(dconst_like(Ue[j], 0.0));
  const double pexp = (1.0 - m.n) / (2.0 * m.n);
  for (int q = 0; q < 6; ++q) {
    double xi, eta, zeta, w, N[6], gN[6][3], detJ;
    qp_ref(q, &xi, &eta, &zeta, &w);
    phys_basis(X, xi, eta, zeta, N, gN, &detJ);
    const double Ainv = hardness(m, vert, l, N);
    S gu[3], gv[3];
    for (int r = 0; r < 3; ++r) {
      gu[r] = S(dconst_like(Ue[0], 0.0));
      gv[r] = S(dconst_like(Ue[0], 0.0));
    }
    double gs[3] = {0, 0, 0};
    for (int i = 0; i < 6; ++i)
      for (int r = 0; r < 3; ++r) {
        gu[r] = gu[r] + gN[i][r] * Ue[2 * i];
        gv[r] = gv[r] + gN[i][r] * Ue[2 * i + 1];
        gs[r] += gN[i][r] * s_nodal[i];
      }
    const S e2 = effective_strain2(gu, gv);
    const S mu = (0.5 * Ainv) * dpow(e2 + m.delta, pexp);
    S eps1[3], eps2[3];
    strain_vectors(gu, gv, eps1, eps2);
    const double wq = w * detJ;
    for (int i = 0; i < 6; ++i) {
      S du = eps1[0] * gN[i][0] + eps1[1] * gN[i][1] + eps1[2] * gN[i][2];
      S dv = eps2[0] * gN[i][0] + eps2[1] * gN[i][1] + eps2[2] * gN[i][2];
      Re[2 * i] = Re[2 * i] + wq * (2.0 * mu * du + m.rho * m.g * gs[0] * N[i]);
      Re[2 * i + 1] = Re[2 * i + 1] + wq * (2.0 * mu * dv + m.rho * m.g * gs[1] * N[i]);
    }
  }
  if (l == 0) {  // basal face: bottom triangle nodes 0..2, Robin (linear sliding) term
    double e1[3], e2v[3], cr[3];
    for (int r = 0; r < 3; ++r) {
      e1[r] = X[1][r] - X[0][r];
      e2v[r] = X[2][r] - X[0][r];
    }
    cr[0] = e1[1] * e2v[2] - e1[2] * e2v[1];
    cr[1] = e1[2] * e2v[0] - e1[0] * e2v[2];
    cr[2] = e1[0] * e2v[1] - e1[1] * e2v[0];
    const double area2 = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    for (int q = 0; q < 3; ++q) {
      const double xi = kTriQp[q][0], eta = kTriQp[q][1];
      const double lam[3] = {1.0 - xi - eta, xi, eta};
      double bq = 0.0;
      S uq = S(dconst_like(Ue[0], 0.0)), vq = S(dconst_like(Ue[0], 0.0));
      for (int a = 0; a < 3; ++a) {
        bq += lam[a] * m.beta[vert[a]];
        uq = uq + lam[a] * Ue[2 * a];
        vq = vq + lam[a] * Ue[2 * a + 1];
      }
      const double wb = kTriW * area2;
      for (int a = 0; a < 3; ++a) {
        Re[2 * a] = Re[2 * a] + (wb * bq * lam[a]) * uq;
        Re[2 * a + 1] = Re[2 * a + 1] + (wb * bq * lam[a]) * vq;
      }
    }
  }
}


void gather_element(const Mesh& m, int l, const int64_t vert[3], const double* U, double Ue[12]) {
  int64_t dofs[12];
  node_dofs(m, l, vert, dofs);
  for (int j = 0; j < 12; ++j) Ue[j] = U[dofs[j]];
}

// Load of the ocean margin condition on the vertical faces over the boundary edges (edges a -> b
// of the counter-clockwise triangles whose reverse b -> a belongs to no triangle; the outward normal
// times the edge length is (dy, -dx)).  A face over layer l is parametrised by t in [0, 1] along the
// edge and zeta in [-1, 1]; on it N = (1 - t or t) (1 -/+ zeta) / 2 and n_c dGamma = (dy or -dx)
// dz/dzeta dt dzeta.  2 x 2 Gauss rule.  F[dof] receives -int f n_c N, f = rho g (s - z) - rho_w g
// max(-z, 0).  tri_mask (nullable): only edges of masked triangles.
void lateral_load(const Mesh& m, const uint8_t* tri_mask, double* F) {
  if (m.margin != 1) return;
  std::map<std::pair<int, int>, int> owner;  // directed edge -> triangle
  for (int t = 0; t < m.ntri; ++t)
    for (int e = 0; e < 3; ++e) owner[{m.tri[3 * t + e], m.tri[3 * t + (e + 1) % 3]}] = t;
  const double gt[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};  // weights 1/2
  const double gz[2] = {-1.0 / std::sqrt(3.0), 1.0 / std::sqrt(3.0)};            // weights 1
  for (const auto& kv : owner) {
    const int a = kv.first.first, b = kv.first.second;
    if (owner.count({b, a})) continue;  // interior edge
    if (tri_mask && !tri_mask[kv.second]) continue;
    const double dx = m.xy[2 * b] - m.xy[2 * a], dy = m.xy[2 * b + 1] - m.xy[2 * a + 1];
    const double sa = m.bed[a] + m.thick[a], sb = m.bed[b] + m.thick[b];
    for (int l = 0; l < m.nlayers; ++l) {
      const double za0 = m.bed[a] + m.sigma[l] * m.thick[a], za1 = m.bed[a] + m.sigma[l + 1] * m.thick[a];
      const double zb0 = m.bed[b] + m.sigma[l] * m.thick[b], zb1 = m.bed[b] + m.sigma[l + 1] * m.thick[b];
      const int64_t lev[2] = {l, l + 1};
      for (int it = 0; it < 2; ++it)
        for (int iz = 0; iz < 2; ++iz) {
          const double t = gt[it], zeta = gz[iz], w = 0.5;
          const double psi[2] = {0.5 * (1.0 - zeta), 0.5 * (1.0 + zeta)};
          const double z = (1 - t) * (psi[0] * za0 + psi[1] * za1) + t * (psi[0] * zb0 + psi[1] * zb1);
          const double s = (1 - t) * sa + t * sb;
          const double dzdzeta = 0.5 * ((1 - t) * (za1 - za0) + t * (zb1 - zb0));
          const double f = m.rho * m.g * (s - z) - m.rho_w * m.g * std::max(-z, 0.0);
          for (int k = 0; k < 2; ++k) {
            const double Na = (1 - t) * psi[k], Nb = t * psi[k];
            for (int c = 0; c < 2; ++c) {
              const double nc = (c == 0 ? dy : -dx) * dzdzeta;
              F[dof_index(m, a, lev[k], c)] -= w * f * nc * Na;
              F[dof_index(m, b, lev[k], c)] -= w * f * nc * Nb;
            }
          }
        }
    }
  }
}

bool mesh_ok(const Mesh& m) {
  if (m.nv <= 0 || m.ntri <= 0 || m.nlayers <= 0) return false;
  for (int64_t i = 0; i < 3 * (int64_t)m.ntri; ++i)
    if (m.tri[i] < 0 || m.tri[i] >= m.nv) return false;
  return true;
}

}  // namespace

extern "C" {

typedef struct {
  int32_t nv, ntri, nlayers, pad;
  const double* xy;
  const int32_t* tri;
  const double* bed;
  const double* thick;
  const double* beta;
  const double* sigma;
  double n, A, rho, g, delta;
  double rho_w;
  int32_t margin, pad2;
  const double* Anode;
} oracle_mesh;

static Mesh unpack(const oracle_mesh* d) {
  Mesh m;
  m.nv = d->nv;
  m.ntri = d->ntri;
  m.nlayers = d->nlayers;
  m.xy = d->xy;
  m.tri = d->tri;
  m.bed = d->bed;
  m.thick = d->thick;
  m.beta = d->beta;
  m.sigma = d->sigma;
  m.n = d->n;
  m.A = d->A;
  m.rho = d->rho;
  m.g = d->g;
  m.delta = d->delta;
  m.rho_w = d->rho_w;
  m.margin = d->margin;
  m.Anode = d->Anode;
  return m;
}

// Basis at an arbitrary reference point of a wedge with node coordinates X[6][3].
void oracle_basis_at(const double* X18, double xi, double eta, double zeta, double* N6,
                     double* gN18, double* detJ) {
  double X[6][3], gN[6][3];
  for (int i = 0; i < 6; ++i)
    for (int r = 0; r < 3; ++r) X[i][r] = X18[3 * i + r];
  phys_basis(X, xi, eta, zeta, N6, gN, detJ);
  for (int i = 0; i < 6; ++i)
    for (int r = 0; r < 3; ++r) gN18[3 * i + r] = gN[i][r];
}

// Reference coordinates and weight of volume quadrature point q (0..5).
void oracle_qp(int q, double* xi, double* eta, double* zeta, double* w) { qp_ref(q, xi, eta, zeta, w); }

// Quadrature-point state of wedge (t, l): out = [u_x,u_y,u_z, v_x,v_y,v_z, eps_e^2, mu, w*detJ, s_x, s_y]
int oracle_qp_state(const oracle_mesh* d, const double* U, int t, int l, int q, double* out) {
  const Mesh m = unpack(d);
  if (t < 0 || t >= m.ntri || l < 0 || l >= m.nlayers || q < 0 || q >= 6) return 1;
  int64_t vert[3];
  double X[6][3];
  wedge_nodes(m, t, l, vert, X);
  double Ue[12];
  gather_element(m, l, vert, U, Ue);
  double xi, eta, zeta, w, N[6], gN[6][3], detJ;
  qp_ref(q, &xi, &eta, &zeta, &w);
  phys_basis(X, xi, eta, zeta, N, gN, &detJ);
  double gu[3] = {0, 0, 0}, gv[3] = {0, 0, 0}, gs[3] = {0, 0, 0};
  for (int i = 0; i < 6; ++i)
    for (int r = 0; r < 3; ++r) {
      gu[r] += gN[i][r] * Ue[2 * i];
      gv[r] += gN[i][r] * Ue[2 * i + 1];
      gs[r] += gN[i][r] * (m.bed[vert[i % 3]] + m.thick[vert[i % 3]]);
    }
  const double e2 = effective_strain2(gu, gv);
  const double mu = 0.5 * hardness(m, vert, l, N) * std::pow(e2 + m.delta, (1.0 - m.n) / (2.0 * m.n));
  for (int r = 0; r < 3; ++r) {
    out[r] = gu[r];
    out[3 + r] = gv[r];
  }
  out[6] = e2;
  out[7] = mu;
  out[8] = w * detJ;
  out[9] = gs[0];
  out[10] = gs[1];
  return 0;
}

// Element residual (12) and element Jacobian (12 x 12, row-major, dRe_i/dUe_j) of wedge (t, l).
int oracle_element(const oracle_mesh* d, const double* U, int t, int l, double* Re, double* Ke) {
  const Mesh m = unpack(d);
  if (t < 0 || t >= m.ntri || l < 0 || l >= m.nlayers) return 1;
  int64_t vert[3];
  for (int a = 0; a < 3; ++a) vert[a] = m.tri[3 * (int64_t)t + a];
  double Ue[12];
  gather_element(m, l, vert, U, Ue);
  Dual Ud[12], Rd[12];
  for (int j = 0; j < 12; ++j) {
    Ud[j] = dconst(Ue[j]);
    Ud[j].d[j] = 1.0;
  }
  element_residual<Dual>(m, t, l, Ud, Rd);
  for (int i = 0; i < 12; ++i) {
    if (Re) Re[i] = Rd[i].v;
    if (Ke)
      for (int j = 0; j < 12; ++j) Ke[12 * i + j] = Rd[i].d[j];
  }
  return 0;
}

// Global residual R (overwritten).  tri_mask (nullable): only columns with mask != 0 contribute.
int oracle_residual(const oracle_mesh* d, const double* U, const uint8_t* tri_mask, double* R) {
  const Mesh m = unpack(d);
  if (!mesh_ok(m)) return 1;
  const int64_t ndof = 2 * (int64_t)m.nv * (m.nlayers + 1);
  std::memset(R, 0, sizeof(double) * ndof);
  for (int t = 0; t < m.ntri; ++t) {
    if (tri_mask && !tri_mask[t]) continue;
    int64_t vert[3];
    for (int a = 0; a < 3; ++a) vert[a] = m.tri[3 * (int64_t)t + a];
    for (int l = 0; l < m.nlayers; ++l) {
      double Ue[12], Re[12];
      int64_t dofs[12];
      gather_element(m, l, vert, U, Ue);
      element_residual<double>(m, t, l, Ue, Re);
      node_dofs(m, l, vert, dofs);
      for (int j = 0; j < 12; ++j) R[dofs[j]] += Re[j];
    }
  }
  lateral_load(m, tri_mask, R);
  return 0;
}

// Number of structural nonzeros of the extruded pattern (all pairs of dofs sharing a wedge).
int oracle_pattern_nnz(const oracle_mesh* d, int64_t* nnz) {
  const Mesh m = unpack(d);
  if (!mesh_ok(m)) return 1;
  const int64_t ndof = 2 * (int64_t)m.nv * (m.nlayers + 1);
  std::vector<std::vector<int32_t>> rows(ndof);
  for (int t = 0; t < m.ntri; ++t) {
    int64_t vert[3], dofs[12];
    for (int a = 0; a < 3; ++a) vert[a] = m.tri[3 * (int64_t)t + a];
    for (int l = 0; l < m.nlayers; ++l) {
      node_dofs(m, l, vert, dofs);
      for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) rows[dofs[i]].push_back((int32_t)dofs[j]);
    }
  }
  int64_t total = 0;
  for (auto& r : rows) {
    std::sort(r.begin(), r.end());
    total += std::unique(r.begin(), r.end()) - r.begin();
  }
  *nnz = total;
  return 0;
}

// Fill rowptr [ndof + 1] and colidx [nnz] (sorted columns per row).
int oracle_pattern(const oracle_mesh* d, int64_t* rowptr, int32_t* colidx) {
  const Mesh m = unpack(d);
  if (!mesh_ok(m)) return 1;
  const int64_t ndof = 2 * (int64_t)m.nv * (m.nlayers + 1);
  std::vector<std::vector<int32_t>> rows(ndof);
  for (int t = 0; t < m.ntri; ++t) {
    int64_t vert[3], dofs[12];
    for (int a = 0; a < 3; ++a) vert[a] = m.tri[3 * (int64_t)t + a];
    for (int l = 0; l < m.nlayers; ++l) {
      node_dofs(m, l, vert, dofs);
      for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) rows[dofs[i]].push_back((int32_t)dofs[j]);
    }
  }
  rowptr[0] = 0;
  for (int64_t r = 0; r < ndof; ++r) {
    auto& v = rows[r];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    std::copy(v.begin(), v.end(), colidx + rowptr[r]);
    rowptr[r + 1] = rowptr[r] + (int64_t)v.size();
    std::vector<int32_t>().swap(v);
  }
  return 0;
}

}  // extern "C"

namespace {
// The wedges of one column (base triangle t), bottom to top: 12-lane dual residual, element matrix
// added into the CSR values, element residual into R (nullable).  Returns 2 if the pattern lacks an
// entry the element needs.
int jacobian_column(const Mesh& m, int t, const double* U, const int64_t* rowptr, const int32_t* colidx,
                    double* vals, double* R) {
  int64_t vert[3];
  for (int a = 0; a < 3; ++a) vert[a] = m.tri[3 * (int64_t)t + a];
  for (int l = 0; l < m.nlayers; ++l) {
    double Ue[12], Re[12], Ke[144];
    int64_t dofs[12];
    gather_element(m, l, vert, U, Ue);
    Dual Ud[12], Rd[12];
    for (int j = 0; j < 12; ++j) {
      Ud[j] = dconst(Ue[j]);
      Ud[j].d[j] = 1.0;
    }
    element_residual<Dual>(m, t, l, Ud, Rd);
    for (int i = 0; i < 12; ++i) {
      Re[i] = Rd[i].v;
      for (int j = 0; j < 12; ++j) Ke[12 * i + j] = Rd[i].d[j];
    }
    node_dofs(m, l, vert, dofs);
    for (int i = 0; i < 12; ++i) {
      if (R) R[dofs[i]] += Re[i];
      const int32_t* b = colidx + rowptr[dofs[i]];
      const int32_t* e = colidx + rowptr[dofs[i] + 1];
      for (int j = 0; j < 12; ++j) {
        const int32_t* p = std::lower_bound(b, e, (int32_t)dofs[j]);
        if (p == e || *p != dofs[j]) return 2;  // pattern does not hold this entry
        vals[p - colidx] += Ke[12 * i + j];
      }
    }
  }
  return 0;
}

// Greedy colouring of the base triangles: each triangle, in index order, takes the smallest colour
// that no earlier triangle sharing one of its vertices has.  Triangles of one colour share no
// vertex, so their columns write disjoint rows.
std::vector<std::vector<int>> triangle_colours(const Mesh& m) {
  std::vector<std::vector<int>> vert_cols(m.nv);
  std::vector<std::vector<int>> classes;
  for (int t = 0; t < m.ntri; ++t) {
    int c = 0;
    for (;; ++c) {
      bool used = false;
      for (int a = 0; a < 3 && !used; ++a)
        for (int u : vert_cols[m.tri[3 * (int64_t)t + a]]) used |= (u == c);
      if (!used) break;
    }
    if (c == (int)classes.size()) classes.emplace_back();
    classes[c].push_back(t);
    for (int a = 0; a < 3; ++a) vert_cols[m.tri[3 * (int64_t)t + a]].push_back(c);
  }
  return classes;
}
}  // namespace

extern "C" {

// Jacobian values on the given pattern (overwritten) and, if R != NULL, the residual.
int oracle_jacobian(const oracle_mesh* d, const double* U, const uint8_t* tri_mask,
                    const int64_t* rowptr, const int32_t* colidx, double* vals, double* R) {
  const Mesh m = unpack(d);
  if (!mesh_ok(m)) return 1;
  const int64_t ndof = 2 * (int64_t)m.nv * (m.nlayers + 1);
  std::memset(vals, 0, sizeof(double) * rowptr[ndof]);
  if (R) std::memset(R, 0, sizeof(double) * ndof);
  for (int t = 0; t < m.ntri; ++t) {
    if (tri_mask && !tri_mask[t]) continue;
    const int rc = jacobian_column(m, t, U, rowptr, colidx, vals, R);
    if (rc) return rc;
  }
  if (R) lateral_load(m, tri_mask, R);
  return 0;
}

// The same Jacobian and residual with the columns taken colour by colour (oracle's own greedy
// colouring), the columns of one colour split among `nthreads` std::threads.  Every matrix entry
// and residual row receives its contributions in colour order whatever nthreads is, so the result
// is bitwise the same for every thread count (it differs from oracle_jacobian only in the order of
// the additions).  Used to time the oracle on all host cores.
int oracle_jacobian_colored(const oracle_mesh* d, const double* U, const int64_t* rowptr,
                            const int32_t* colidx, double* vals, double* R, int nthreads) {
  const Mesh m = unpack(d);
  if (!mesh_ok(m) || nthreads < 1) return 1;
  const int64_t ndof = 2 * (int64_t)m.nv * (m.nlayers + 1);
  std::memset(vals, 0, sizeof(double) * rowptr[ndof]);
  if (R) std::memset(R, 0, sizeof(double) * ndof);
  const std::vector<std::vector<int>> classes = triangle_colours(m);
  std::atomic<int> status{0};
  for (const std::vector<int>& cls : classes) {
    const int64_t n = (int64_t)cls.size();
    const int nt = (int)std::min<int64_t>(nthreads, n);
    std::vector<std::thread> pool;
    for (int k = 0; k < nt; ++k) {
      pool.emplace_back([&, k]() {
        for (int64_t i = n * k / nt; i < n * (k + 1) / nt; ++i) {
          const int rc = jacobian_column(m, cls[i], U, rowptr, colidx, vals, R);
          if (rc) status.store(rc);
        }
      });
    }
    for (std::thread& th : pool) th.join();
    if (status.load()) return status.load();
  }
  if (R) lateral_load(m, nullptr, R);
  return 0;
}

// Discrete energy Pi_h(U) whose gradient is the residual (same quadrature):
//   sum_q w detJ [A^(-1/n) 2n/(n+1) (eps_e^2 + delta)^((n+1)/(2n)) + rho g grad s . (u, v)]
//   + sum_bed_q w |J_b| beta |u|^2 / 2
// (The paper does not write the energy; it follows from Eq. effvisc / effeps because
//  d(eps_e^2) along phi_i e_x equals eps_1 . grad phi_i.)
double oracle_energy(const oracle_mesh* d, const double* U) {
  const Mesh m = unpack(d);
  if (!mesh_ok(m)) return NAN;
  const double pexp = (m.n + 1.0) / (2.0 * m.n);
  const double cn = 2.0 * m.n / (m.n + 1.0);
  double total = 0.0;
  for (int t = 0; t < m.ntri; ++t) {
    int64_t vert[3];
    for (int a = 0; a < 3; ++a) vert[a] = m.tri[3 * (int64_t)t + a];
    for (int l = 0; l < m.nlayers; ++l) {
      double X[6][3], Ue[12];
      wedge_nodes(m, t, l, vert, X);
      gather_element(m, l, vert, U, Ue);
      for (int q = 0; q < 6; ++q) {
        double xi, eta, zeta, w, N[6], gN[6][3], detJ;
        qp_ref(q, &xi, &eta, &zeta, &w);
        phys_basis(X, xi, eta, zeta, N, gN, &detJ);
        double gu[3] = {0, 0, 0}, gv[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, uq = 0, vq = 0;
        for (int i = 0; i < 6; ++i) {
          uq += N[i] * Ue[2 * i];
          vq += N[i] * Ue[2 * i + 1];
          for (int r = 0; r < 3; ++r) {
            gu[r] += gN[i][r] * Ue[2 * i];
            gv[r] += gN[i][r] * Ue[2 * i + 1];
            gs[r] += gN[i][r] * (m.bed[vert[i % 3]] + m.thick[vert[i % 3]]);
          }
        }
        const double e2 = effective_strain2(gu, gv);
        const double coef = hardness(m, vert, l, N) * cn;
        total += w * detJ * (coef * std::pow(e2 + m.delta, pexp) + m.rho * m.g * (gs[0] * uq + gs[1] * vq));
      }
      if (l == 0) {
        double e1[3], e2v[3], cr[3];
        for (int r = 0; r < 3; ++r) {
          e1[r] = X[1][r] - X[0][r];
          e2v[r] = X[2][r] - X[0][r];
        }
        cr[0] = e1[1] * e2v[2] - e1[2] * e2v[1];
        cr[1] = e1[2] * e2v[0] - e1[0] * e2v[2];
        cr[2] = e1[0] * e2v[1] - e1[1] * e2v[0];
        const double area2 = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        for (int q = 0; q < 3; ++q) {
          const double lam[3] = {1.0 - kTriQp[q][0] - kTriQp[q][1], kTriQp[q][0], kTriQp[q][1]};
          double bq = 0, uq = 0, vq = 0;
          for (int a = 0; a < 3; ++a) {
            bq += lam[a] * m.beta[vert[a]];
            uq += lam[a] * Ue[2 * a];
            vq += lam[a] * Ue[2 * a + 1];
          }
          total += kTriW * area2 * 0.5 * bq * (uq * uq + vq * vq);
        }
      }
    }
  }
  if (m.margin == 1) {  // the margin load is constant: its energy is F_lat . U
    const int64_t ndof = 2 * (int64_t)m.nv * (m.nlayers + 1);
    std::vector<double> F(ndof, 0.0);
    lateral_load(m, nullptr, F.data());
    for (int64_t i = 0; i < ndof; ++i) total += F[i] * U[i];
  }
  return total;
}

// Shallow-ice + sliding initial guess (not in the paper; textbook SIA):
//   u(z) = -(2A/(n+1)) (rho g)^n |grad s|^(n-1) grad s (H^(n+1) - (s - z)^(n+1)) - rho g H grad s / beta
// with the nodal surface gradient = area-weighted mean of the P1 gradients of the
// triangles around the vertex.
int oracle_sia(const oracle_mesh* d, double* U) {
  const Mesh m = unpack(d);
  if (!mesh_ok(m)) return 1;
  std::vector<double> gsx(m.nv, 0.0), gsy(m.nv, 0.0), wsum(m.nv, 0.0);
  for (int t = 0; t < m.ntri; ++t) {
    int64_t v[3];
    double x[3], y[3], s[3];
    for (int a = 0; a < 3; ++a) {
      v[a] = m.tri[3 * (int64_t)t + a];
      x[a] = m.xy[2 * v[a]];
      y[a] = m.xy[2 * v[a] + 1];
      s[a] = m.bed[v[a]] + m.thick[v[a]];
    }
    // P1 gradient by solving the 2x2 system of the two edge differences
    const double ax = x[1] - x[0], ay = y[1] - y[0], bx = x[2] - x[0], by = y[2] - y[0];
    const double det = ax * by - ay * bx;
    const double ds1 = s[1] - s[0], ds2 = s[2] - s[0];
    const double sx = (ds1 * by - ds2 * ay) / det;
    const double sy = (ax * ds2 - bx * ds1) / det;
    const double area = 0.5 * det;
    for (int a = 0; a < 3; ++a) {
      gsx[v[a]] += area * sx;
      gsy[v[a]] += area * sy;
      wsum[v[a]] += area;
    }
  }
  const double rg = m.rho * m.g;
  for (int a = 0; a < m.nv; ++a) {
    const double sx = gsx[a] / wsum[a], sy = gsy[a] / wsum[a];
    const double gnorm = std::sqrt(sx * sx + sy * sy);
    const double H = m.thick[a], s = m.bed[a] + H;
    for (int l = 0; l <= m.nlayers; ++l) {
      const double z = m.bed[a] + m.sigma[l] * H;
      const double depth = s - z;
      const double def = 2.0 * m.A / (m.n + 1.0) * std::pow(rg, m.n) * std::pow(gnorm, m.n - 1.0) *
                         (std::pow(H, m.n + 1.0) - std::pow(depth, m.n + 1.0));
      const double slide = rg * H / m.beta[a];
      U[dof_index(m, a, l, 0)] = -(def + slide) * sx;
      U[dof_index(m, a, l, 1)] = -(def + slide) * sy;
    }
  }
  return 0;
}

}  // extern "C"
