// Host-side mesh preprocessing in FP64 (see mesh_host.h).
//
// Readings of the paper applied here (Section 2.1 of arXiv 2203.00925):
//  * cell centre = centre of gravity = vertex mean of the simplex; mu_i its measure;
//  * face area vector S_f = |sigma_f| n_f, oriented from the owner L to the other
//    cell R (outwards on the boundary); L is the smaller internal cell index;
//  * node neighbours of a cell (Algorithm "grad") = the set of cells sharing at least
//    one vertex with it; Dirichlet boundary faces sharing a vertex add one point at the
//    face centroid ("ghost cells neighbour by node"); the normal matrix is
//    M_i = sum d d^T with d = x_j - x_i;
//  * vertex weights (Algorithm "ls") = unweighted linear least-squares fit over the
//    cells around the vertex, the mean when fewer than dim+1 cells or when the
//    centred scatter C of their centres has det C / (tr C / dim)^dim < 1e-10;
//  * diamond coefficients (eq. "diamond"): c = G^{-T} S_f with the rows of G the edge
//    vectors e1 = x_R - x_L (x_R = face centroid on the boundary), e2 = x_A - x_C,
//    e3 = x_B - x_C (2D: e2 = x_B - x_A), so that grad u_f . S_f = c . du;
//  * two-point part A_T of the Poisson operator: coefficient c1 per face.
#include "mesh_host.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <limits>
#include <numeric>

namespace fvgb {
namespace {

constexpr int kEINVAL = 1, kEMESH = 2;
constexpr double kDegenerateRatio = 1e-10;

uint64_t spread3(uint64_t v) {
  v &= 0x1fffffULL;
  v = (v | v << 32) & 0x1f00000000ffffULL;
  v = (v | v << 16) & 0x1f0000ff0000ffULL;
  v = (v | v << 8) & 0x100f00f00f00f00fULL;
  v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
  v = (v | v << 2) & 0x1249249249249249ULL;
  return v;
}

uint64_t spread2(uint64_t v) {
  v &= 0xffffffffULL;
  v = (v | v << 16) & 0x0000ffff0000ffffULL;
  v = (v | v << 8) & 0x00ff00ff00ff00ffULL;
  v = (v | v << 4) & 0x0f0f0f0f0f0f0f0fULL;
  v = (v | v << 2) & 0x3333333333333333ULL;
  v = (v | v << 1) & 0x5555555555555555ULL;
  return v;
}

// Solve the n x n system A y = b (row-major A, n <= 4) by Gaussian elimination with
// partial pivoting. Returns false on an exactly singular pivot.
bool gauss_solve(int n, double* A, double* b) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int r = k + 1; r < n; ++r)
      if (std::fabs(A[r * n + k]) > std::fabs(A[p * n + k])) p = r;
    if (A[p * n + k] == 0.0) return false;
    if (p != k) {
      for (int c = 0; c < n; ++c) std::swap(A[k * n + c], A[p * n + c]);
      std::swap(b[k], b[p]);
    }
    for (int r = k + 1; r < n; ++r) {
      double f = A[r * n + k] / A[k * n + k];
      for (int c = k; c < n; ++c) A[r * n + c] -= f * A[k * n + c];
      b[r] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int c = k + 1; c < n; ++c) s -= A[k * n + c] * b[c];
    b[k] = s / A[k * n + k];
  }
  return true;
}

double det_n(int n, const double* M) {
  if (n == 2) return M[0] * M[3] - M[1] * M[2];
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
         M[2] * (M[3] * M[7] - M[4] * M[6]);
}

// Inverse of a symmetric positive definite 2x2 / 3x3 matrix by the adjugate, packed
// as (xx, xy, yy) or (xx, xy, xz, yy, yz, zz). Returns false when det <= 0.
bool sym_inverse(int d, const double* M, double* out) {
  double det = det_n(d, M);
  if (!(det > 0.0)) return false;
  if (d == 2) {
    out[0] = M[3] / det;
    out[1] = -M[1] / det;
    out[2] = M[0] / det;
    return true;
  }
  double a = M[0], b = M[1], c = M[2], e = M[4], f = M[5], i = M[8];
  out[0] = (e * i - f * f) / det;
  out[1] = (c * f - b * i) / det;
  out[2] = (b * f - c * e) / det;
  out[3] = (a * i - c * c) / det;
  out[4] = (b * c - a * f) / det;
  out[5] = (a * e - b * b) / det;
  return true;
}

struct FaceRec {
  int32_t v[3];     // sorted vertex ids (v[2] = -1 in 2D)
  int32_t c0, k0;   // first cell and its local face index
  int32_t c1, k1;   // second cell (-1 on the boundary)
};

}  // namespace

int build_host_mesh(int dim, int64_t n_vert, const double* xyz_in, int64_t n_cell,
                    const int32_t* cell_vert, int64_t n_bface, const int32_t* bface_vert,
                    const int32_t* bface_tag,
                    const std::vector<std::vector<BCInput>>& bcsets, int reorder,
                    HostMesh& m, std::string& err, const int32_t* cell_part, int n_part) {
  if (dim != 2 && dim != 3) { err = "dim must be 2 or 3"; return kEINVAL; }
  if (n_vert <= 0 || n_cell <= 0 || n_bface <= 0 || !xyz_in || !cell_vert || !bface_vert ||
      !bface_tag) {
    err = "empty mesh or null input array";
    return kEINVAL;
  }
  if (n_cell > (int64_t)std::numeric_limits<int32_t>::max() / 4 ||
      n_vert > (int64_t)std::numeric_limits<int32_t>::max()) {
    err = "mesh too large for int32 indices";
    return kEINVAL;
  }
  if (reorder != 0 && reorder != 2) { err = "reorder must be 0 (none) or 2 (Morton)"; return kEINVAL; }
  if (bcsets.empty()) { err = "at least one boundary-condition set is required"; return kEINVAL; }
  const int d = dim, nv = dim + 1;
  const int64_t N = n_cell, V = n_vert;
  m.dim = d;
  m.N = N;
  m.V = V;

  for (int64_t i = 0; i < N * nv; ++i)
    if (cell_vert[i] < 0 || cell_vert[i] >= V) { err = "cell vertex index out of range"; return kEMESH; }
  for (int64_t i = 0; i < n_bface * d; ++i)
    if (bface_vert[i] < 0 || bface_vert[i] >= V) { err = "boundary face vertex index out of range"; return kEMESH; }

  // ---- orientation and centres in the caller's order --------------------------------
  std::vector<double> ucen((size_t)N * d);
  int64_t bad = -1;
#pragma omp parallel for reduction(max : bad)
  for (int64_t c = 0; c < N; ++c) {
    const int32_t* cv = cell_vert + c * nv;
    double E[9];
    for (int k = 0; k < d; ++k)
      for (int a = 0; a < d; ++a) E[k * d + a] = xyz_in[(int64_t)cv[k + 1] * d + a] - xyz_in[(int64_t)cv[0] * d + a];
    if (!(det_n(d, E) > 0.0)) bad = std::max(bad, c);
    for (int a = 0; a < d; ++a) {
      double s = 0.0;
      for (int k = 0; k < nv; ++k) s += xyz_in[(int64_t)cv[k] * d + a];
      ucen[c * d + a] = s / nv;
    }
  }
  if (bad >= 0) { err = "cell " + std::to_string(bad) + " has non-positive orientation"; return kEMESH; }

  // ---- parts (independent meshes packed together) -------------------------------------
  if (n_part < 1) { err = "n_part must be >= 1"; return kEINVAL; }
  std::vector<int32_t> part(N, 0);
  if (cell_part) {
    for (int64_t c = 0; c < N; ++c) {
      if (cell_part[c] < 0 || cell_part[c] >= n_part) { err = "cell part id out of range"; return kEINVAL; }
      part[c] = cell_part[c];
      if (reorder == 0 && c > 0 && part[c] < part[c - 1]) {
        err = "without reordering the parts must be contiguous and in order";
        return kEINVAL;
      }
    }
  }

  // ---- cell order ---------------------------------------------------------------------
  m.cell_perm.resize(N);
  std::iota(m.cell_perm.begin(), m.cell_perm.end(), 0);
  if (reorder == 2) {
    // Morton key of the centre inside the bounding box of its part's centres
    std::vector<double> lo((size_t)n_part * 3, 1e300), hi((size_t)n_part * 3, -1e300);
    for (int64_t c = 0; c < N; ++c)
      for (int a = 0; a < d; ++a) {
        lo[part[c] * 3 + a] = std::min(lo[part[c] * 3 + a], ucen[c * d + a]);
        hi[part[c] * 3 + a] = std::max(hi[part[c] * 3 + a], ucen[c * d + a]);
      }
    std::vector<uint64_t> key(N);
    const double levels = d == 3 ? 2097151.0 : 4294967295.0;
#pragma omp parallel for
    for (int64_t c = 0; c < N; ++c) {
      uint64_t k = 0;
      for (int a = 0; a < d; ++a) {
        const double l = lo[part[c] * 3 + a], h = hi[part[c] * 3 + a];
        double span = h > l ? h - l : 1.0;
        uint64_t q = (uint64_t)std::llround((ucen[c * d + a] - l) / span * levels);
        k |= (d == 3 ? spread3(q) : spread2(q)) << a;
      }
      key[c] = k;
    }
    std::stable_sort(m.cell_perm.begin(), m.cell_perm.end(), [&](int32_t x, int32_t y) {
      if (part[x] != part[y]) return part[x] < part[y];
      return key[x] < key[y];
    });
  }
  m.part_cell_begin.assign(n_part + 1, 0);
  for (int64_t c = 0; c < N; ++c) m.part_cell_begin[part[c] + 1]++;
  for (int q = 0; q < n_part; ++q) {
    if (m.part_cell_begin[q + 1] == 0) { err = "part " + std::to_string(q) + " has no cells"; return kEINVAL; }
    m.part_cell_begin[q + 1] += m.part_cell_begin[q];
  }

  // ---- vertex order: first touch in the new cell order --------------------------------
  std::vector<int32_t> vnew(V, -1);
  m.vert_perm.clear();
  m.vert_perm.reserve(V);
  for (int64_t i = 0; i < N; ++i) {
    const int32_t* cv = cell_vert + (int64_t)m.cell_perm[i] * nv;
    for (int k = 0; k < nv; ++k)
      if (vnew[cv[k]] < 0) { vnew[cv[k]] = (int32_t)m.vert_perm.size(); m.vert_perm.push_back(cv[k]); }
  }
  if ((int64_t)m.vert_perm.size() != V) { err = "a vertex is not used by any cell"; return kEMESH; }
  m.xyz.resize((size_t)V * d);
  for (int64_t v = 0; v < V; ++v)
    for (int a = 0; a < d; ++a) m.xyz[v * d + a] = xyz_in[(int64_t)m.vert_perm[v] * d + a];
  m.cells.resize((size_t)N * nv);
  for (int64_t i = 0; i < N; ++i)
    for (int k = 0; k < nv; ++k) m.cells[i * nv + k] = vnew[cell_vert[(int64_t)m.cell_perm[i] * nv + k]];

  // ---- centres and measures -------------------------------------------------------------
  m.cen.assign((size_t)d * N, 0.0);
  m.vol.resize(N);
  const double inv_fact = d == 3 ? 1.0 / 6.0 : 0.5;
#pragma omp parallel for
  for (int64_t i = 0; i < N; ++i) {
    const int32_t* cv = &m.cells[i * nv];
    double E[9];
    for (int k = 0; k < d; ++k)
      for (int a = 0; a < d; ++a) E[k * d + a] = m.xyz[(int64_t)cv[k + 1] * d + a] - m.xyz[(int64_t)cv[0] * d + a];
    m.vol[i] = det_n(d, E) * inv_fact;
    for (int a = 0; a < d; ++a) {
      double s = 0.0;
      for (int k = 0; k < nv; ++k) s += m.xyz[(int64_t)cv[k] * d + a];
      m.cen[a * N + i] = s / nv;
    }
  }

  // ---- faces: bucket the (cell, local face) records by smallest vertex ----------------
  std::vector<int64_t> bstart(V + 1, 0);
  auto local_face = [&](int64_t i, int k, int32_t* key) {
    int n = 0;
    for (int j = 0; j < nv; ++j)
      if (j != k) key[n++] = m.cells[i * nv + j];
    std::sort(key, key + d);
    if (d == 2) key[2] = -1;
  };
  for (int64_t i = 0; i < N; ++i)
    for (int k = 0; k < nv; ++k) {
      int32_t key[3];
      local_face(i, k, key);
      bstart[key[0] + 1]++;
    }
  for (int64_t v = 0; v < V; ++v) bstart[v + 1] += bstart[v];
  struct Ent { int32_t b, c, cell, k; };
  std::vector<Ent> ents((size_t)N * nv);
  {
    std::vector<int64_t> fill(bstart.begin(), bstart.end() - 1);
    for (int64_t i = 0; i < N; ++i)
      for (int k = 0; k < nv; ++k) {
        int32_t key[3];
        local_face(i, k, key);
        ents[fill[key[0]]++] = Ent{key[1], key[2], (int32_t)i, k};
      }
  }
  std::vector<FaceRec> faces;
  faces.reserve((size_t)N * nv / 2 + 16);
  bool nonmanifold = false;
  for (int64_t v = 0; v < V; ++v) {
    auto b0 = ents.begin() + bstart[v], b1 = ents.begin() + bstart[v + 1];
    std::sort(b0, b1, [](const Ent& x, const Ent& y) {
      if (x.b != y.b) return x.b < y.b;
      if (x.c != y.c) return x.c < y.c;
      return x.cell < y.cell;
    });
    for (auto it = b0; it != b1;) {
      auto jt = it + 1;
      while (jt != b1 && jt->b == it->b && jt->c == it->c) ++jt;
      int64_t cnt = jt - it;
      if (cnt > 2) nonmanifold = true;
      FaceRec f;
      f.v[0] = (int32_t)v; f.v[1] = it->b; f.v[2] = it->c;
      f.c0 = it->cell; f.k0 = it->k;
      f.c1 = cnt == 2 ? (it + 1)->cell : -1;
      f.k1 = cnt == 2 ? (it + 1)->k : -1;
      faces.push_back(f);
      it = jt;
    }
  }
  if (nonmanifold) { err = "a face is shared by more than two cells"; return kEMESH; }
  std::stable_sort(faces.begin(), faces.end(), [](const FaceRec& x, const FaceRec& y) {
    bool bx = x.c1 < 0, by = y.c1 < 0;
    if (bx != by) return !bx;  // interior first
    if (x.c0 != y.c0) return x.c0 < y.c0;
    return x.c1 < y.c1;
  });
  const int64_t F = (int64_t)faces.size();
  int64_t Fi = 0;
  while (Fi < F && faces[Fi].c1 >= 0) ++Fi;
  const int64_t Fb = F - Fi;
  m.F = F;
  m.Fi = Fi;
  if (Fb != n_bface) {
    err = "boundary face list has " + std::to_string(n_bface) + " faces, mesh boundary has " +
          std::to_string(Fb);
    return kEMESH;
  }

  m.fL.resize(F); m.fR.resize(F);
  m.fvert.resize((size_t)d * F);
  m.S.resize((size_t)d * F); m.xf.resize((size_t)d * F); m.coef.resize((size_t)d * F);
  m.ftag.assign(F, 0);
  m.cell_face.resize((size_t)nv * N);
  for (int64_t f = 0; f < F; ++f) {
    const FaceRec& r = faces[f];
    m.fL[f] = r.c0;
    m.fR[f] = r.c1;
    for (int a = 0; a < d; ++a) m.fvert[a * F + f] = r.v[a];
    m.cell_face[(int64_t)r.k0 * N + r.c0] = (int32_t)f;
    if (r.c1 >= 0) m.cell_face[(int64_t)r.k1 * N + r.c1] = ~(int32_t)f;
  }

  // ---- face geometry and diamond coefficients -------------------------------------------
  bool degenerate_face = false;
#pragma omp parallel for reduction(|| : degenerate_face)
  for (int64_t f = 0; f < F; ++f) {
    double P[3][3], S[3], xf[3], xL[3], xR[3];
    for (int k = 0; k < d; ++k)
      for (int a = 0; a < d; ++a) P[k][a] = m.xyz[(int64_t)m.fvert[k * F + f] * d + a];
    for (int a = 0; a < d; ++a) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += P[k][a];
      xf[a] = s / d;
      xL[a] = m.cen[a * N + m.fL[f]];
      xR[a] = m.fR[f] >= 0 ? m.cen[a * N + m.fR[f]] : xf[a];
    }
    if (d == 3) {
      double u[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
      double w[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
      S[0] = 0.5 * (u[1] * w[2] - u[2] * w[1]);
      S[1] = 0.5 * (u[2] * w[0] - u[0] * w[2]);
      S[2] = 0.5 * (u[0] * w[1] - u[1] * w[0]);
    } else {
      S[0] = P[1][1] - P[0][1];
      S[1] = -(P[1][0] - P[0][0]);
    }
    double e1[3], dot = 0.0;
    for (int a = 0; a < d; ++a) { e1[a] = xR[a] - xL[a]; dot += e1[a] * S[a]; }
    if (dot < 0.0) { for (int a = 0; a < d; ++a) S[a] = -S[a]; dot = -dot; }
    if (!(dot > 0.0)) degenerate_face = true;
    double c[3] = {0.0, 0.0, 0.0};
    if (d == 3) {
      double e2[3], e3[3];
      for (int a = 0; a < 3; ++a) { e2[a] = P[0][a] - P[2][a]; e3[a] = P[1][a] - P[2][a]; }
      auto cross = [](const double* x, const double* y, double* z) {
        z[0] = x[1] * y[2] - x[2] * y[1];
        z[1] = x[2] * y[0] - x[0] * y[2];
        z[2] = x[0] * y[1] - x[1] * y[0];
      };
      double d1[3], d2[3], d3[3];
      cross(e2, e3, d1); cross(e3, e1, d2); cross(e1, e2, d3);
      double det = e1[0] * d1[0] + e1[1] * d1[1] + e1[2] * d1[2];
      // columns of G^{-1} are the dual vectors (e2 x e3, e3 x e1, e1 x e2) / det
      c[0] = (d1[0] * S[0] + d1[1] * S[1] + d1[2] * S[2]) / det;
      c[1] = (d2[0] * S[0] + d2[1] * S[1] + d2[2] * S[2]) / det;
      c[2] = (d3[0] * S[0] + d3[1] * S[1] + d3[2] * S[2]) / det;
    } else {
      double e2[2] = {P[1][0] - P[0][0], P[1][1] - P[0][1]};
      double det = e1[0] * e2[1] - e1[1] * e2[0];
      c[0] = (e2[1] * S[0] - e2[0] * S[1]) / det;
      c[1] = (-e1[1] * S[0] + e1[0] * S[1]) / det;
    }
    for (int a = 0; a < d; ++a) {
      m.S[a * F + f] = S[a];
      m.xf[a * F + f] = xf[a];
      m.coef[a * F + f] = c[a];
    }
  }
  if (degenerate_face) { err = "degenerate face (zero area or centroids on the face plane)"; return kEMESH; }

  // ---- boundary tags: match the caller's boundary list to the mesh boundary --------------
  {
    struct BKey { int32_t v[3]; int32_t tag; int64_t idx; };
    std::vector<BKey> ub(n_bface), mb(Fb);
    for (int64_t i = 0; i < n_bface; ++i) {
      BKey k;
      for (int a = 0; a < d; ++a) k.v[a] = vnew[bface_vert[i * d + a]];
      std::sort(k.v, k.v + d);
      if (d == 2) k.v[2] = -1;
      k.tag = bface_tag[i];
      k.idx = i;
      ub[i] = k;
    }
    for (int64_t j = 0; j < Fb; ++j) {
      BKey k;
      for (int a = 0; a < 3; ++a) k.v[a] = faces[Fi + j].v[a];
      k.tag = 0;
      k.idx = Fi + j;
      mb[j] = k;
    }
    auto lt = [](const BKey& x, const BKey& y) {
      for (int a = 0; a < 3; ++a) if (x.v[a] != y.v[a]) return x.v[a] < y.v[a];
      return false;
    };
    std::sort(ub.begin(), ub.end(), lt);
    std::sort(mb.begin(), mb.end(), lt);
    for (int64_t j = 0; j < Fb; ++j) {
      if (lt(ub[j], mb[j]) || lt(mb[j], ub[j])) {
        err = "boundary face list does not match the mesh boundary";
        return kEMESH;
      }
      if (ub[j].tag <= 0) { err = "boundary tags must be positive"; return kEMESH; }
      m.ftag[mb[j].idx] = ub[j].tag;
    }
  }

  // ---- cells around each vertex (sorted) -------------------------------------------------
  m.vptr.assign(V + 1, 0);
  for (int64_t i = 0; i < N * nv; ++i) m.vptr[m.cells[i] + 1]++;
  for (int64_t v = 0; v < V; ++v) m.vptr[v + 1] += m.vptr[v];
  m.vcell.resize((size_t)N * nv);
  {
    std::vector<int32_t> fill(m.vptr.begin(), m.vptr.end() - 1);
    for (int64_t i = 0; i < N; ++i)
      for (int k = 0; k < nv; ++k) m.vcell[fill[m.cells[i * nv + k]]++] = (int32_t)i;
  }
  // sum over the cells around each vertex of (x_c - x_A): the multiplicity-weighted
  // gradient's per-vertex geometry
  m.vs1.assign((size_t)d * V, 0.0);
  for (int64_t v = 0; v < V; ++v)
    for (int32_t t = m.vptr[v]; t < m.vptr[v + 1]; ++t)
      for (int a = 0; a < d; ++a) m.vs1[a * V + v] += m.cen[a * N + m.vcell[t]] - m.xyz[v * d + a];

  // ---- node-neighbour sets ----------------------------------------------------------------
  m.nptr.assign(N + 1, 0);
  {
    std::vector<std::vector<int32_t>> lists(N);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < N; ++i) {
      std::vector<int32_t>& L = lists[i];
      for (int k = 0; k < nv; ++k) {
        int32_t v = m.cells[i * nv + k];
        L.insert(L.end(), m.vcell.begin() + m.vptr[v], m.vcell.begin() + m.vptr[v + 1]);
      }
      std::sort(L.begin(), L.end());
      L.erase(std::unique(L.begin(), L.end()), L.end());
      L.erase(std::remove(L.begin(), L.end(), (int32_t)i), L.end());
    }
    for (int64_t i = 0; i < N; ++i) m.nptr[i + 1] = m.nptr[i] + (int32_t)lists[i].size();
    if ((int64_t)m.nptr[N] != (int64_t)m.nptr[N]) { err = "neighbour list too large"; return kEINVAL; }
    m.nidx.resize(m.nptr[N]);
#pragma omp parallel for
    for (int64_t i = 0; i < N; ++i) std::copy(lists[i].begin(), lists[i].end(), m.nidx.begin() + m.nptr[i]);
  }

  // ---- least-squares vertex weights (Algorithm "ls") -------------------------------------
  m.valpha.resize(m.vcell.size());
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < V; ++v) {
    const int32_t b0 = m.vptr[v], b1 = m.vptr[v + 1];
    const int n = b1 - b0;
    const int q = d + 1;
    double XtX[16] = {0}, s1[3] = {0, 0, 0}, C[9] = {0};
    for (int t = b0; t < b1; ++t) {
      double r[4] = {1.0, 0, 0, 0};
      for (int a = 0; a < d; ++a) r[1 + a] = m.cen[a * N + m.vcell[t]] - m.xyz[v * d + a];
      for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b) XtX[a * q + b] += r[a] * r[b];
    }
    bool degenerate = n < d + 1;
    if (!degenerate) {
      for (int a = 0; a < d; ++a) s1[a] = XtX[1 + a];
      double tr = 0.0;
      for (int a = 0; a < d; ++a) {
        for (int b = 0; b < d; ++b) C[a * d + b] = XtX[(1 + a) * q + 1 + b] - s1[a] * s1[b] / n;
        tr += C[a * d + a];
      }
      double scale = std::pow(tr / d, d);
      double ratio = det_n(d, C) / scale;
      degenerate = !(ratio >= kDegenerateRatio);
    }
    double y[4] = {1.0, 0.0, 0.0, 0.0};
    if (!degenerate) {
      double A[16];
      std::copy(XtX, XtX + 16, A);
      degenerate = !gauss_solve(q, A, y);
    }
    for (int t = b0; t < b1; ++t) {
      if (degenerate) { m.valpha[t] = 1.0 / n; continue; }
      double a_ = y[0];
      for (int a = 0; a < d; ++a) a_ += y[1 + a] * (m.cen[a * N + m.vcell[t]] - m.xyz[v * d + a]);
      m.valpha[t] = a_;
    }
  }

  // ---- boundary-condition sets ------------------------------------------------------------
  const int nsym = d == 3 ? 6 : 3;
  m.bcs.resize(bcsets.size());
  for (size_t s = 0; s < bcsets.size(); ++s) {
    BCSetHost& B = m.bcs[s];
    B.bkind.resize(Fb);
    B.bval.assign(Fb, 0.0);
    for (int64_t j = 0; j < Fb; ++j) {
      int32_t tag = m.ftag[Fi + j];
      const BCInput* hit = nullptr;
      for (const BCInput& b : bcsets[s])
        if (b.tag == tag) hit = &b;
      if (!hit) { err = "boundary tag " + std::to_string(tag) + " has no condition in set " + std::to_string(s); return kEMESH; }
      if (hit->kind < 0 || hit->kind > 2) { err = "unknown boundary kind"; return kEINVAL; }
      B.bkind[j] = (int8_t)hit->kind;
      B.bval[j] = hit->kind == 1 ? hit->value : 0.0;
    }
    // Dirichlet vertices: the smallest Dirichlet tag touching a vertex gives its value
    B.vdir.assign(V, std::numeric_limits<double>::quiet_NaN());
    std::vector<int32_t> vtag(V, std::numeric_limits<int32_t>::max());
    std::vector<int32_t> dptr(V + 1, 0);
    int nd = 0;
    for (int64_t j = 0; j < Fb; ++j) {
      if (B.bkind[j] != 1) continue;
      ++nd;
      for (int a = 0; a < d; ++a) {
        int32_t v = m.fvert[a * F + Fi + j];
        dptr[v + 1]++;
        if (m.ftag[Fi + j] < vtag[v]) { vtag[v] = m.ftag[Fi + j]; B.vdir[v] = B.bval[j]; }
      }
    }
    B.n_dirichlet_faces = nd;
    for (int64_t v = 0; v < V; ++v) dptr[v + 1] += dptr[v];
    std::vector<int32_t> dface(dptr[V]);
    {
      std::vector<int32_t> fill(dptr.begin(), dptr.end() - 1);
      for (int64_t j = 0; j < Fb; ++j) {
        if (B.bkind[j] != 1) continue;
        for (int a = 0; a < d; ++a) dface[fill[m.fvert[a * F + Fi + j]]++] = (int32_t)(Fi + j);
      }
    }
    // ghost points per cell: Dirichlet faces sharing a vertex with the cell
    B.gptr.assign(N + 1, 0);
    std::vector<std::vector<int32_t>> gl(N), gm(N);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < N; ++i) {
      for (int k = 0; k < nv; ++k) {
        int32_t v = m.cells[i * nv + k];
        gl[i].insert(gl[i].end(), dface.begin() + dptr[v], dface.begin() + dptr[v + 1]);
      }
      std::sort(gl[i].begin(), gl[i].end());
      // each face appears once per vertex it shares with the cell: keep one, count them
      std::vector<int32_t>& g = gl[i];
      size_t w = 0;
      for (size_t r = 0; r < g.size();) {
        size_t e = r;
        while (e < g.size() && g[e] == g[r]) ++e;
        gm[i].push_back((int32_t)(e - r));
        g[w++] = g[r];
        r = e;
      }
      g.resize(w);
    }
    for (int64_t i = 0; i < N; ++i) B.gptr[i + 1] = B.gptr[i] + (int32_t)gl[i].size();
    B.gface.resize(B.gptr[N]);
    B.gmult.resize(B.gptr[N]);
    for (int64_t i = 0; i < N; ++i) {
      std::copy(gl[i].begin(), gl[i].end(), B.gface.begin() + B.gptr[i]);
      std::copy(gm[i].begin(), gm[i].end(), B.gmult.begin() + B.gptr[i]);
    }
    // inverse normal matrices of the least-squares gradient
    B.minv.resize((size_t)nsym * N);
    B.minv_v.resize((size_t)nsym * N);
    bool singular = false;
#pragma omp parallel for reduction(|| : singular)
    for (int64_t i = 0; i < N; ++i) {
      double M[9] = {0};
      auto add = [&](const double* dx) {
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) M[a * d + b] += dx[a] * dx[b];
      };
      for (int32_t t = m.nptr[i]; t < m.nptr[i + 1]; ++t) {
        double dx[3];
        for (int a = 0; a < d; ++a) dx[a] = m.cen[a * N + m.nidx[t]] - m.cen[a * N + i];
        add(dx);
      }
      for (int32_t t = B.gptr[i]; t < B.gptr[i + 1]; ++t) {
        double dx[3];
        for (int a = 0; a < d; ++a) dx[a] = m.xf[a * F + B.gface[t]] - m.cen[a * N + i];
        add(dx);
      }
      double inv[6];
      if (!sym_inverse(d, M, inv)) { singular = true; continue; }
      for (int k = 0; k < nsym; ++k) B.minv[k * N + i] = inv[k];
      // multiplicity-weighted variant: the stencils around the cell's vertices
      double Mv[9] = {0};
      auto addv = [&](const double* dx, double wgt) {
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) Mv[a * d + b] += wgt * dx[a] * dx[b];
      };
      for (int k = 0; k < nv; ++k) {
        const int32_t v = m.cells[i * nv + k];
        for (int32_t t = m.vptr[v]; t < m.vptr[v + 1]; ++t) {
          const int32_t c = m.vcell[t];
          if (c == i) continue;
          double dx[3];
          for (int a = 0; a < d; ++a) dx[a] = m.cen[a * N + c] - m.cen[a * N + i];
          addv(dx, 1.0);
        }
      }
      for (int32_t t = B.gptr[i]; t < B.gptr[i + 1]; ++t) {
        double dx[3];
        for (int a = 0; a < d; ++a) dx[a] = m.xf[a * F + B.gface[t]] - m.cen[a * N + i];
        addv(dx, (double)B.gmult[t]);
      }
      if (!sym_inverse(d, Mv, inv)) { singular = true; continue; }
      for (int k = 0; k < nsym; ++k) B.minv_v[k * N + i] = inv[k];
    }
    if (singular) { err = "singular least-squares gradient stencil"; return kEMESH; }
    // two-point operator A_T: four slots per cell (cell-major); an unused slot points
    // at the cell itself with coefficient 0 so that the kernel needs no branch
    B.at_nbr.assign((size_t)4 * N, 0);
    B.at_coef.assign((size_t)4 * N, 0.0);
    B.at_diag.assign(N, 0.0);
#pragma omp parallel for
    for (int64_t i = 0; i < N; ++i) {
      double diag = 0.0;
      for (int k = 0; k < 4; ++k) B.at_nbr[i * 4 + k] = (int32_t)i;
      for (int k = 0; k < nv; ++k) {
        int32_t e = m.cell_face[k * N + i];
        int32_t f = e >= 0 ? e : ~e;
        double c1 = m.coef[f];
        if (f < Fi) {
          B.at_nbr[i * 4 + k] = e >= 0 ? m.fR[f] : m.fL[f];
          B.at_coef[i * 4 + k] = c1;
          diag += c1;
        } else if (B.bkind[f - Fi] == 1) {
          diag += c1;
        }
      }
      B.at_diag[i] = diag;
    }
    // symmetric Jacobi scaling (a cell without any coupling keeps scale 1)
    B.at_isd.assign(N, 1.0);
    B.at_scoef.assign((size_t)4 * N, 0.0);
    for (int64_t i = 0; i < N; ++i)
      if (B.at_diag[i] > 0.0) B.at_isd[i] = 1.0 / std::sqrt(B.at_diag[i]);
#pragma omp parallel for
    for (int64_t i = 0; i < N; ++i)
      for (int k = 0; k < 4; ++k)
        B.at_scoef[i * 4 + k] = B.at_coef[i * 4 + k] * B.at_isd[i] * B.at_isd[B.at_nbr[i * 4 + k]];
  }
  return 0;
}

}  // namespace fvgb
