// Smoothed-aggregation hierarchy for the two-point Poisson operator (see amg_host.h).
#include "amg_host.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <unordered_map>

namespace fvgb {
namespace {

// C = A * B (Gustavson, dense accumulator per row; column order of each row: first touch).
HostCsr spgemm(const HostCsr& A, const HostCsr& B) {
  HostCsr C;
  C.n = A.n;
  C.m = B.m;
  C.ptr.assign(A.n + 1, 0);
  std::vector<int64_t> mark(B.m, -1);
  std::vector<double> acc(B.m, 0.0);
  std::vector<int32_t> cols;
  for (int64_t i = 0; i < A.n; ++i) {
    cols.clear();
    for (int64_t a = A.ptr[i]; a < A.ptr[i + 1]; ++a) {
      const int32_t k = A.idx[a];
      const double av = A.val[a];
      for (int64_t b = B.ptr[k]; b < B.ptr[k + 1]; ++b) {
        const int32_t j = B.idx[b];
        if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; cols.push_back(j); }
        acc[j] += av * B.val[b];
      }
    }
    for (int32_t j : cols) { C.idx.push_back(j); C.val.push_back(acc[j]); }
    C.ptr[i + 1] = (int64_t)C.idx.size();
  }
  return C;
}

HostCsr transpose(const HostCsr& A) {
  HostCsr T;
  T.n = A.m;
  T.m = A.n;
  T.ptr.assign(A.m + 1, 0);
  for (int32_t j : A.idx) T.ptr[j + 1]++;
  for (int64_t j = 0; j < A.m; ++j) T.ptr[j + 1] += T.ptr[j];
  T.idx.resize(A.idx.size());
  T.val.resize(A.val.size());
  std::vector<int64_t> pos(T.ptr.begin(), T.ptr.end() - 1);
  for (int64_t i = 0; i < A.n; ++i)
    for (int64_t a = A.ptr[i]; a < A.ptr[i + 1]; ++a) {
      const int64_t q = pos[A.idx[a]]++;
      T.idx[q] = (int32_t)i;
      T.val[q] = A.val[a];
    }
  return T;
}

struct KeyHash {
  size_t operator()(const std::array<int64_t, 4>& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int64_t v : k) { h ^= (uint64_t)v; h *= 1099511628211ull; }
    return (size_t)h;
  }
};

}  // namespace

std::string amg_build(int dim, int64_t N, const int32_t* nbr4, const double* coef4,
                      const double* diag, const double* cen, const double* vol,
                      const std::vector<int64_t>& part_begin, AmgHost& out) {
  out = AmgHost();
  if (N <= 0) return "empty mesh";
  // level-0 operator in CSR
  HostCsr A;
  A.n = A.m = N;
  A.ptr.assign(N + 1, 0);
  for (int64_t i = 0; i < N; ++i) {
    A.idx.push_back((int32_t)i);
    A.val.push_back(diag[i]);
    for (int k = 0; k < 4; ++k) {
      const int32_t j = nbr4[4 * i + k];
      const double c = coef4[4 * i + k];
      if (j == i || c == 0.0) continue;
      A.idx.push_back(j);
      A.val.push_back(-c);
    }
    A.ptr[i + 1] = (int64_t)A.idx.size();
  }
  // unknown positions and parts
  std::vector<double> pts(dim * N);
  for (int a = 0; a < dim; ++a)
    for (int64_t i = 0; i < N; ++i) pts[dim * i + a] = cen[a * N + i];
  std::vector<int32_t> part(N);
  for (size_t p = 0; p + 1 < part_begin.size(); ++p)
    for (int64_t i = part_begin[p]; i < part_begin[p + 1]; ++i) part[i] = (int32_t)p;
  double vsum = 0.0;
  for (int64_t i = 0; i < N; ++i) vsum += vol[i];
  double s = std::pow((dim == 3 ? 6.0 : 4.0) * vsum / (double)N, 1.0 / dim) * 1.01;
  const double w = 2.0 / 3.0;
  int64_t n = N;
  for (int lev = 0; n > kAmgCoarseMax; ++lev) {
    if (lev >= 24) return "multigrid coarsening did not reach the coarse size";
    double lo[3] = {1e300, 1e300, 1e300};
    for (int64_t i = 0; i < n; ++i)
      for (int a = 0; a < dim; ++a) lo[a] = std::min(lo[a], pts[dim * i + a]);
    // aggregates: cubes of side s per part, numbered in order of first appearance
    std::vector<int32_t> agg(n);
    std::unordered_map<std::array<int64_t, 4>, int32_t, KeyHash> id;
    id.reserve((size_t)(n / 4 + 16));
    int32_t nc = 0;
    for (int64_t i = 0; i < n; ++i) {
      std::array<int64_t, 4> key{part[i], 0, 0, 0};
      for (int a = 0; a < dim; ++a) key[1 + a] = (int64_t)std::floor((pts[dim * i + a] - lo[a]) / s);
      auto it = id.find(key);
      if (it == id.end()) it = id.emplace(key, nc++).first;
      agg[i] = it->second;
    }
    if ((double)nc > 0.8 * (double)n) {   // no coarsening at this size: widen the cubes
      s *= 2.0;
      --lev;
      continue;
    }
    // smoothed interpolation P = (I - w D^-1 A) P_t
    AmgHostLevel L;
    L.dinv.resize(n);
    HostCsr Pm;
    Pm.n = n;
    Pm.m = nc;
    Pm.ptr.assign(n + 1, 0);
    {
      std::vector<int64_t> mark(nc, -1);
      std::vector<double> acc(nc, 0.0);
      std::vector<int32_t> cols;
      for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t a = A.ptr[i]; a < A.ptr[i + 1]; ++a)
          if (A.idx[a] == i) d += A.val[a];
        if (!(d > 0.0)) return "non-positive diagonal in the multigrid hierarchy";
        L.dinv[i] = 1.0 / d;
        cols.clear();
        mark[agg[i]] = i; acc[agg[i]] = 1.0; cols.push_back(agg[i]);
        for (int64_t a = A.ptr[i]; a < A.ptr[i + 1]; ++a) {
          const int32_t J = agg[A.idx[a]];
          if (mark[J] != i) { mark[J] = i; acc[J] = 0.0; cols.push_back(J); }
          acc[J] -= w * L.dinv[i] * A.val[a];
        }
        for (int32_t J : cols) { Pm.idx.push_back(J); Pm.val.push_back(acc[J]); }
        Pm.ptr[i + 1] = (int64_t)Pm.idx.size();
      }
    }
    HostCsr Rm = transpose(Pm);
    HostCsr Ac = spgemm(Rm, spgemm(A, Pm));
    // coarse positions (aggregate centroids) and parts
    std::vector<double> cp(dim * nc, 0.0);
    std::vector<int32_t> cnt(nc, 0), cpart(nc, 0);
    for (int64_t i = 0; i < n; ++i) {
      for (int a = 0; a < dim; ++a) cp[dim * agg[i] + a] += pts[dim * i + a];
      cnt[agg[i]]++;
      cpart[agg[i]] = part[i];
    }
    for (int32_t J = 0; J < nc; ++J)
      for (int a = 0; a < dim; ++a) cp[dim * J + a] /= cnt[J];
    L.A = std::move(A);
    L.P = std::move(Pm);
    L.R = std::move(Rm);
    out.levels.push_back(std::move(L));
    A = std::move(Ac);
    pts.swap(cp);
    part.swap(cpart);
    n = nc;
    s *= 2.0;
  }
  // dense inverse of the coarsest operator (Cholesky, then the inverse column by column)
  out.coarse = A;
  std::vector<double> M(n * n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t a = A.ptr[i]; a < A.ptr[i + 1]; ++a) M[i * n + A.idx[a]] += A.val[a];
  std::vector<double> Lc(n * n, 0.0);
  for (int64_t j = 0; j < n; ++j) {
    double d = M[j * n + j];
    for (int64_t k = 0; k < j; ++k) d -= Lc[j * n + k] * Lc[j * n + k];
    if (!(d > 0.0)) return "coarsest multigrid operator is not positive definite";
    const double ljj = std::sqrt(d);
    Lc[j * n + j] = ljj;
    for (int64_t i = j + 1; i < n; ++i) {
      double v = M[i * n + j];
      for (int64_t k = 0; k < j; ++k) v -= Lc[i * n + k] * Lc[j * n + k];
      Lc[i * n + j] = v / ljj;
    }
  }
  out.coarse_inv.assign(n * n, 0.0);
  std::vector<double> y(n);
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t i = 0; i < n; ++i) {          // L y = e_c
      double v = i == c ? 1.0 : 0.0;
      for (int64_t k = 0; k < i; ++k) v -= Lc[i * n + k] * y[k];
      y[i] = v / Lc[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {     // L^T x = y
      double v = y[i];
      for (int64_t k = i + 1; k < n; ++k) v -= Lc[k * n + i] * out.coarse_inv[k * n + c];
      out.coarse_inv[i * n + c] = v / Lc[i * n + i];
    }
  }
  return "";
}

}  // namespace fvgb
