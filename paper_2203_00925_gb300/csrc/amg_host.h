// Host-side setup of the algebraic-multigrid inner solver of the Poisson refinement loop.
// The paper's Poisson solves (Tables "comp1", "comp2") use FGMRES preconditioned by
// PETSc's smoothed-aggregation multigrid (GAMG); this is a GPU-side counterpart for the
// two-point operator A_T. Plain C++, no CUDA: the library uploads what it builds.
//
// Hierarchy: level 0 is A_T. Each level groups its unknowns into aggregates - cubes of
// side s in the space of the unknowns' positions (cell centres, then aggregate centroids),
// never across the parts of an ensemble - with s chosen so that a fine aggregate holds
// about 6 cells in 3D (4 in 2D) and doubled per level. Tentative interpolation P_t is
// the aggregate indicator, smoothed once by damped Jacobi: P = (I - w D^-1 A) P_t with
// w = 2/3; restriction R = P^T; coarse operator A_c = R A P (Galerkin). The coarsest
// level (at most kAmgCoarseMax unknowns) is inverted densely (Cholesky).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace fvgb {

constexpr int64_t kAmgCoarseMax = 640;

struct HostCsr {
  int64_t n = 0, m = 0;                 // rows, columns
  std::vector<int64_t> ptr;             // [n+1]
  std::vector<int32_t> idx;
  std::vector<double> val;
};

struct AmgHostLevel {
  HostCsr A;                 // operator of this level
  std::vector<double> dinv;  // 1 / diag(A)
  HostCsr P;                 // interpolation from the next level (n x n_next)
  HostCsr R;                 // restriction to the next level (n_next x n) = P^T
};

struct AmgHost {
  std::vector<AmgHostLevel> levels;   // all but the coarsest
  HostCsr coarse;                     // coarsest operator
  std::vector<double> coarse_inv;     // its dense inverse, row-major
};

// The fine operator as the library stores A_T: row i is diag[i] x_i - sum_k coef[i][k]
// x_{nbr[i][k]} (4 slots per row; unused slots hold i with coefficient 0). cen is [dim][N]
// (cell centres), vol [N], part_begin [P+1] the contiguous cell range of every part.
// Returns "" on success, else a message.
std::string amg_build(int dim, int64_t N, const int32_t* nbr4, const double* coef4,
                      const double* diag, const double* cen, const double* vol,
                      const std::vector<int64_t>& part_begin, AmgHost& out);

}  // namespace fvgb
