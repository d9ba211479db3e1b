// Host-side mesh preprocessing (FP64): topology, geometry, locality reordering and the
// precomputed operators of the finite-volume method (Section 2.1 of Manapy,
// arXiv 2203.00925). Everything here runs once per mesh upload.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace fvgb {

struct BCSetHost {
  std::vector<int8_t> bkind;      // [Fb] fvgb_bc_kind of every boundary face
  std::vector<double> bval;       // [Fb] Dirichlet value (0 otherwise)
  std::vector<double> minv;       // SoA [nsym][N] inverse of the LS normal matrix M_i
  std::vector<int32_t> gptr;      // [N+1] Dirichlet ghost points of each cell (CSR)
  std::vector<int32_t> gface;     //        boundary face index (global face id)
  std::vector<int32_t> gmult;     //        vertices the face shares with the cell
  std::vector<double> minv_v;     // SoA [nsym][N] inverse of the multiplicity-weighted matrix
  std::vector<double> vdir;       // [V] Dirichlet vertex value, NaN when not Dirichlet
  std::vector<int32_t> at_nbr;    // [N][4] two-point operator: neighbour (the cell itself if none)
  std::vector<double> at_coef;    // [N][4] off-diagonal coefficient c1 (0 if none)
  std::vector<double> at_diag;    // [N]
  // the same operator scaled symmetrically to unit diagonal, D^-1/2 A_T D^-1/2, for the
  // inner CG: at_scoef[i][k] = at_coef[i][k] / sqrt(d_i d_j), at_isd[i] = 1 / sqrt(d_i)
  std::vector<double> at_scoef;   // [N][4]
  std::vector<double> at_isd;     // [N]
  int n_dirichlet_faces = 0;
};

struct HostMesh {
  int dim = 0;
  int64_t N = 0, V = 0, F = 0, Fi = 0;  // faces [0, Fi) interior, [Fi, F) boundary
  std::vector<int32_t> cell_perm;       // internal -> caller's cell index
  std::vector<int32_t> vert_perm;       // internal -> caller's vertex index
  std::vector<double> xyz;              // [V][dim] internal vertex order
  std::vector<int32_t> cells;           // [N][dim+1] internal vertex ids
  std::vector<double> cen;              // SoA [dim][N] centre of gravity
  std::vector<double> vol;              // [N] measure mu_i
  std::vector<int32_t> fL, fR;          // [F] owner / other cell (-1 on the boundary)
  std::vector<int32_t> fvert;           // SoA [dim][F] face vertices A, B(, C)
  std::vector<double> S;                // SoA [dim][F] area vector |sigma| n, L -> R
  std::vector<double> xf;               // SoA [dim][F] face centroid
  std::vector<double> coef;             // SoA [dim][F] diamond coefficients c1, c2(, c3)
  std::vector<int32_t> ftag;            // [F] boundary tag (0 interior)
  std::vector<int32_t> cell_face;       // SoA [dim+1][N]: f if the cell is L, ~f if R
  std::vector<int32_t> nptr, nidx;      // node-neighbour sets (CSR, sorted)
  std::vector<int32_t> vptr, vcell;     // cells around each vertex (CSR, sorted)
  std::vector<double> valpha;           // LS interpolation weight of each (vertex, cell)
  std::vector<double> vs1;              // SoA [dim][V] sum over the cells around A of (x_c - x_A)
  std::vector<BCSetHost> bcs;
  std::vector<int64_t> part_cell_begin; // [P+1] internal cell range of each part
};

struct BCInput {
  int32_t tag;
  int32_t kind;
  double value;
};

// Returns 0 on success, otherwise a fvgb_status code with a message in err.
int build_host_mesh(int dim, int64_t n_vert, const double* xyz, int64_t n_cell,
                    const int32_t* cell_vert, int64_t n_bface, const int32_t* bface_vert,
                    const int32_t* bface_tag,
                    const std::vector<std::vector<BCInput>>& bcsets, int reorder,
                    HostMesh& out, std::string& err, const int32_t* cell_part = nullptr,
                    int n_part = 1);

}  // namespace fvgb
