/*
 * fvgb.h - C ABI of the GB300 finite-volume library (libfvgb.so).
 *
 * The library implements, on one GPU, the per-step hot path of the cell-centred
 * finite-volume method of Manapy (Kissami & Ratnani, arXiv 2203.00925):
 * least-squares cell gradients (Algorithm "grad"), least-squares vertex
 * interpolation (Algorithm "ls"), upwind convective fluxes (eq. 15 with psi = 0),
 * diamond-scheme diffusive fluxes (eq. "diamond"), the face-to-cell gather of eq. 4
 * with the explicit update of eq. 6, and the same face operator used matrix-free as
 * the Poisson operator of eq. 7 / eq. "laplace" inside an iterative solve. The
 * streamer step couples them as in eq. 10.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns an fvgb_status; nothing throws or aborts across the ABI.
 *   fvgb_last_error() gives a message for the last failing call of the thread.
 * - Device arrays (suffix _dev) are owned by the caller, live on the device the mesh
 *   was uploaded on, and are laid out in the mesh's INTERNAL cell order (cells are
 *   reordered for locality at upload). fvgb_mesh_cell_perm / fvgb_permute convert
 *   to and from the caller's order. Vector fields are structure-of-arrays:
 *   [dim][n] with component stride n.
 * - The element type of per-cell transport arrays ("real") is double for a mesh
 *   uploaded with FVGB_FP64 and float for FVGB_FP32 / FVGB_MIXED. Poisson data
 *   (right-hand side f, potential phi) are always double.
 * - stream is a cudaStream_t (NULL = the legacy default stream). Calls are
 *   stream-ordered; a call returns once its work is enqueued, except where it says
 *   that it synchronises the stream.
 * - A mesh handle is not thread-safe: use one handle from one host thread and one
 *   stream at a time.
 * - Asynchronous errors: a transport update (fvgb_fv_residual, fvgb_fv_step, the
 *   transport of fvgb_streamer_step) that writes a non-finite value sets a status word on
 *   the device instead of failing at once; the word stays set until it is reported by
 *   fvgb_sync, by the next fvgb_poisson_solve (or the solve of the next streamer step), or
 *   at the end of a graph-mode fvgb_streamer_step call, each of which returns
 *   FVGB_ENONFINITE and clears it. Grid-wide waits inside the persistent CG kernel are
 *   bounded (1 s) and give FVGB_ETIMEOUT instead of hanging; a wait of the network's
 *   tensor-core kernels for its matrix products (also bounded, 1 s) latches a timeout
 *   in the same status word, reported as FVGB_ETIMEOUT.
 * - Sizes are int64_t; element indices inside the library are int32 (meshes up to
 *   2^31 - 1 cells, faces and neighbour entries).
 */
#ifndef FVGB_H
#define FVGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fvgb_mesh_s* fvgb_mesh;
typedef struct fvgb_mpnn_s* fvgb_mpnn;

typedef enum {
  FVGB_OK = 0,
  FVGB_EINVAL = 1,        /* bad argument (null pointer, size, index, option) */
  FVGB_EMESH = 2,         /* malformed mesh: bad index, non-positive cell, non-manifold
                             face, boundary list not matching the mesh boundary,
                             boundary tag without a condition */
  FVGB_ENOMEM = 3,        /* device or host allocation failed */
  FVGB_ECUDA = 4,         /* a CUDA runtime call failed */
  FVGB_ENOCONV = 5,       /* iterative solve stopped at its iteration limit */
  FVGB_ENONFINITE = 6,    /* NaN or Inf met in a solve */
  FVGB_ETIMEOUT = 7,      /* a bounded device-side wait gave up */
  FVGB_EUNSUPPORTED = 8   /* valid request this build does not implement */
} fvgb_status;

typedef enum { FVGB_FP64 = 0, FVGB_FP32 = 1, FVGB_MIXED = 2 } fvgb_prec;

/* Boundary-condition kinds (Section 4, boundary conditions; annex):
 *  WALL      - no flux of any kind through the face;
 *  DIRICHLET - ghost value g = value at the face centroid (also a least-squares
 *              point of the cells around the face, and the vertex value of every
 *              vertex of the face);
 *  NEUMANN   - homogeneous Neumann: the ghost copies the interior cell (its value
 *              and velocity), no diffusive flux. */
typedef enum { FVGB_BC_WALL = 0, FVGB_BC_DIRICHLET = 1, FVGB_BC_NEUMANN = 2 } fvgb_bc_kind;

typedef struct {
  int32_t tag;      /* boundary tag as given in bface_tag */
  int32_t kind;     /* fvgb_bc_kind */
  double value;     /* Dirichlet value (ignored otherwise) */
} fvgb_bc;

/* One set of boundary conditions: one entry per tag present on the boundary. */
typedef struct {
  int32_t n_bc;
  const fvgb_bc* bc;
} fvgb_bcset;

/* Upload a simplicial mesh and precompute its geometry (Section 2.1: cell centres of
 * gravity, measures mu_i, face area vectors |sigma| n, least-squares matrices and
 * weights of Algorithms "grad" and "ls", diamond coefficients of eq. "diamond").
 *
 *  dim         2 (triangles) or 3 (tetrahedra)
 *  xyz         host, [n_vert][dim] row-major, FP64 coordinates
 *  cell_vert   host, [n_cell][dim+1] vertex ids, positively oriented
 *              (det[x1-x0, x2-x0(, x3-x0)] > 0)
 *  bface_vert  host, [n_bface][dim] vertex ids of every boundary face, any order
 *  bface_tag   host, [n_bface] positive tags
 *  bcsets      n_bcset >= 1 boundary-condition sets; operators name one by index
 *  reorder     0 keep the caller's order, 2 Morton (Z-order) order of cell centres
 *  prec        fvgb_prec of the transport arrays (see conventions)
 *  stream      stream for the uploads; the call synchronises it before returning
 *  out         receives the handle (owned by the caller, release with fvgb_mesh_free)
 * Errors: FVGB_EINVAL, FVGB_EMESH (nothing allocated), FVGB_ENOMEM, FVGB_ECUDA. */
fvgb_status fvgb_mesh_upload(int32_t dim, int64_t n_vert, const double* xyz,
                             int64_t n_cell, const int32_t* cell_vert,
                             int64_t n_bface, const int32_t* bface_vert,
                             const int32_t* bface_tag, int32_t n_bcset,
                             const fvgb_bcset* bcsets, int32_t reorder, int32_t prec,
                             void* stream, fvgb_mesh* out);

/* One mesh of an ensemble (the batched workload: many independent meshes
 * advanced together). Arrays as in fvgb_mesh_upload; bcsets points at n_bcset sets for
 * this mesh (the same number for every mesh; tags are the mesh's own). */
typedef struct {
  int64_t n_vert;
  const double* xyz;
  int64_t n_cell;
  const int32_t* cell_vert;
  int64_t n_bface;
  const int32_t* bface_vert;
  const int32_t* bface_tag;
  const fvgb_bcset* bcsets;
} fvgb_mesh_part;

/* Upload n_part independent meshes as one mesh whose cells, faces and vertices are the
 * meshes' packed one after the other (part p's cells form one contiguous internal range,
 * Morton-ordered within the part). Every operator then runs over all parts in one launch;
 * fvgb_poisson_solve solves every part to its own tolerance (per-part norms, CG scalars and
 * stopping tests); fvgb_streamer_step advances all parts with one time step.
 * Boundary tags must be < 65536 and n_part <= 128. Errors as fvgb_mesh_upload. */
fvgb_status fvgb_mesh_upload_ensemble(int32_t dim, int32_t n_part, const fvgb_mesh_part* parts,
                                      int32_t n_bcset, int32_t reorder, int32_t prec,
                                      void* stream, fvgb_mesh* out);

/* Number of parts (1 for fvgb_mesh_upload) and, when cell_begin is not NULL, the internal
 * cell range of each part: cell_begin[0..n_part] (host, n_part + 1 entries). */
fvgb_status fvgb_mesh_parts(fvgb_mesh m, int32_t* n_part, int64_t* cell_begin);

/* Per-part results of the last fvgb_poisson_solve on this mesh (host arrays of n_part
 * entries, any may be NULL): final relative residual, outer steps, inner CG iterations. */
fvgb_status fvgb_solve_parts(fvgb_mesh m, double* rel_res, int32_t* outer_its,
                             int32_t* inner_its);

/* Release every device and host allocation of the mesh (synchronises the device). */
fvgb_status fvgb_mesh_free(fvgb_mesh m);

/* Mesh sizes: cells, faces, vertices and node-neighbour entries (sum over cells of
 * the number of cells sharing a vertex with the cell). Any pointer may be NULL. */
fvgb_status fvgb_mesh_info(fvgb_mesh m, int64_t* n_cell, int64_t* n_face,
                           int64_t* n_vert, int64_t* n_nbr);

/* perm_host[internal index] = caller's cell index (host array of n_cell int32). */
fvgb_status fvgb_mesh_cell_perm(fvgb_mesh m, int32_t* perm_host);

/* perm_host[internal index] = caller's vertex index (host array of n_vert int32); vertex
 * arrays such as the output of fvgb_vertex_values are in this internal order. */
fvgb_status fvgb_mesh_vert_perm(fvgb_mesh m, int32_t* perm_host);

/* Reorder n_comp per-cell arrays of elem_bytes-sized elements (4 or 8) between the
 * caller's order and the internal order. src_dev and dst_dev must not overlap.
 * to_internal = 1: dst[i] = src[perm[i]]; 0: dst[perm[i]] = src[i]. */
fvgb_status fvgb_permute(fvgb_mesh m, const void* src_dev, void* dst_dev, int32_t n_comp,
                         int32_t elem_bytes, int32_t to_internal, void* stream);

/* Least-squares cell gradient of Algorithm "grad" (Section 2.1): for every cell,
 * grad u_i = M_i^{-1} sum_j d_ij (u_j - u_i) over the set of cells sharing a vertex
 * with cell i, plus the face centroids of Dirichlet faces of set bcset that share a
 * vertex with it (value g), d = x_j - x_i, M_i = sum d d^T.
 *  u_dev     [n_cell] real      grad_dev [dim][n_cell] real */
fvgb_status fvgb_gradient(fvgb_mesh m, int32_t bcset, const void* u_dev, void* grad_dev,
                          void* stream);

/* Multiplicity-weighted variant of the gradient of Algorithm "grad" (not in the paper;
 * the vertex-factorised form): every neighbour cell j, and every Dirichlet ghost point,
 * counts once per vertex it shares with cell i - grad u_i = Mv_i^{-1} sum m_ij d_ij
 * (u_j - u_i). Exact for linear fields like fvgb_gradient but a different stencil weighting,
 * computed as per-vertex sums over the cells around each vertex (a fraction of the
 * node-neighbour gathers). Arguments and layout as fvgb_gradient. */
fvgb_status fvgb_gradient_vertex(fvgb_mesh m, int32_t bcset, const void* u_dev, void* grad_dev,
                                 void* stream);

/* Least-squares vertex values of Algorithm "ls": u_A = sum_c alpha_{A,c} u_c over the
 * cells around vertex A (linear least-squares fit; mean when the fit is degenerate);
 * vertices on a Dirichlet face of set bcset take g.
 *  u_dev [n_cell] real   uv_dev [n_vert] real (internal vertex order) */
fvgb_status fvgb_vertex_values(fvgb_mesh m, int32_t bcset, const void* u_dev, void* uv_dev,
                               void* stream);

/* Transport coefficients of eq. 1: velocity (a per-cell field [dim][n_cell] real when
 * vel_dev is not NULL, else the constant vel_const), diffusivity D >= 0, source
 * S_i ([n_cell] real or NULL), boundary conditions bcset, and the convective face value
 * of eq. 15: recon = 0 first-order upwind (psi = 0); recon = 1 MUSCL with the
 * Barth-Jespersen limiter, u_up = u_c + psi_c grad u_c . (x_f - x_c) for the upwind cell c
 * (grad from Algorithm "grad" with the same boundary conditions; psi_c = min over the
 * cell's faces of min(1, (bound - u_c) / (grad u_c . (x_f - x_c))), the bounds being the
 * max / min of u_c, its face neighbours and its Dirichlet values); a boundary ghost on
 * the upwind side keeps its first-order value. Other values: FVGB_EINVAL. */
typedef struct {
  const void* vel_dev;
  double vel_const[3];
  double diff;
  const void* src_dev;
  int32_t bcset;
  int32_t recon;
} fvgb_tcoef;

/* Residual of eq. 4: res_i = (sum over faces entering i - leaving i of F_f) / mu_i + S_i,
 * F_f = (V_f . S_f) u_up - D grad u_f . S_f, V_f = (V_L + V_R)/2,
 * u_up from the cell on the upwind side: L if V_f . S_f >= 0, else R (eq. 15; see
 * fvgb_tcoef.recon).
 *  u_dev, res_dev: [n_cell] real, distinct buffers. */
fvgb_status fvgb_fv_residual(fvgb_mesh m, const fvgb_tcoef* tc, const void* u_dev,
                             void* res_dev, void* stream);

/* fvgb_fv_residual that allocates nothing. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they need a residual,
 * such as a host program whose device memory is handed out by its own pool (a stray
 * cudaMalloc there can fail or fragment the pool) or a time-critical loop in which
 * cudaMalloc / cudaFree would add latency and implicit synchronisation. Arguments,
 * results and errors are those of fvgb_fv_residual, except that only first-order upwind
 * is offered (recon = 1 gives FVGB_EUNSUPPORTED; values other than 0 and 1 give
 * FVGB_EINVAL, as in fvgb_fv_residual).
 *  - Scratch (the face fluxes and vertex values) lives in one fixed 8 MiB device array
 *    owned by the library, which every GPU that loads the library holds until the
 *    process exits. A mesh needs n_face + n_vert reals of it (rounded up to 256 bytes
 *    after the fluxes): up to about 1,048,000 doubles or 2,097,000 floats, i.e. FP64
 *    tetrahedral meshes of roughly 480,000 cells. Larger meshes get FVGB_EINVAL with a
 *    message; use fvgb_fv_residual for them.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and caches it together with the
 *    unique id of the current CUDA context; make that first call before any stream
 *    capture. A call in a different context of the device (after cudaDeviceReset, or
 *    once the primary context was released and re-created) looks the address up again,
 *    so a stale address is never used.
 *  - Every call shares the one array and leaves its contents behind; each call writes
 *    the scratch it reads, so nothing needs clearing, but calls that overlap on the GPU
 *    (other streams, other meshes, other host threads) race on it: serialise them.
 *  - The mesh's device must be the current device. */
fvgb_status fvgb_fv_residual_noalloc(fvgb_mesh m, const fvgb_tcoef* tc, const void* u_dev,
                                     void* res_dev, void* stream);

/* nsteps explicit time steps of eq. 6 in place on u_dev: per step
 * u^(k) = u^n + stage_alpha[k] dt Res(u^(k-1)), k = 0..nstage-1, u^{n+1} = u^(last).
 * nstage = 1 with stage_alpha = {1} (or stage_alpha = NULL) is explicit Euler;
 * {0.5, 0.5, 1} is the paper's three-stage scheme. nstage <= 8. When tc->src_dev is
 * set it is held fixed over the steps. */
fvgb_status fvgb_fv_step(fvgb_mesh m, const fvgb_tcoef* tc, void* u_dev, double dt,
                         int32_t nsteps, const double* stage_alpha, int32_t nstage,
                         void* stream);

/* Poisson operator of eq. 7 / eq. "laplace" in FP64, integrated form with positive
 * sign: y = A x = -mu Lap_h(x) with homogeneous boundary values of set bcset
 * (Dirichlet faces and vertices take 0; Neumann and wall faces carry no flux).
 *  x_dev, y_dev: [n_cell] double, distinct. */
fvgb_status fvgb_poisson_apply(fvgb_mesh m, int32_t bcset, const double* x_dev,
                               double* y_dev, void* stream);

/* Right-hand side of the Poisson system for Lap phi = f: b = -mu f + mu Lap_h(0; g).
 *  f_dev, b_dev: [n_cell] double. f_dev may be NULL (f = 0). */
fvgb_status fvgb_poisson_rhs(fvgb_mesh m, int32_t bcset, const double* f_dev, double* b_dev,
                             void* stream);

typedef struct {
  double rtol;          /* stop when ||b - A phi||_2 <= rtol ||b||_2 (FP64) */
  double inner_rtol;    /* inner CG reduces its (scaled) residual by this factor (e.g. 0.1) */
  int32_t maxit_inner;  /* per inner CG solve */
  int32_t maxit_outer;  /* outer FP64 refinement steps */
  int32_t prec;         /* inner solve arithmetic: FVGB_FP64 or FVGB_FP32 (mixed) */
  int32_t inner;        /* inner solve of the two-point operator A_T: 0 conjugate gradients
                           (to inner_rtol, at most maxit_inner iterations); k = 1..8: k
                           V-cycles of smoothed-aggregation multigrid (damped Jacobi,
                           hierarchy built on the host at the first such solve of the
                           boundary set and precision - that call synchronises and may
                           take seconds on large meshes - then kept with the mesh). The
                           paper solves its Poisson systems with FGMRES + PETSc's
                           aggregation multigrid (Tables "comp1", "comp2"). */
} fvgb_solve_opts;

typedef struct {
  int32_t outer_its;
  int32_t inner_its_total;
  double rel_res;       /* final ||b - A phi|| / ||b|| in FP64 */
  double bnorm;         /* ||b||_2 */
} fvgb_solve_info;

/* Solve Lap phi = f (eq. 1.1 discretised by eq. 7) for phi on set bcset.
 * Outer loop in FP64 (defect correction / iterative refinement on the full diamond
 * operator A): r = b - A phi, stop when ||r|| <= rtol ||b||; otherwise an inner
 * conjugate-gradient solve of A_T delta = r on the symmetric positive definite
 * two-point part A_T of A (coefficient |S_f|^2 / ((x_R - x_L) . S_f) per face), in
 * opts->prec arithmetic with FP64 dot products, then phi += delta. The CG runs on the
 * Jacobi-scaled system D^-1/2 A_T D^-1/2 y = D^-1/2 r (D = diag A_T), delta = D^-1/2 y:
 * diagonally preconditioned CG, with the scaling applied once per inner solve.
 *  f_dev    [n_cell] double (NULL = 0)
 *  phi_dev  [n_cell] double, in: initial guess, out: solution
 *  info     host, may be NULL
 * The call synchronises the stream once per outer step (to read the FP64 residual).
 * Returns FVGB_ENOCONV (with info filled and phi the last iterate) if rtol is not met
 * within maxit_outer steps, FVGB_ENONFINITE on NaN/Inf, FVGB_ETIMEOUT if a grid-wide
 * barrier of the persistent CG kernel gave up. */
/* Sizes of the multigrid levels built for (bcset, prec) (fine to coarsest) in sizes[0..cap);
 * returns the number of levels, 0 when none has been built. */
int32_t fvgb_amg_levels(fvgb_mesh m, int32_t bcset, int32_t prec, int64_t* sizes, int32_t cap);

fvgb_status fvgb_poisson_solve(fvgb_mesh m, int32_t bcset, const double* f_dev,
                               double* phi_dev, const fvgb_solve_opts* opts,
                               fvgb_solve_info* info, void* stream);

/* Plasma spot of the branching streamer (Section 4, "Streamer Branching"): a source of
 * electron-ion pairs S(x) = amplitude exp(-|x - centre|^2 / sigma^2) (the paper prints the
 * exponent without its minus sign; this is the decaying reading), switched on during
 * [t_on, t_on + duration). It adds to S_e of eq. 10, i.e. to both n_e and n_i. A step
 * [t, t + dt] takes the spot's average over its overlap with that window,
 * S(x) |[t, t + dt] n [t_on, t_on + duration]| / dt, so steps of any length deposit the
 * spot's exact total; the three stages of eq. 6 all use that step average. The paper's
 * values: amplitude 1e25, sigma 0.005, t_on 1.26e-8 s, duration 0.5e-9 s. */
typedef struct {
  double centre[3];     /* spot centre (x, y, z; z ignored in 2D) */
  double amplitude;     /* > 0 */
  double sigma;         /* > 0 */
  double t_on;
  double duration;      /* >= 0 */
} fvgb_spot;

/* Electron drift-diffusion + Poisson step of eq. 10 with the synthetic coefficients:
 * v = -mu E, alpha = A exp(-B/|E|) (0 at |E| = 0), S = alpha |v| n_e, constant D_e,
 * Lap phi = -(e/eps0)(n_i - n_e). Per step: solve for phi (warm start from phi_dev),
 * E = -grad phi (least-squares gradient, set bcset_phi), then
 * n_e += dt Res(n_e) (set bcset_ne, velocity field v, diffusivity D_e, source S, face
 * values per recon) and n_i += dt S. */
typedef struct {
  double mu, A, B, De;
  double dt;
  int32_t bcset_ne;
  int32_t bcset_phi;
  fvgb_solve_opts solve;
  fvgb_mpnn warm;        /* learned warm start (see fvgb_mpnn_*) or NULL: when set, each
                            step after the first on this mesh predicts the increment of
                            phi from the change of n_i - n_e since the previous step and
                            phi, and starts the Poisson solve of every part from
                            phi + s prediction: s = 1 where that start has the smaller
                            FP64 residual ||b - A phi||, elsewhere s = <r0, A pred> /
                            ||A pred||^2 (r0 = b - A phi), the scale that minimises the
                            residual along the prediction; so the start's residual is not
                            larger than without the network (s = 0 where the prediction
                            is 0); the solve still converges to rtol either way */
  int32_t extrapolate;   /* 1: start each solve from the linear extrapolation in time
                            2 phi^{n-1} - phi^{n-2} (after two steps on this mesh); with
                            a network, the network then predicts the extrapolation's
                            error from the change of the charge change (its second
                            difference in time) */
  int32_t recon;         /* convective face value of the n_e transport (fvgb_tcoef.recon):
                            0 first-order upwind, 1 MUSCL + Barth-Jespersen (eq. 15) */
  int32_t stages;        /* time scheme: 0 or 1 explicit Euler; 3 the three stages of eq. 6
                            (alpha = 1/2, 1/2, 1), each with its own Poisson solve (from the
                            previous stage's phi), field and source from the stage densities;
                            the step's solve info then sums the stages' iterations and keeps
                            their largest residual; phi and E on return are the last stage's.
                            Three-stage steps run host-driven also in graph mode. */
  double t0;             /* time at the start of the call's first step (step n of the call
                            starts at t0 + n dt); only the plasma spots depend on it */
  int32_t n_spot;        /* plasma spots (0..4) added to the source, see fvgb_spot */
  const fvgb_spot* spots;  /* host array of n_spot spots (read during the call; in graph
                              mode copied into the captured step) */
} fvgb_streamer_params;

/* ne_dev, ni_dev: [n_cell] real; phi_dev: [n_cell] double (in: guess, out: last
 * potential); E_dev: [dim][n_cell] real or NULL (out: last field).
 * info: host, [nsteps] entries or NULL. Returns the first failing solve's status. */
fvgb_status fvgb_streamer_step(fvgb_mesh m, const fvgb_streamer_params* p, void* ne_dev,
                               void* ni_dev, double* phi_dev, void* E_dev, int32_t nsteps,
                               fvgb_solve_info* info, void* stream);

/* Graph mode for fvgb_streamer_step (off by default). When on, a whole step - source,
 * right-hand side, the FP64 refinement loop of the Poisson solve as a CUDA-graph
 * conditional WHILE node around the cooperative inner CG, then field and transport - is
 * captured once as a CUDA graph (for the given arrays and parameters; a change of either
 * recaptures) and replayed per step. The loop decisions run on the device, so a call with
 * nsteps steps synchronises the stream once, at its end; a failing solve is then
 * reported for the first step that failed (later steps of the call have run). */
fvgb_status fvgb_set_graph_mode(fvgb_mesh m, int32_t on);

/* Autotuner (no counterpart in the paper): pick the launch shape - threads per block
 * and elements per thread - of the four gather kernels (0 least-squares gradient,
 * 1 vertex values, 2 face fluxes, 3 face-to-cell update) by timing every candidate
 * (threads 128..1024 x 1, 2, 4 elements) with CUDA events on this mesh. Shapes are cached
 * per device and mesh class (dimension, precision, size bucket floor(log2 n_cell)); a
 * later mesh of the same class reuses them unless force = 1. Results never depend on the
 * shape. shapes_out (host, 8 ints or NULL) receives (threads, elements) per kernel.
 * Synchronises the stream; drops a captured step graph. */
fvgb_status fvgb_autotune(fvgb_mesh m, int32_t force, int32_t* shapes_out, void* stream);

/* Set one kernel's launch shape by hand (kernel 0..3 as above; threads a multiple of 32
 * in [32, 1024], elements per thread in [1, 64]). */
fvgb_status fvgb_set_launch_shape(fvgb_mesh m, int32_t kernel, int32_t threads, int32_t ipt);

/* Integral of a cell field over the domain, sum_i mu_i u_i (the mass of eq. 2 summed
 * over the cells), accumulated in FP64 in a fixed order (bitwise reproducible).
 *  u_dev [n_cell] real; *out_host receives the sum. Synchronises the stream. */
fvgb_status fvgb_integral(fvgb_mesh m, const void* u_dev, double* out_host, void* stream);

/* Counters for measurement (no counterpart in the paper's method).
 *  kernel_launches  kernels launched by the library since the last reset (all meshes)
 *  cg_launches      inner CG kernels launched for this mesh
 *  cg_iterations    CG iterations they ran
 *  cg_ms            summed device time of those kernels, measured with CUDA events on the
 *                   launching stream when timing was enabled (0 otherwise)
 *  solves, outer_its  Poisson solves and their outer refinement steps
 *  learned_starts   parts of host-driven streamer solves that evaluated a learned start
 *  learned_kept     of those, the parts whose learned correction entered the start with a
 *                   positive scale */
typedef struct {
  int64_t kernel_launches;
  int64_t cg_launches;
  int64_t cg_iterations;
  double cg_ms;
  int64_t solves;
  int64_t outer_its;
  int64_t learned_starts;
  int64_t learned_kept;
} fvgb_stats;

/* Turn CUDA-event timing of the inner CG kernels on (1) or off (0). */
fvgb_status fvgb_stats_enable(fvgb_mesh m, int32_t time_cg);

/* Copy the counters into *out (host); reset = 1 zeroes them afterwards. */
fvgb_status fvgb_stats_get(fvgb_mesh m, fvgb_stats* out, int32_t reset);

/* Forget the warm-start history (earlier charges and potentials) of this mesh: the next
 * steps start from phi alone until the history is rebuilt. */
fvgb_status fvgb_streamer_reset(fvgb_mesh m);

/* Training pair of the learned warm start (no counterpart in the paper) from the history
 * that the last fvgb_streamer_step kept on this mesh (steps with warm start or
 * extrapolation requested keep one). With phi^n the potential at the start of that step,
 * phi^{n+1} = phi_dev its solution, q = n_i - n_e at step starts, dq^n = q^n - q^{n-1}:
 *  which = 0 (a start from the previous potential): dq^n, phi^n, phi^{n+1} - phi^n;
 *    needs two steps of history since the last reset;
 *  which = 1 (a start from the extrapolation 2 phi^n - phi^{n-1}): dq^n - dq^{n-1}, phi^n,
 *    phi^{n+1} - 2 phi^n + phi^{n-1}; needs three steps.
 * All arrays [n_cell] double on the device (outputs written by the call, stream-ordered).
 * Errors: FVGB_EINVAL for a bad argument or too short a history. */
fvgb_status fvgb_streamer_pair(fvgb_mesh m, int32_t which, const double* phi_dev, double* dq_dev,
                               double* phi_prev_dev, double* dphi_dev, void* stream);

/* ---- Learned warm start (no counterpart in the paper) --------------------------------
 * A message-passing network predicts the potential increment of a streamer step:
 *   f_i = [ (e/eps0) dq_i mu_i^(2/3) / (V s0),  phi_prev_i / (V s1) ]
 *   h0 = relu(W_enc f + b_enc) (width 64);
 *   layer(l, h; graph): m_i = sum_j w_ij (h_j - h_i), h + relu(W_l [h ; m] + b_l);
 *   h1 = layer(0, h0; interior faces, w = c1 / max c1 of set bcset);
 *   local architecture (multilevel = 0): h2 = layer(1, h1; interior faces);
 *   multilevel architecture (multilevel = 1): the middle layer runs on the aggregate
 *   hierarchy of fvgb_mpnn_hierarchy, which reaches the whole part: at every
 *   level, the mean over each aggregate of the level below (h1 for the first), then two
 *   applications of layer(1, c; face-adjacent aggregates, w = 1/6); then back up, every
 *   level adds its aggregate's value, down to h2 = h1 + c_1 of the cell's aggregate;
 *   h3 = layer(2, h2; interior faces);
 *   out = N(f) = w_dec . h3 + b_dec; increment = V s2 (N(f) - N(f with f0 = 0)), i.e. the
 *   response to the charge change (what the network gives for an unchanged charge is
 *   removed, so no change predicts no increment).
 * Layer products run on the tensor cores (BF16 weights and activations, FP32
 * accumulation); master weights, gradients and Adam state are FP32.
 * Parameters: one FP32 vector of fvgb_mpnn_param_count() entries, blocks in order
 * W_enc [64][2], b_enc [64], then per layer W_l [64][128] (inputs [h ; m]), b_l [64],
 * then w_dec [64], b_dec [1]. A network belongs to one 3D mesh (FVGB_EINVAL otherwise);
 * move weights between meshes with get/set. */

/* The aggregate hierarchy of the network (host arrays; needs no GPU). cen: [3][n_cell]
 * cell centres; part_begin: n_part + 1 cell offsets (0 ... n_cell, parts non-empty).
 * Per part, with [lo, hi] the bounding box of its centres and r_1 = max(1, round((n /
 * 6)^(1/3))) boxes per axis, a cell's level-1 box index per axis is min(r_1 - 1,
 * floor((x - lo) / (hi - lo) r_1)) (0 when hi = lo); level k + 1 halves the indices (r_{k+1}
 * = ceil(r_k / 2)); levels continue while some part has r > 2 and stop once every part is
 * one box (16 at most). Aggregates are the non-empty boxes, numbered part by part in
 * increasing (x, y, z) order. Outputs: *n_levels = L; level_n[0..L) (room for 16) nodes per
 * level; if parent is not NULL, the aggregate (level-local) of every node of the level
 * below, levels one after the other (n_cell + level_n[0] + ... + level_n[L-2] entries); if
 * nbr is not NULL, per level and aggregate 8 slots of face-adjacent aggregates (level-
 * local), the unused ones holding the aggregate itself. Errors: FVGB_EINVAL for bad
 * arguments or a non-finite centre. */
fvgb_status fvgb_mpnn_hierarchy(int64_t n_cell, const double* cen, int32_t n_part, const int64_t* part_begin,
                                int32_t* n_levels, int64_t* level_n, int32_t* parent, int32_t* nbr);
fvgb_status fvgb_mpnn_create(fvgb_mesh m, int32_t bcset, int32_t multilevel, fvgb_mpnn* out);
fvgb_status fvgb_mpnn_free(fvgb_mpnn net);
int64_t fvgb_mpnn_param_count(void);
/* Set the FP32 parameters (host array) and reset the optimiser state. */
fvgb_status fvgb_mpnn_set_params(fvgb_mpnn net, const float* theta_host);
fvgb_status fvgb_mpnn_get_params(fvgb_mpnn net, float* theta_host);
/* Input / output scales V, s0, s1, s2 (all > 0) of the formulas above. */
fvgb_status fvgb_mpnn_set_scales(fvgb_mpnn net, double V, double s0, double s1, double s2);
/* dphi_dev = predicted increment from dq_dev (change of n_i - n_e) and phi_prev_dev
 * (all [n_cell] double, device). Stream-ordered, no synchronisation. */
fvgb_status fvgb_mpnn_predict(fvgb_mpnn net, const double* dq_dev, const double* phi_prev_dev,
                              double* dphi_dev, void* stream);
/* Loss mean_i (pred_i - dphi_i / (V s2))^2, pred = N(f) - N(f0 = 0), and its gradient (host, param_count floats,
 * or NULL) for one sample; synchronises the stream. */
fvgb_status fvgb_mpnn_loss_grad(fvgb_mpnn net, const double* dq_dev, const double* phi_prev_dev,
                                const double* dphi_dev, double* loss_host, float* grad_host,
                                void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on one sample; loss_host may be NULL (then
 * the call does not synchronise). */
fvgb_status fvgb_mpnn_train_step(fvgb_mpnn net, const double* dq_dev, const double* phi_prev_dev,
                                 const double* dphi_dev, float lr, double* loss_host,
                                 void* stream);

/* Synchronise the stream and report the latched asynchronous status of the mesh (see the
 * conventions above), then clear it: FVGB_ETIMEOUT when a tensor-core wait of the network
 * kernels ran out, FVGB_ENONFINITE when a transport update wrote a non-finite value since
 * the last report, FVGB_OK otherwise. */
fvgb_status fvgb_sync(fvgb_mesh m, void* stream);

/* Test hook of the bounded grid barrier of the persistent CG kernel (no counterpart in the
 * paper; for tests of the timeout path only). skip_block >= 0 makes that block of the
 * kernel's grid never arrive at a barrier, so that the other blocks' waits run out and the
 * solve returns FVGB_ETIMEOUT; timeout_ms > 0 replaces the 1 s wait limit. skip_block = -1
 * and timeout_ms = 0 restore normal operation. A captured step graph is dropped.
 * Errors: FVGB_EINVAL for skip_block outside [-1, grid) or timeout_ms outside [0, 1000]. */
fvgb_status fvgb_test_barrier(fvgb_mesh m, int32_t skip_block, double timeout_ms);

/* Message of the last failing call in this thread ("" if none). */
const char* fvgb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FVGB_H */
