/* libdg -- GB300 (sm_103a) modal discontinuous Galerkin solver for the Euler
 * equations, after Schaal, Bauer, Chandrashekar, Pakmor, Klingenberg and
 * Springel (2015), "Astrophysical hydrodynamics with a high order
 * discontinuous Galerkin scheme and adaptive mesh refinement".
 *
 * C ABI: plain pointers and sizes only.  Every call returns a status code
 * (DG_OK = 0) and never throws.  Host-side argument errors are returned
 * synchronously; errors detected on the device (non-physical state after the
 * positivity limiter) latch a status word that dg_status() reads.
 *
 * Data layout (all state buffers are CALLER-OWNED device memory):
 *   weights   W[var][coef][cell]    var = rho, rho v_1..rho v_dim, rho e
 *             (nv = dim + 2), coef = basis function index (N of them),
 *             cell = cell index (fastest).  Element type: double for
 *             DG_FP64, DG_MIXED and DG_MIXED_TC handles, float for DG_FP32
 *             and DG_FP32_TC handles.
 *   points    u[var][q][cell] (double), xyz[axis][q][cell] (double)
 * Cells are listed by base cell in lexicographic order (x fastest); a refined
 * base cell is replaced by its 2^dim children in the order A..H of the paper's
 * refinement section (child number = sum of child bits, x bit first).
 * Basis functions: products of scaled Legendre polynomials sqrt(2n+1) P_n of
 * total degree <= k (eq. set_basis_functions), ordered by total degree, then
 * x exponent descending, then y exponent descending; coefficient 0 is the
 * cell mean (eq. weights), coefficients 1..dim are the x, y, z slopes.  (The
 * optional tensor-product space DG_BASIS_TENSOR continues this order past
 * total degree k; see below.)
 *
 * Streams: every call that touches device data takes a cudaStream_t passed
 * as `void* stream` (NULL = legacy default stream) and is asynchronous with
 * respect to the host.  Scalars computed on the device (timestep, totals, L1
 * error) are written to device memory.
 */
#ifndef DG_H
#define DG_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
enum {
  DG_OK = 0,
  DG_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, unsupported combination) */
  DG_ERR_CUDA = 2,         /* a CUDA runtime call failed; dg_last_error() has the message */
  DG_ERR_OOM = 3,          /* device allocation failed */
  DG_ERR_NONPHYSICAL = 4,  /* device flag: a cell mean with rho <= 0 or p <= 0 was seen */
  DG_ERR_TIMEOUT = 5,      /* device flag: a bounded wait gave up */
  DG_ERR_UNSUPPORTED = 6   /* (dim, k, precision, basis) combination, or a call on a handle, not built */
};

enum { DG_BC_PERIODIC = 0, DG_BC_TRANSMISSIVE = 1 };
enum { DG_LIMITER_NONE = 0, DG_LIMITER_COMPONENT = 1, DG_LIMITER_CHARACTERISTIC = 2 };
/* Precision of a handle.
 * DG_FP64:    FP64 state and arithmetic.
 * DG_FP32:    FP32 state and arithmetic.
 * DG_FP32_TC: FP32 state with the cell kernel's contractions on the tensor
 *             cores (split TF32 operands, FP32 accumulation); 2D uniform
 *             meshes, k = 1..3 (DG_ERR_UNSUPPORTED otherwise).
 * DG_MIXED:   FP64 state (the W arrays are double, the stage combination is
 *             FP64) with the right-hand side evaluated in FP32 in perturbation
 *             form: each cell subtracts the flux of its own mean state from
 *             the point and face fluxes it integrates, which leaves the
 *             discrete right-hand side unchanged and makes the FP32 rounding
 *             scale with the solution's variation rather than its size.  The
 *             CFL timestep, totals, the positivity limiter's decisions and
 *             the adjoint run in FP64; the slope limiter's arithmetic runs in
 *             FP32 on the rounded state (a cell it leaves alone keeps its
 *             FP64 weights exactly).
 * DG_MIXED_TC: DG_MIXED with the cell kernel's two contractions on the
 *             tensor cores (split TF32, FP32 accumulation); 2D uniform meshes,
 *             k = 1..3. */
enum { DG_FP64 = 0, DG_FP32 = 1, DG_FP32_TC = 2, DG_MIXED = 3, DG_MIXED_TC = 4 };

/* Polynomial space of a cell (dg_options.basis).
 * DG_BASIS_TOTAL: the paper's basis (Sec. 2.2, eq. set_basis_functions): the
 *             products of scaled Legendre polynomials of total degree <= k,
 *             N(k) = (k+1)(k+2)/2 in 2D, (k+1)(k+2)(k+3)/6 in 3D.
 * DG_BASIS_TENSOR: the same products with every exponent <= k (the tensor
 *             product space Q_k, N = (k+1)^2 in 2D), ordered by total degree,
 *             then x exponent descending, so that its first N(k) functions are
 *             those of DG_BASIS_TOTAL.  Same quadrature rules (the (k+1)-point
 *             Gauss rule integrates the mass products of Q_k exactly).  Built
 *             for dim 2, k = 1..3, DG_FP64 and DG_FP32, without the slope or
 *             positivity limiter; dg_limit, dg_rk_step_adjoint,
 *             dg_node_weights, dg_set_gravity, dg_adapt_mark, dg_adapt_set
 *             and dg_regrid return DG_ERR_UNSUPPORTED on such a handle.  At k = 0 both
 *             spaces are the constants and the handle is a DG_BASIS_TOTAL one. */
enum { DG_BASIS_TOTAL = 0, DG_BASIS_TENSOR = 1 };

/* Mesh description (paper Secs. 2.2 and 4): cubical cells on the box
 * [lo, hi]; n[a] base cells along axis a (the base edge length must be equal
 * on all axes); bc[a] per axis.  Static refinement: each box refines the
 * inclusive base-cell index range [lo_0..lo_{dim-1}, hi_0..hi_{dim-1}] once
 * (one level: the level jump between neighbours is then at most one, as the
 * paper requires).  The description is copied by dg_create. */
typedef struct {
  int dim;                     /* 2 or 3 */
  int n[3];                    /* base cells per axis (entries beyond dim ignored) */
  double lo[3], hi[3];         /* domain box */
  int bc[3];                   /* DG_BC_PERIODIC or DG_BC_TRANSMISSIVE per axis */
  int n_refine_boxes;          /* number of refinement boxes (0 = uniform mesh) */
  const int32_t* refine_boxes; /* host pointer, n_refine_boxes * 2 * dim ints */
} dg_mesh_desc;

/* Scheme options (defaults from dg_default_options follow the paper's runs:
 * CFL 0.2 (Sec. 2.5), beta = 1, Mtilde = 0.5 (Sec. 5), eps = 1e-10 (Sec. 3.4)). */
typedef struct {
  int rk_order;      /* 1..4: SSP RK tableaux of Appendix D (order 4 is the 5-stage method) */
  double cfl;        /* CFL number of eq. time_step */
  int slope_limiter; /* DG_LIMITER_* (Secs. 3.1-3.3; bounded minmod) */
  double beta;       /* limiter parameter beta in [0.5, 1] */
  double Mtilde;     /* TVB bound: a slope is kept when |sqrt(3) slope| <= Mtilde * dx */
  int positivity;    /* 1: positivity limiter of Sec. 3.4 after every stage */
  double eps;        /* positivity floor of density and pressure at the limiter's points; an FP32
                        state also keeps 2^-20 of the absolute weight sums (at most half the mean),
                        above the FP32 rounding of the stored limited weights */
  int precision;     /* DG_FP64, DG_FP32, DG_FP32_TC, DG_MIXED or DG_MIXED_TC (state,
                        fluxes and contractions); the totals, L1 error, timestep and
                        positivity check stay FP64 */
  int autotune;      /* 1: dg_create times the stage kernels on the mesh at every
                        feasible tile (16, 32 or 64 cells or faces per thread block) and keeps the
                        fastest, FP32 2D handles also trying the one-thread-per-
                        cell kernel and the packed-pair cell kernel; 0 (default):
                        fixed tiles.  The tiled kernels and the packed-pair kernel
                        give identical results for every tile; the one-thread-per-
                        cell kernel sums in another order (FP32 rounding).  See
                        dg_tiles. */
  int basis;         /* DG_BASIS_TOTAL (default) or DG_BASIS_TENSOR; the weight
                        arrays W[var][coef][cell] then hold N = (k+1)^2 coefficients
                        per variable (dg_sizes) */
} dg_options;

typedef struct dg_handle dg_handle;

/* Fills *opt with the defaults above (rk_order = 3, no limiter, FP64, the
 * total-degree basis). */
int dg_default_options(dg_options* opt);

/* Creates a solver for a mesh, polynomial degree k and adiabatic index gamma
 * (paper Sec. 2).  Builds the cell list, neighbour and face tables and the
 * quadrature tables (Appendices A-C) on the host, uploads them and allocates
 * the library-owned scratch (stage registers, face-flux buffer, reduction
 * partials) on the current CUDA device.  Supported: dim 2 with k = 0..3,
 * dim 3 with k = 0..2.  On failure *out is NULL and the status says why
 * (dg_last_error(NULL) has the message). */
int dg_create(const dg_mesh_desc* mesh, int k, double gamma, const dg_options* opt,
              dg_handle** out);

/* Frees the handle and its device memory.  NULL is accepted. */
int dg_destroy(dg_handle* h);

/* Last error message of a handle (or of the last failed dg_create if h is NULL). */
const char* dg_last_error(const dg_handle* h);

/* Limiter activity since the handle was created or last reset: counts_dev[0]
 * = cell passes in which the slope limiter (Secs. 3.2-3.3) changed the
 * slopes, counts_dev[1] = cell passes in which the positivity limiter (Sec.
 * 3.4) scaled the weights, counts_dev[2] = cell passes that the exact FP32
 * prechecks could not clear and the FP64 positivity pass examined.
 * counts_dev: device memory, three int64 values, written asynchronously on
 * the stream; reset != 0 zeroes the counters after the copy. */
int dg_limiter_counts(dg_handle* h, int64_t* counts_dev, int reset, void* stream);

/* Tiles of the stage kernels in use: cells per thread block of the cell
 * kernel and faces per block of the face kernel (the fixed defaults, or the
 * autotuner's choice when dg_options.autotune was set).  A tensor-core cell
 * kernel (DG_FP32_TC, DG_MIXED_TC) reports its fixed tile of 128 cells (one
 * MMA row per cell); cell tile 1 means the one-
 * thread-per-cell FP32 kernel and cell tile 2 the packed-pair FP32 kernel,
 * both of which the autotuner also considers; face tile
 * 0 means the fused face + cell kernel (tiles of 8 x 4 cells computing their
 * own faces, no separate face kernel).  Host outputs. */
int dg_tiles(const dg_handle* h, int* cell_tile, int* face_tile);

/* Sets the tiles by hand (the autotuner's choices can be overridden):
 * cell_tile 16, 32 or 64 cells per block of the tiled cell kernel, or 1 for
 * the one-thread-per-cell kernel (FP32 2D handles of the total-degree basis
 * only), or 2 for the packed-pair kernel (same handles: 64 cells per block,
 * two variables per thread in paired FP32 multiply-adds, each lane rounded as
 * the one-variable-per-thread kernel rounds it, so bit-identical results);
 * face_tile 16, 32 or
 * 64, or 0 for the fused face + cell kernel: each block takes a tile of 8 x 4
 * cells, computes the fluxes of the tile's faces in shared memory (the
 * neighbours' traces across the tile's edges from their weights) and then
 * the cell update -- one launch per stage and no face-flux array, with the
 * same results to rounding (single 2D uniform meshes, FP64 or FP32 state,
 * the total-degree basis, not with cell_tile 1 or 2; the cell tile value is then
 * unused).  DG_ERR_ARG for other values, DG_ERR_UNSUPPORTED where the (dim,
 * k, precision, basis, mesh) has no such kernel.  Not to be called while another call on the handle is
 * being captured. */
int dg_set_tiles(dg_handle* h, int cell_tile, int face_tile);

/* Sizes: cells, basis functions N(k) (eq. nof_basis_functions and its 2D
 * analogue; (k+1)^2 for DG_BASIS_TENSOR), variables nv, volume Gauss points per cell (k+1)^dim, points of
 * the (k+3)^dim rule used by dg_l1_density, refined base cells (nodes). */
int dg_sizes(const dg_handle* h, int64_t* n_cells, int* n_basis, int* n_vars, int* n_qpoints,
             int* n_l1points, int* n_nodes);

/* Physical coordinates of the volume Gauss points (xyz[axis][q][cell]) and of
 * the (k+3)^dim rule's points; q runs with the x index fastest. */
int dg_quad_points(const dg_handle* h, double* xyz_dev, void* stream);
int dg_l1_points(const dg_handle* h, double* xyz_dev, void* stream);

/* L2 projection of point values onto the basis (Sec. 2.3):
 * W_j = 2^-dim sum_q u(xi_q) phi_j(xi_q) w_q with the (k+1)^dim Gauss rule.
 * u_dev: double [nv][Q][cell]; W_dev: handle precision [nv][N][cell]. */
int dg_project(dg_handle* h, const double* u_dev, void* W_dev, void* stream);

/* Time derivative dW/dt = -R(W) of eq. spatial_discretisation: volume
 * integral (eq. dg_term2) plus surface integral with the HLLC flux at the
 * face Gauss points (eq. dg_term3), hanging faces integrated at the fine
 * sub-face points.  No limiter.  W_dev and dWdt_dev must not alias. */
int dg_rhs(dg_handle* h, const void* W_dev, void* dWdt_dev, void* stream);

/* CFL timestep (eq. time_step, or eq. time_step_pos with positivity on),
 * from the cell means, minimum over all cells, written to *dt_dev (double). */
int dg_compute_dt(dg_handle* h, const void* W_dev, double* dt_dev, void* stream);

/* One SSP-RK step in place (Appendix D, main loop of Sec. 4.5):
 * W <- W + dt sum_i b_i k_i with k_i = -R(U_i); every stage state U_i (i>=2)
 * and the new state are limited when limiting is enabled.  dt > 0 uses that
 * value; dt <= 0 computes the CFL timestep on the device first.  If
 * dt_used_dev is not NULL the timestep is written there (double). */
int dg_rk_step(dg_handle* h, void* W_dev, double dt, double* dt_used_dev, void* stream);

/* n_steps CFL steps in place, recorded once into a CUDA graph per (W_dev,
 * n_steps, dt_hist_dev) and replayed; dt_hist_dev (optional,
 * double[n_steps][n_problems]) receives the timesteps.  The first call for a
 * given key records the graph (make it outside any stream capture).  A
 * handle keeps at most 64 recorded graphs (with dg_advance_dt's); recording
 * one more drops them all, to be recorded anew on their next use. */
int dg_advance(dg_handle* h, void* W_dev, int n_steps, double* dt_hist_dev, void* stream);

/* n_steps steps in place with the fixed timestep dt (> 0, else DG_ERR_ARG),
 * as dg_rk_step with that dt, recorded once into a CUDA graph per (W_dev,
 * n_steps, dt) and replayed (convergence and accuracy studies that must end
 * at a given time).  Always a graph, whatever dg_set_advance_mode says. */
int dg_advance_dt(dg_handle* h, void* W_dev, int n_steps, double dt, void* stream);

/* ---- ensembles of independent problems --------------------------------
 * dg_create_batch: one handle for n_problems independent problems (same dim,
 * uniform meshes, equal gamma -- DG_ERR_UNSUPPORTED otherwise) advanced
 * together.  Their cells are concatenated in problem order into one state
 * W[var][coef][cell]; each problem keeps its own edge length, boundaries and
 * CFL timestep (dt_used_dev / dt_hist_dev then hold one double per problem,
 * per step).  Every other entry point accepts a batch handle; dg_totals and
 * dg_l1_density reduce over all problems together. */
int dg_create_batch(const dg_mesh_desc* meshes, const double* gamma, int n_problems, int k,
                    const dg_options* opt, dg_handle** out);

/* n_steps steps of every problem of a batch (each with its own CFL
 * timestep) as one CUDA-graph launch; same as dg_advance. */
int dg_batch_advance(dg_handle* h, void* W_dev, int n_steps, double* dt_hist_dev, void* stream);

/* How dg_advance (and dg_batch_advance) run their steps.
 *   DG_ADVANCE_GRAPH       one CUDA graph per (W, n_steps, dt_hist) holding
 *                          every kernel launch of the steps (recorded on first
 *                          use, replayed afterwards);
 *   DG_ADVANCE_PERSISTENT  one cooperative launch of a persistent kernel that
 *                          runs all phases of the steps (timestep, face fluxes,
 *                          cell updates, limiters) separated by grid-wide
 *                          barriers; bit-identical results.  Its barrier waits
 *                          are bounded: a wait that gives up stops the kernel
 *                          and latches DG_ERR_TIMEOUT (dg_status).
 * The persistent kernel serves 2D handles with the total-degree basis, an
 * FP64 or FP32 state and the CUDA-core stage kernels (not DG_FP32_TC / DG_MIXED / DG_MIXED_TC, not the
 * one-thread-per-cell tile), without a gravity source, with at most 5 RK
 * stages.  DG_ADVANCE_GRAPH is the default on every handle: on one GB300 a
 * graph's kernel boundary costs about as much as the persistent kernel's
 * grid barrier, and the graph measured faster from 32^2 to 128^2 cells.
 * Setting DG_ADVANCE_PERSISTENT on a handle that does not support it
 * returns DG_ERR_UNSUPPORTED; dg_advance_mode reports the path dg_advance
 * takes now.  The first persistent dg_advance on a state
 * builds a step plan in device memory (synchronous copy; make that first call
 * outside any stream capture). */
enum { DG_ADVANCE_GRAPH = 0, DG_ADVANCE_PERSISTENT = 1 };
int dg_set_advance_mode(dg_handle* h, int mode);
int dg_advance_mode(const dg_handle* h, int* mode);

/* Kernel-boundary overlap (on by default): the face, cell, timestep and
 * limiter kernels of a step are launched with programmatic stream
 * serialization, so the device may schedule a kernel while the one ahead of
 * it drains; each kernel waits (griddepcontrol.wait) until its predecessor has
 * completed and its writes are visible before touching any state, so results
 * do not change.  on = 0 launches them with plain stream order.  Cached step
 * graphs are recorded anew.  Not to be called while another call on the
 * handle is being captured. */
int dg_set_overlap(dg_handle* h, int on);
int dg_overlap(const dg_handle* h, int* on);

/* Number of problems and, if cell_offsets_host is not NULL, the first cell
 * of every problem (n_problems + 1 entries, the last one = n_cells). */
int dg_n_problems(const dg_handle* h, int* n_problems, int64_t* cell_offsets_host);

/* Adjoint of one unlimited step with a frozen timestep dt (> 0):
 * lam_n = (d W_{n+1} / d W_n)^T lam_np1, where W_n_dev is the checkpointed
 * state the step started from (the paper has no adjoint; this is the exact
 * transpose of the Butcher-form step of Appendix D).  The stage states are
 * recomputed from W_n; the reverse sweep applies the transposed linearised
 * right-hand side, whose HLLC and Euler-flux Jacobian-transpose products are
 * hand-written reverse-mode derivatives (one forward evaluation, then the
 * adjoints in reverse order).  lam_n_dev may alias lam_np1_dev.  Requires slope_limiter = NONE
 * and positivity = 0 (DG_ERR_ARG otherwise).  The first call allocates the
 * handle's adjoint work arrays (2 s state arrays for s stages, plus the face
 * cotangents). */
int dg_rk_step_adjoint(dg_handle* h, const void* W_n_dev, double dt, const void* lam_np1_dev,
                       void* lam_n_dev, void* stream);

/* Slope limiter (Secs. 3.2-3.3, with the AMR neighbour projections of
 * Sec. 4.4) followed by the positivity limiter (Sec. 3.4), in place. */
int dg_limit(dg_handle* h, void* W_dev, void* stream);

/* Conserved totals sum_K |K| w_{1,i} (FP64, deterministic two-pass
 * reduction) -> totals_dev[nv] (double). */
int dg_totals(dg_handle* h, const void* W_dev, double* totals_dev, void* stream);

/* L1 density error (eq. L1_norm) with the (k+3)^dim Gauss rule per cell:
 * (1/V) sum_K int_K |rho_h - rho_ref| dV; rho_ref_dev: double [Q1][cell] at
 * the points of dg_l1_points.  Result in *out_dev (double). */
int dg_l1_density(dg_handle* h, const void* W_dev, const double* rho_ref_dev, double* out_dev,
                  void* stream);

/* AMR node weights w_node = 2^-dim sum_c P_c^T w^c over the children of every
 * refined base cell (eq. deref_weights) -> Wnode_dev [nv][N][node]. */
int dg_node_weights(dg_handle* h, const void* W_dev, void* Wnode_dev, void* stream);

/* Gravity (eq. gravity_term, Sec. 2.4; timestep Sec. 2.5): sets the external
 * acceleration a = -grad Phi, given at the volume points of every cell in the
 * order of dg_quad_points as accel_dev double [dim][Q][cell] (device; read on
 * `stream`, copied into the handle in its state precision).  While set, every
 * right-hand side adds the source s = (0, rho a, m . a) projected with the
 * volume Gauss rule, 2^-dim sum_q s(u_q) phi_j(xi_q) w_q, and the timestep is
 * the smaller of the hydro bound and c / (sqrt(2 gamma (gamma - 1)) |a|) per
 * cell (c of the cell mean, |a| the largest over the cell's points; no CFL
 * factor on this bound).  NULL removes the field.  DG_FP64 and DG_FP32 single
 * problems only (DG_ERR_UNSUPPORTED otherwise); dg_regrid drops the field and
 * the stepping calls return DG_ERR_ARG until it is set again; the adjoint
 * refuses a handle with gravity. */
int dg_set_gravity(dg_handle* h, const double* accel_dev, void* stream);

/* ---- Mesh adaptation of the two-level mesh (Secs. 4.1, 4.3-4.5) ----
 * Single problems with k >= 1 only (DG_ERR_UNSUPPORTED otherwise); the tensor-core
 * precisions keep their uniform-mesh restriction (dg_regrid refuses a mesh
 * with nodes).  Base cells are numbered lexicographically (x fastest).
 *
 * dg_adapt_mark: decides the next refinement from the state W_dev (the
 * handle's precision and layout) on `stream`.  A leaf base cell meets the
 * criterion when max_a |w_{rho,1+a}| > alpha * w_t (eq. cell_ref), a refined
 * base cell (a node) when the same maximum over its node weights exceeds
 * w_t / alpha (eq. node_ref); a base cell is refined on the next mesh when it
 * or any of the 3^dim - 1 base cells around it (sharing a face, edge or
 * corner; periodic axes wrap) meets its criterion, which keeps one buffer
 * layer around every flagged cell (Sec. 4.1).  The paper takes w_t = 0.01,
 * alpha = 1.1.  Synchronises `stream`; returns the next mesh's cell count in
 * *n_cells_new and the number of base cells whose refinement changes in
 * *n_changed (either may be NULL); flags_host (NULL or int32 [n_base]) gets
 * the next refinement (1 refined, 0 leaf).  The decision is kept in the
 * handle for dg_regrid.  DG_ERR_ARG unless w_t > 0 and alpha >= 1.
 *
 * dg_adapt_set: the same with the next refinement given by flags_host
 * (int32 [n_base], nonzero = refined).
 *
 * dg_regrid: rebuilds the handle's mesh tables on the device for the marked
 * refinement and writes the state on the new mesh to W_new_dev ([nv][N]
 * [n_cells_new], caller-owned, must not alias W_old_dev): unchanged cells are
 * copied, a newly refined cell's children get w^c = P_c w (eq. ref_weights,
 * exact for the coarse polynomial), a derefined node's cell gets
 * w = 2^-dim sum_c P_c^T w^c (eq. deref_weights, conserving every mean).
 * Synchronises `stream` once (to size the face arrays); buffers that no
 * longer fit are reallocated.  Afterwards every entry point works on the new
 * mesh (dg_sizes reports its counts; cached step graphs are recorded anew).
 * DG_ERR_ARG when no refinement is marked; after DG_ERR_OOM or DG_ERR_CUDA
 * from dg_regrid the handle's tables are incomplete and it must be destroyed. */
int dg_adapt_mark(dg_handle* h, const void* W_dev, double w_t, double alpha, int32_t* flags_host,
                  int64_t* n_cells_new, int64_t* n_changed, void* stream);
int dg_adapt_set(dg_handle* h, const int32_t* flags_host, int64_t* n_cells_new, int64_t* n_changed,
                 void* stream);
int dg_regrid(dg_handle* h, const void* W_old_dev, void* W_new_dev, void* stream);

/* Host copies of the mesh tables, for checks:
 * neighbour table nbr[side][cell] (side = 2*axis + {0:-, 1:+}; >= 0 a leaf
 * cell, -1 no neighbour, <= -2 the node -(v+2)); levels[cell]. */
int dg_neighbor_table(const dg_handle* h, int32_t* host_out);
int dg_cell_levels(const dg_handle* h, int32_t* host_out);

/* ---- instrumentation ---------------------------------------------------
 * Per-kernel timing: while enabled, every kernel launch of the handle is
 * bracketed by two CUDA events recorded on the launch stream.  dg_advance and
 * dg_advance_dt then replay graphs recorded with those event pairs as
 * event-record nodes (kept apart from the unprofiled graphs) and wait for
 * each replay on the host (synchronous while profiling).  dg_profile_end
 * waits for the recorded events and returns, per kernel kind, the number of
 * launches and the summed device time in milliseconds. */
enum { DG_KERNEL_FACE = 0, DG_KERNEL_CELL = 1, DG_KERNEL_LIMIT = 2, DG_KERNEL_DT = 3,
       DG_KERNEL_OTHER = 4, DG_KERNEL_ADJOINT = 5, DG_KERNEL_KINDS = 6 };
int dg_profile_begin(dg_handle* h);
int dg_profile_end(dg_handle* h, int* launches, double* total_ms, int n_kinds);

/* ---- allocation-free totals (no handle) --------------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- a host application that owns every
 * device allocation and forbids libraries from allocating, or code running
 * while a stream is captured in global mode, where allocation calls are not
 * permitted.  They cannot create a handle (dg_create allocates), but can
 * still reduce the conserved totals sum_K |K| w_{1,i} of a state they hold.
 * It allocates nothing: its per-block partial sums live in one fixed device
 * array inside the library (8 * 5 * DG_NOALLOC_MAX_CELLS / 256 bytes =
 * 2.5 MiB), which every GPU that loads the library keeps until the process
 * exits.
 *   W_dev       state [dim+2][n_basis][n_cells], caller-owned device memory:
 *               double for precision DG_FP64, DG_MIXED or DG_MIXED_TC, float
 *               for DG_FP32 or DG_FP32_TC
 *   levels_dev  optional device int32[n_cells] refinement level per cell
 *               (NULL: all cells have edge dx0); |K| = (dx0 / 2^level)^dim
 *   totals_dev  device double[dim+2] result
 * Returns DG_ERR_ARG for bad arguments or n_cells > DG_NOALLOC_MAX_CELLS,
 * DG_ERR_CUDA if one of its own CUDA calls or launches fails (errors left by
 * earlier, unrelated calls of the thread are neither returned nor cleared).
 * It runs on the current device, which must be the one holding W_dev,
 * levels_dev and totals_dev.  The first call on a device looks up the
 * array's device address (once per device, with that device current); make
 * that first call before any stream capture.  The cached address does not
 * survive cudaDeviceReset: do not call this again in a process that has
 * reset the device.  All calls share the array: calls that overlap on the
 * GPU (other streams, other threads) race. */
#define DG_NOALLOC_MAX_CELLS (1 << 24)
int dg_totals_noalloc(int dim, int n_basis, int64_t n_cells, int precision, double dx0,
                      const int32_t* levels_dev, const void* W_dev, double* totals_dev,
                      void* stream);

/* Test hook for the status path of the tensor-core cell kernel's bounded
 * waits (no counterpart in the paper).  Arms the handle's next tensor-core
 * cell-kernel launch made outside a CUDA graph (dg_rhs, dg_rk_step, ...):
 * in that launch the first CTA does not issue its first tensor-core multiply
 * nor the commit that would complete its barrier, and polls that barrier
 * with a short limit (2^12 tries instead of 2^24).  The wait therefore gives
 * up while none of the CTA's tensor-core work is in flight; the CTA stops,
 * frees its tensor memory and latches DG_ERR_TIMEOUT, which dg_status then
 * returns.  The outputs of that launch are invalid; later launches run
 * normally.  DG_ERR_UNSUPPORTED for handles without the tensor-core kernel
 * (precisions other than DG_FP32_TC and DG_MIXED_TC). */
int dg_test_force_timeout(dg_handle* h);

/* Test hook (no counterpart in the paper): the flux formulas' own reciprocal
 * (Euler flux 1/rho, HLLC) and square root (HLLC sound speeds) of n device
 * doubles x_dev[i] (normal; nonzero for a reciprocal, positive for a root),
 * into out_dev: op 0 FP64 reciprocal, 1 FP64 root, 2 FP32 reciprocal and 3
 * FP32 root of (float)x, widened.  All refine the hardware's approximations
 * and stay within an ulp or two of the correctly rounded value; the test
 * checks that bound.  Asynchronous on the stream; DG_ERR_ARG for NULL
 * pointers, n < 0 or another op. */
int dg_test_flux_math(int op, const double* x_dev, double* out_dev, int64_t n, void* stream);

/* Test hook (host only: no device work, usable without a GPU): the mesh
 * tables dg_create builds for meshes[0] (n_problems = 1; Sec. 4: base cells,
 * refined base cells replaced by their 2^dim children, hanging faces), or
 * dg_create_batch for n_problems meshes (cells, faces and table entries
 * concatenated in problem order, indices shifted by the offsets).
 * counts[3] receives the numbers of cells, faces and refined base cells.
 * Each non-NULL array is filled (caller-owned host memory; call first with
 * NULL arrays to size them):
 *   nbr[2*dim][cells]   as dg_neighbor_table;
 *   levels[cells]       as dg_cell_levels;
 *   faces[3][faces]     minus cell, plus cell (-1 for the missing cell of a
 *                       face on a transmissive boundary), and the packed
 *                       face info axis | vm << 2 |
 *                       vp << 5, where a nonzero variant vm (vp) marks the
 *                       minus (plus) side as the coarse side of a hanging
 *                       face and gives 1 + the quadrant of that side's face
 *                       the sub-face covers;
 *   sface[2*dim][cells] the face of each cell side (side = 2*axis + {0:-, 1:+});
 *                       on the coarse side of a hanging face its first
 *                       sub-face, the others following in quadrant order;
 *   prob[cells]         the problem of each cell.
 * DG_ERR_ARG for NULL meshes or counts, n_problems < 1, or meshes that
 * dg_create / dg_create_batch reject with DG_ERR_ARG; DG_ERR_UNSUPPORTED for a
 * batch with refined meshes. */
int dg_test_mesh_tables(const dg_mesh_desc* meshes, int n_problems, int64_t* counts, int32_t* nbr,
                        int32_t* levels, int32_t* faces, int32_t* sface, int32_t* prob);

/* Test hook (host only): the stage program dg_create derives from the SSP
 * Runge-Kutta tableau of order rk_order (1..4; Appendix D), unlimited
 * (limited = 0) or with the limiter pass after every stage (limited = 1).
 * A step runs the program's ops in order on registers R[0] = the caller's
 * state W and scratch registers R[1..n_regs]: op i evaluates K = dW/dt at
 * R[in_reg]; then, for each output o in order,
 *   R[out[o]] = ck[o] * dt * K + sum_r C[o][r] * R[in[r]],
 * an input equal to in_reg reading that register's value at the start of
 * the op; then, when lim_src >= 0, R[lim_dst] = limit(R[lim_src]).  (The
 * FP64-state mixed modes keep the unlimited registers as FP32 differences
 * from W; the program is the same.)  With ops_out non-NULL it receives
 * max_ops records of DG_TEST_OP_DOUBLES doubles each: in_reg, n_in, n_out,
 * lim_src, lim_dst, in[4], out[3] (-1 past n_in, n_out), C[3][4]
 * (row-major), ck[3].  *n_ops and *n_regs are always written.  DG_ERR_ARG for
 * a bad order or flag, NULL counters or max_ops below the op count. */
#define DG_TEST_OP_DOUBLES 27
int dg_test_stage_program(int rk_order, int limited, double* ops_out, int max_ops, int* n_ops, int* n_regs);

/* Reads and clears the device status word (DG_OK, DG_ERR_NONPHYSICAL, ...).
 * Synchronises the handle's last stream. */
int dg_status(dg_handle* h, int* device_status_host);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */
