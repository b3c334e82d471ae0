/* Oracle C API -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 CPU implementation of the modal DG scheme of Schaal et
 * al. (2015) for the Euler equations, used to check the CUDA library.  Only
 * tests/, __graft_entry__.smoke() and the cpu_baseline / reference leg of
 * bench.py may load it.  It shares no code with the library.
 *
 * Layouts (the library's interface format): weights W[var][coef][cell],
 * point values u[var][q][cell], coordinates xyz[axis][q][cell], neighbour
 * table nbr[side][cell] (side = 2*axis + {0:-,1:+}).
 */
#ifndef DG_ORACLE_H
#define DG_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_problem orc_problem;

/* boxes: n_boxes x (2*dim) inclusive base-cell index ranges (lo..., hi...) */
orc_problem* orc_create(int dim, const int* n, const double* lo, const double* hi, const int* bc,
                        int n_boxes, const int* boxes, int k, double gamma, int rk_order,
                        double cfl, int limiter, double beta, double Mtilde, int positivity,
                        double eps, int tensor);
void orc_destroy(orc_problem* p);
const char* orc_last_error(void);

int64_t orc_n_cells(const orc_problem* p);
int orc_n_nodes(const orc_problem* p);
int orc_n_basis(const orc_problem* p);
int orc_n_vars(const orc_problem* p);
int orc_n_qpoints(const orc_problem* p);
int orc_n_l1points(const orc_problem* p);

void orc_cell_levels(const orc_problem* p, int32_t* level);
void orc_cell_dx(const orc_problem* p, double* dx);
void orc_neighbor_table(const orc_problem* p, int32_t* out);
void orc_node_children(const orc_problem* p, int32_t* out); /* [nodes][2^d] */
void orc_quad_points(const orc_problem* p, double* xyz);
void orc_l1_points(const orc_problem* p, double* xyz);

void orc_project(const orc_problem* p, const double* u_q, double* W);
void orc_rhs(const orc_problem* p, const double* W, double* dWdt);
double orc_compute_dt(const orc_problem* p, const double* W);
/* external acceleration a = -grad Phi at the volume points, [dim][Q][cells]
   (copied); NULL removes it.  Adds the gravity source (eq. gravity_term) to the
   right-hand side and the gravity bound (Sec. 2.5) to the timestep. */
void orc_set_accel(orc_problem* p, const double* accel);
double orc_rk_step(const orc_problem* p, double* W, double dt);
/* OpenMP threads of orc_rk_step's right-hand side: n > 1 evaluates it cell by
 * cell (gather form, no races), n <= 1 with the face scatter (default). */
void orc_set_threads(orc_problem* p, int n);
void orc_slope_limit(const orc_problem* p, double* W);
void orc_positivity_limit(const orc_problem* p, double* W);
void orc_limit(const orc_problem* p, double* W);
void orc_totals(const orc_problem* p, const double* W, double* totals);
double orc_l1_density(const orc_problem* p, const double* W, const double* rho_exact);
/* per-cell evaluations for sampled comparisons: out[k][v][l] for cells[k] */
void orc_rhs_cells(const orc_problem* p, const double* W, const int32_t* cells, int n, double* out);
void orc_limit_cells(const orc_problem* p, const double* W, const int32_t* cells, int n, double* out);
void orc_node_weights(const orc_problem* p, const double* W, double* Wnode);
/* base cells of the mesh (lexicographic) */
int orc_n_base(const orc_problem* p);
/* new refinement flag per base cell: criteria of eqs. cell_ref / node_ref plus one buffer layer */
void orc_adapt_flags(const orc_problem* p, const double* W, double w_t, double alpha, int* flags);
/* W_new on p_new's mesh from W_old on p_old's (same base grid): copy, refine or merge */
void orc_adapt_project(const orc_problem* p_new, const orc_problem* p_old, const double* W_old,
                       double* W_new);
void orc_rk_step_jvp(const orc_problem* p, const double* W, const double* V, double dt,
                     double* W_out, double* JV);

/* building blocks, for pins */
void orc_gauss_legendre(int n, double* x, double* w);
void orc_gauss_lobatto(int n, double* x, double* w);
void orc_legendre(int n, double x, double* P, double* dP);
void orc_basis_exponents(int dim, int k, int* e); /* [N][3] */
/* the same for the tensor-product basis Q_k ((k+1)^dim functions) */
void orc_basis_exponents_tensor(int dim, int k, int* e);
double orc_basis_phi_tensor(int dim, int k, int l, const double* xi);
double orc_basis_phi(int dim, int k, int l, const double* xi);
double orc_basis_dphi(int dim, int k, int l, int a, const double* xi);
void orc_refinement_matrix(int dim, int k, int child, double* P); /* [N][N], (j,l) */
void orc_eigen_matrices(int dim, double gamma, const double* u, int a, double* L, double* R);
void orc_flux(int dim, double gamma, const double* u, int a, double* f);
void orc_flux_jacobian(int dim, double gamma, const double* u, int a, double* J); /* [nv][nv] */
void orc_hllc(int dim, double gamma, const double* uL, const double* uR, int a, double* F);
int orc_rk_tableau(int order, double* A, double* b, double* c);
double orc_rk_ode(int order, int problem, double y0, double t_end, int nsteps);
double orc_minmod_b(double a, double b, double c, double Mtilde, double dx);
double orc_solve_tau(int dim, double gamma, double eps, const double* ubar, const double* u);

#ifdef __cplusplus
}
#endif
#endif
