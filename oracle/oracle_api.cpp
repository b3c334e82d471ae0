// Oracle C API (test infrastructure only): thin extern "C" wrappers around
// the plain FP64 scheme in scheme.hpp.
#include "oracle.h"

#include <cstring>
#include <string>

#include "scheme.hpp"

struct orc_problem {
  orc::Problem P;
};

static std::string g_err;

extern "C" {

const char* orc_last_error(void) { return g_err.c_str(); }

orc_problem* orc_create(int dim, const int* n, const double* lo, const double* hi, const int* bc,
                        int n_boxes, const int* boxes, int k, double gamma, int rk_order,
                        double cfl, int limiter, double beta, double Mtilde, int positivity,
                        double eps, int tensor) {
  try {
    if (dim != 2 && dim != 3) throw std::runtime_error("dim must be 2 or 3");
    if (k < 0 || k > 6) throw std::runtime_error("k must be 0..6");
    auto* o = new orc_problem();
    orc::Problem& P = o->P;
    P.dim = dim;
    P.k = k;
    P.gamma = gamma;
    P.rk_order = rk_order;
    P.cfl = cfl;
    P.limiter = limiter;
    P.beta = beta;
    P.Mtilde = Mtilde;
    P.positivity = positivity;
    P.eps = eps;
    P.tensor = tensor != 0;
    P.mesh.build(dim, n, lo, hi, bc, n_boxes, boxes);
    P.setup();
    return o;
  } catch (const std::exception& e) {
    g_err = e.what();
    return nullptr;
  }
}

void orc_destroy(orc_problem* p) { delete p; }

int64_t orc_n_cells(const orc_problem* p) { return p->P.mesh.ncells; }
int orc_n_nodes(const orc_problem* p) { return p->P.mesh.nnodes; }
int orc_n_basis(const orc_problem* p) { return p->P.N; }
int orc_n_vars(const orc_problem* p) { return p->P.nv; }
int orc_n_qpoints(const orc_problem* p) { return p->P.vol.n; }
int orc_n_l1points(const orc_problem* p) { return p->P.l1rule.n; }

void orc_cell_levels(const orc_problem* p, int32_t* level) {
  for (int c = 0; c < p->P.mesh.ncells; ++c) level[c] = p->P.mesh.level[c];
}
void orc_cell_dx(const orc_problem* p, double* dx) {
  for (int c = 0; c < p->P.mesh.ncells; ++c) dx[c] = p->P.mesh.dx(c);
}
void orc_neighbor_table(const orc_problem* p, int32_t* out) {
  std::memcpy(out, p->P.mesh.nbr.data(), p->P.mesh.nbr.size() * sizeof(int32_t));
}
void orc_node_children(const orc_problem* p, int32_t* out) {
  const auto& M = p->P.mesh;
  for (int m = 0; m < M.nnodes; ++m)
    for (int ch = 0; ch < (1 << M.dim); ++ch) out[m * (1 << M.dim) + ch] = M.node_children[m][ch];
}
void orc_quad_points(const orc_problem* p, double* xyz) { p->P.rule_points(p->P.vol, xyz); }
void orc_l1_points(const orc_problem* p, double* xyz) { p->P.rule_points(p->P.l1rule, xyz); }

void orc_project(const orc_problem* p, const double* u_q, double* W) { p->P.project(u_q, W); }
void orc_rhs(const orc_problem* p, const double* W, double* dWdt) { p->P.rhs(W, dWdt); }
double orc_compute_dt(const orc_problem* p, const double* W) { return p->P.compute_dt(W); }
void orc_set_accel(orc_problem* p, const double* accel) {
  auto& P = p->P;
  if (!accel) {
    P.accel.clear();
    return;
  }
  P.accel.assign(accel, accel + (size_t)P.dim * P.vol.n * P.mesh.ncells);
}
double orc_rk_step(const orc_problem* p, double* W, double dt) { return p->P.rk_step(W, dt); }
void orc_set_threads(orc_problem* p, int n) { p->P.threads = n > 1 ? n : 1; }
void orc_slope_limit(const orc_problem* p, double* W) { p->P.slope_limit(W); }
void orc_positivity_limit(const orc_problem* p, double* W) { p->P.positivity_limit(W); }
void orc_limit(const orc_problem* p, double* W) { p->P.limit(W); }
void orc_totals(const orc_problem* p, const double* W, double* totals) { p->P.totals(W, totals); }
double orc_l1_density(const orc_problem* p, const double* W, const double* rho_exact) {
  return p->P.l1_density(W, rho_exact);
}
void orc_rhs_cells(const orc_problem* p, const double* W, const int32_t* cells, int n, double* out) {
  const size_t per = (size_t)p->P.nv * p->P.N;
  for (int i = 0; i < n; ++i) p->P.rhs_one(W, cells[i], out + per * i);
}
void orc_limit_cells(const orc_problem* p, const double* W, const int32_t* cells, int n, double* out) {
  const size_t per = (size_t)p->P.nv * p->P.N;
  for (int i = 0; i < n; ++i) p->P.limit_one(W, cells[i], out + per * i);
}
void orc_node_weights(const orc_problem* p, const double* W, double* Wnode) {
  p->P.node_weights(W, Wnode);
}
int orc_n_base(const orc_problem* p) { return p->P.mesh.n[0] * p->P.mesh.n[1] * p->P.mesh.n[2]; }
void orc_adapt_flags(const orc_problem* p, const double* W, double w_t, double alpha, int* flags) {
  const std::vector<int> f = p->P.adapt_flags(W, w_t, alpha);
  for (size_t b = 0; b < f.size(); ++b) flags[b] = f[b];
}
void orc_adapt_project(const orc_problem* p_new, const orc_problem* p_old, const double* W_old,
                       double* W_new) {
  p_new->P.adapt_project(p_old->P, W_old, W_new);
}
void orc_rk_step_jvp(const orc_problem* p, const double* W, const double* V, double dt,
                     double* W_out, double* JV) {
  p->P.rk_step_jvp(W, V, dt, W_out, JV);
}

void orc_gauss_legendre(int n, double* x, double* w) {
  std::vector<double> xx, ww;
  orc::gauss_legendre(n, xx, ww);
  for (int i = 0; i < n; ++i) { x[i] = xx[i]; w[i] = ww[i]; }
}
void orc_gauss_lobatto(int n, double* x, double* w) {
  std::vector<double> xx, ww;
  orc::gauss_lobatto(n, xx, ww);
  for (int i = 0; i < n; ++i) { x[i] = xx[i]; w[i] = ww[i]; }
}
void orc_legendre(int n, double x, double* P, double* dP) { orc::legendre_all(n, x, P, dP); }
void orc_basis_exponents(int dim, int k, int* e) {
  orc::Basis b(dim, k);
  for (int l = 0; l < b.N; ++l)
    for (int a = 0; a < 3; ++a) e[l * 3 + a] = b.e[l][a];
}
void orc_basis_exponents_tensor(int dim, int k, int* e) {
  const orc::Basis B(dim, k, true);
  for (int l = 0; l < B.N; ++l)
    for (int a = 0; a < 3; ++a) e[3 * l + a] = B.e[l][a];
}
double orc_basis_phi_tensor(int dim, int k, int l, const double* xi) { return orc::Basis(dim, k, true).phi(l, xi); }
double orc_basis_phi(int dim, int k, int l, const double* xi) { return orc::Basis(dim, k).phi(l, xi); }
double orc_basis_dphi(int dim, int k, int l, int a, const double* xi) {
  return orc::Basis(dim, k).dphi(l, a, xi);
}
void orc_refinement_matrix(int dim, int k, int child, double* Pm) {
  orc::Problem P;
  P.dim = dim;
  P.k = k;
  P.rk_order = 1;
  P.setup();
  const int N = P.N;
  for (int i = 0; i < N * N; ++i) Pm[i] = P.Pref[(size_t)child * N * N + i];
}
void orc_eigen_matrices(int dim, double gamma, const double* u, int a, double* L, double* R) {
  orc::eigen_matrices(dim, gamma, u, a, L, R);
}
void orc_flux(int dim, double gamma, const double* u, int a, double* f) {
  orc::euler_flux(dim, gamma, u, a, f);
}
void orc_flux_jacobian(int dim, double gamma, const double* u, int a, double* J) {
  const int nv = dim + 2;
  for (int j = 0; j < nv; ++j) {
    orc::Dual ud[5], fd[5];
    for (int i = 0; i < nv; ++i) ud[i] = orc::Dual(u[i], i == j ? 1.0 : 0.0);
    orc::euler_flux(dim, gamma, ud, a, fd);
    for (int i = 0; i < nv; ++i) J[i * nv + j] = fd[i].d;
  }
}
void orc_hllc(int dim, double gamma, const double* uL, const double* uR, int a, double* F) {
  orc::hllc(dim, gamma, uL, uR, a, F);
}
int orc_rk_tableau(int order, double* A, double* b, double* c) {
  orc::Tableau t = orc::tableau(order);
  for (int i = 0; i < t.s * t.s; ++i) A[i] = t.A[i];
  for (int i = 0; i < t.s; ++i) { b[i] = t.b[i]; c[i] = t.c[i]; }
  return t.s;
}
// Integrate a scalar ODE dy/dt = f(y) with the same Butcher stepper as the
// scheme: problem 0: f = -y; problem 1: f = y^2.
double orc_rk_ode(int order, int problem, double y0, double t_end, int nsteps) {
  orc::Tableau t = orc::tableau(order);
  std::vector<double> y(1, y0);
  const double dt = t_end / nsteps;
  for (int n = 0; n < nsteps; ++n)
    orc::rk_butcher<double>(
        t, y, dt,
        [&](const std::vector<double>& U, std::vector<double>& K) {
          K[0] = problem == 0 ? -U[0] : U[0] * U[0];
        },
        std::function<void(std::vector<double>&)>());
  return y[0];
}
double orc_minmod_b(double a, double b, double c, double Mtilde, double dx) {
  orc::Problem P;
  P.Mtilde = Mtilde;
  return P.minmodB(a, b, c, dx);
}
double orc_solve_tau(int dim, double gamma, double eps, const double* ubar, const double* u) {
  orc::Problem P;
  P.dim = dim;
  P.nv = dim + 2;
  P.gamma = gamma;
  P.eps = eps;
  return P.solve_tau(ubar, u);
}

}  // extern "C"
