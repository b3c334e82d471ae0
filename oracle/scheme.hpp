// Oracle (test infrastructure only): the modal DG scheme for the Euler
// equations -- L2 projection, right-hand side, SSP Runge-Kutta stepping,
// timestep, slope and positivity limiters, AMR projections, conservation
// totals and the L1 density error -- as plain, slow FP64 loops.
//
// Every function follows the paper's statement of it (section / equation
// named in its comment).  Where the paper is silent or garbled the reading
// taken is stated at the function.  Nothing here is blocked, fused or
// reordered for speed.
#pragma once
#include <algorithm>
#include <cmath>
#include <functional>
#include <stdexcept>
#include <map>
#include <vector>

#include "euler.hpp"
#include "mesh.hpp"
#include "quadrature.hpp"

namespace orc {

enum { LIM_NONE = 0, LIM_COMPONENT = 1, LIM_CHARACTERISTIC = 2 };

// Butcher tableaux of the SSP RK methods (Appendix D, Tables RK_2, RK_3,
// RK_4; order 1 is the forward Euler method).  A is s x s row-major.
struct Tableau {
  int s = 0;
  std::vector<double> A, b, c;
};
inline Tableau tableau(int order) {
  Tableau t;
  if (order == 1) {
    t.s = 1; t.A = {0}; t.b = {1}; t.c = {0};
  } else if (order == 2) {
    t.s = 2; t.A = {0, 0, 1, 0}; t.b = {0.5, 0.5}; t.c = {0, 1};
  } else if (order == 3) {
    t.s = 3;
    t.A = {0, 0, 0, 1, 0, 0, 0.25, 0.25, 0};
    t.b = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
    t.c = {0, 1, 0.5};
  } else if (order == 4) {
    t.s = 5;
    t.A.assign(25, 0.0);
    t.A[1 * 5 + 0] = 0.39175222700392;
    t.A[2 * 5 + 0] = 0.21766909633821;
    t.A[2 * 5 + 1] = 0.36841059262959;
    t.A[3 * 5 + 0] = 0.08269208670950;
    t.A[3 * 5 + 1] = 0.13995850206999;
    t.A[3 * 5 + 2] = 0.25189177424738;
    t.A[4 * 5 + 0] = 0.06796628370320;
    t.A[4 * 5 + 1] = 0.11503469844438;
    t.A[4 * 5 + 2] = 0.20703489864929;
    t.A[4 * 5 + 3] = 0.54497475021237;
    t.b = {0.14681187618661, 0.24848290924556, 0.10425883036650, 0.27443890091960,
           0.22600748319395};
    t.c = {0, 0.39175222700392, 0.58607968896779, 0.47454236302687, 0.93501063100924};
  } else {
    throw std::runtime_error("rk order must be 1..4");
  }
  return t;
}

// Explicit RK step in Butcher form (Appendix D, eq. rhs):
//   k_i = L(U_i),  U_i = w + dt sum_{j<i} a_ij k_j,  w_new = w + dt sum_i b_i k_i,
// where L = -R is the time derivative.  When limiting is on, every stage state
// U_i (i >= 2) and the new state are limited before use (main loop, Sec. 4.5).
template <class T>
void rk_butcher(const Tableau& tb, std::vector<T>& w, double dt,
                const std::function<void(const std::vector<T>&, std::vector<T>&)>& L,
                const std::function<void(std::vector<T>&)>& limit) {
  const size_t n = w.size();
  std::vector<std::vector<T>> k(tb.s, std::vector<T>(n));
  std::vector<T> U(n);
  for (int i = 0; i < tb.s; ++i) {
    U = w;
    for (int j = 0; j < i; ++j) {
      const double a = tb.A[i * tb.s + j];
      if (a == 0.0) continue;
      for (size_t m = 0; m < n; ++m) U[m] += (dt * a) * k[j][m];
    }
    if (i > 0 && limit) limit(U);
    L(U, k[i]);
  }
  for (int i = 0; i < tb.s; ++i)
    for (size_t m = 0; m < n; ++m) w[m] += (dt * tb.b[i]) * k[i][m];
  if (limit) limit(w);
}

struct Problem {
  Mesh mesh;
  Basis basis;
  int dim = 2, k = 1, N = 1, nv = 4;
  double gamma = 1.4;
  int rk_order = 2;
  double cfl = 0.2;
  int limiter = LIM_NONE;
  int threads = 1;               // OpenMP threads of rk_step's right-hand side (gather form if > 1)
  bool tensor = false;           // tensor-product basis Q_k instead of the total-degree basis
  double beta = 1.0, Mtilde = 0.5;
  int positivity = 0;
  double eps = 1e-10;

  std::vector<double> gx, gw;    // 1D Gauss-Legendre, k+1 points
  std::vector<double> lx, lw;    // 1D Gauss-Lobatto, m points (positivity limiter)
  TensorRule vol;                // (k+1)^dim volume rule
  TensorRule l1rule;             // (k+3)^dim rule for the L1 error
  std::vector<double> phi_vol;   // [q][l]
  std::vector<double> dphi_vol;  // [a][q][l]
  int nfq = 1;                   // face points (k+1)^(dim-1)
  std::vector<double> fw;        // face weights [nfq]
  // phi at face points: [a][side][variant][q][l]; variant 0 = whole face,
  // variant 1+s = the sub-face quadrant s mapped into this cell's frame
  std::vector<double> phi_face;
  int nvariant = 1;
  std::vector<double> Pref;      // refinement matrices [child][j][l]
  std::vector<std::array<double, 3>> Spts;  // union point set S (eq. union_quad_points)
  Tableau tb;
  // external acceleration a = -grad Phi at the volume points, [a][q][cell];
  // empty: no gravity (eq. gravity_term)
  std::vector<double> accel;

  size_t idx(int v, int l, int c) const { return ((size_t)v * N + l) * mesh.ncells + c; }
  size_t size() const { return (size_t)nv * N * mesh.ncells; }
  int tang(int a, int i) const {  // i-th tangential axis of a face with normal a
    int t = 0;
    for (int b = 0; b < dim; ++b) {
      if (b == a) continue;
      if (t == i) return b;
      ++t;
    }
    return -1;
  }
  // point of face (a, side) in the cell frame; variant as above
  void face_point(int a, int side, int variant, int q, double* xi) const {
    xi[0] = xi[1] = xi[2] = 0.0;
    xi[a] = side ? 1.0 : -1.0;
    int qq = q;
    for (int i = 0; i < dim - 1; ++i) {
      const int t = tang(a, i);
      double eta = gx[qq % (k + 1)];
      qq /= (k + 1);
      if (variant > 0) {
        const int bit = ((variant - 1) >> i) & 1;
        eta = 0.5 * (eta + (2.0 * bit - 1.0));
      }
      xi[t] = eta;
    }
  }
  double pf(int a, int side, int variant, int q, int l) const {
    return phi_face[((((size_t)a * 2 + side) * nvariant + variant) * nfq + q) * N + l];
  }

  void setup() {
    basis = Basis(dim, k, tensor);
    N = basis.N;
    nv = dim + 2;
    gauss_legendre(k + 1, gx, gw);
    vol = TensorRule(dim, gx, gw);
    std::vector<double> x3, w3;
    gauss_legendre(k + 3, x3, w3);
    l1rule = TensorRule(dim, x3, w3);
    phi_vol.assign((size_t)vol.n * N, 0.0);
    dphi_vol.assign((size_t)dim * vol.n * N, 0.0);
    for (int q = 0; q < vol.n; ++q)
      for (int l = 0; l < N; ++l) {
        phi_vol[(size_t)q * N + l] = basis.phi(l, vol.xi[q].data());
        for (int a = 0; a < dim; ++a)
          dphi_vol[((size_t)a * vol.n + q) * N + l] = basis.dphi(l, a, vol.xi[q].data());
      }
    nfq = 1;
    for (int i = 0; i < dim - 1; ++i) nfq *= (k + 1);
    fw.assign(nfq, 1.0);
    for (int q = 0; q < nfq; ++q) {
      int qq = q;
      for (int i = 0; i < dim - 1; ++i) {
        fw[q] *= gw[qq % (k + 1)];
        qq /= (k + 1);
      }
    }
    nvariant = 1 + (1 << (dim - 1));
    phi_face.assign((size_t)dim * 2 * nvariant * nfq * N, 0.0);
    for (int a = 0; a < dim; ++a)
      for (int s = 0; s < 2; ++s)
        for (int v = 0; v < nvariant; ++v)
          for (int q = 0; q < nfq; ++q) {
            double xi[3];
            face_point(a, s, v, q, xi);
            for (int l = 0; l < N; ++l)
              phi_face[((((size_t)a * 2 + s) * nvariant + v) * nfq + q) * N + l] = basis.phi(l, xi);
          }
    // refinement matrices (eq. ref_pa_integral): (P_c)_{j,l} = 2^-d int phi_j(eta)
    // phi_l((eta + o_c)/2) d eta, the coarse function taken at the mapped point
    const int nch = 1 << dim;
    Pref.assign((size_t)nch * N * N, 0.0);
    for (int ch = 0; ch < nch; ++ch)
      for (int q = 0; q < vol.n; ++q) {
        double xc[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) xc[a] = 0.5 * (vol.xi[q][a] + (((ch >> a) & 1) ? 1.0 : -1.0));
        for (int j = 0; j < N; ++j)
          for (int l = 0; l < N; ++l)
            Pref[((size_t)ch * N + j) * N + l] +=
                std::ldexp(1.0, -dim) * basis.phi(j, vol.xi[q].data()) * basis.phi(l, xc) * vol.w[q];
      }
    // positivity point set S = S_1 u ... u S_dim (eq. union_quad_points):
    // Gauss-Lobatto in direction a, Gauss-Legendre in the others;
    // m = smallest integer >= (k+3)/2
    const int m = (k + 4) / 2;
    gauss_lobatto(std::max(m, 2), lx, lw);
    Spts.clear();
    for (int a = 0; a < dim; ++a) {
      const int cnt = (int)lx.size() * nfq;
      for (int i = 0; i < cnt; ++i) {
        double xi[3] = {0, 0, 0};
        xi[a] = lx[i % lx.size()];
        int qq = i / (int)lx.size();
        for (int t = 0; t < dim - 1; ++t) {
          xi[tang(a, t)] = gx[qq % (k + 1)];
          qq /= (k + 1);
        }
        Spts.push_back({xi[0], xi[1], xi[2]});
      }
    }
    tb = tableau(rk_order);
  }

  // -------------------------------------------------------------------------
  // u(xi) in cell c: sum_l w_l phi_l (eq. solution_representation)
  template <class T>
  void eval(const T* W, int c, const double* phi_row, T* u) const {
    for (int v = 0; v < nv; ++v) {
      T s = T(0.0);
      for (int l = 0; l < N; ++l) s += W[idx(v, l, c)] * phi_row[l];
      u[v] = s;
    }
  }

  // Time derivative dw/dt = -R_K (eqs. dg_projected, dg_term2, dg_term3,
  // spatial_discretisation).  With dV = (dx/2)^d d xi and d/dx = (2/dx) d/dxi:
  //   dw_j/dt = 2^(1-d)/dx [ sum_a sum_q f_a(u_q) dphi_j/dxi_a w_q
  //                          - sum_faces sum_q fbar_q phi_j w_q ].
  // Faces: a face between equal-level cells is visited once from its minus
  // side; a face between a fine cell and a coarser one is visited from the
  // fine cell at the fine face's Gauss points, the coarse cell integrating
  // that sub-face with weights w_q / 2^(d-1) (Fig. dg_amr).  Non-periodic
  // boundaries are transmissive: the outer state equals the inner trace.
  template <class T>
  void rhs(const T* W, T* dW) const {
    const int nc = mesh.ncells;
    std::vector<T> V(size(), T(0.0)), S(size(), T(0.0));
    T u[5], f[5];
    for (int c = 0; c < nc; ++c) {
      for (int q = 0; q < vol.n; ++q) {
        eval(W, c, &phi_vol[(size_t)q * N], u);
        for (int a = 0; a < dim; ++a) {
          euler_flux(dim, gamma, u, a, f);
          for (int v = 0; v < nv; ++v)
            for (int j = 0; j < N; ++j)
              V[idx(v, j, c)] += f[v] * (dphi_vol[((size_t)a * vol.n + q) * N + j] * vol.w[q]);
        }
      }
    }
    const double sub_w = std::ldexp(1.0, -(dim - 1));
    T uc[5], un[5], F[5];
    for (int c = 0; c < nc; ++c) {
      for (int a = 0; a < dim; ++a)
        for (int s = 0; s < 2; ++s) {
          const int nb = mesh.nbr[(size_t)(2 * a + s) * nc + c];
          int kind;  // 0 boundary, 1 same level, 2 coarser neighbour
          if (nb == -1) kind = 0;
          else if (nb <= -2) continue;
          else if (mesh.level[nb] == mesh.level[c]) {
            if (s == 0) continue;
            kind = 1;
          } else if (mesh.level[nb] == mesh.level[c] - 1) kind = 2;
          else throw std::runtime_error("unsupported level jump");
          int variant = 0;
          if (kind == 2) {
            int quad = 0;
            for (int i = 0; i < dim - 1; ++i) quad |= (mesh.coord[c][tang(a, i)] & 1) << i;
            variant = 1 + quad;
          }
          for (int q = 0; q < nfq; ++q) {
            double tmp[64];
            for (int l = 0; l < N; ++l) tmp[l] = pf(a, s, 0, q, l);
            eval(W, c, tmp, uc);
            if (kind == 0) {
              for (int v = 0; v < nv; ++v) un[v] = uc[v];
            } else {
              for (int l = 0; l < N; ++l) tmp[l] = pf(a, 1 - s, variant, q, l);
              eval(W, nb, tmp, un);
            }
            if (s == 1) hllc(dim, gamma, uc, un, a, F);
            else hllc(dim, gamma, un, uc, a, F);
            const double sc = s ? 1.0 : -1.0;
            for (int v = 0; v < nv; ++v)
              for (int j = 0; j < N; ++j) S[idx(v, j, c)] += F[v] * (sc * pf(a, s, 0, q, j) * fw[q]);
            if (kind != 0) {
              const double wn = fw[q] * (kind == 2 ? sub_w : 1.0);
              for (int v = 0; v < nv; ++v)
                for (int j = 0; j < N; ++j)
                  S[idx(v, j, nb)] += F[v] * (-sc * pf(a, 1 - s, variant, q, j) * wn);
            }
          }
        }
    }
    std::vector<T> G(accel.empty() ? 0 : size(), T(0.0));
    if (!accel.empty())
      for (int c = 0; c < nc; ++c) source_moments(W, c, &G[0], nc);
    for (int c = 0; c < nc; ++c) {
      const double pre = std::ldexp(1.0, 1 - dim) / mesh.dx(c);
      for (int v = 0; v < nv; ++v)
        for (int j = 0; j < N; ++j) {
          dW[idx(v, j, c)] = pre * (V[idx(v, j, c)] - S[idx(v, j, c)]);
          if (!accel.empty()) dW[idx(v, j, c)] += std::ldexp(1.0, -dim) * G[idx(v, j, c)];
        }
    }
  }

  // Gravity source (eq. gravity_term): s = (0, rho a, m . a) with a = -grad Phi,
  // projected with the volume rule, sum_q s(u_q) phi_j(xi_q) w_q; the moment of
  // cell c goes to out[(v * N + j) * stride + c] (the caller scales it by
  // 2^-d = |K|^-1 (dx/2)^d).
  template <class T>
  void source_moments(const T* W, int c, T* out, int stride) const {
    T u[5];
    const int nc = mesh.ncells;
    for (int q = 0; q < vol.n; ++q) {
      eval(W, c, &phi_vol[(size_t)q * N], u);
      T s[5];
      s[0] = T(0.0);
      s[nv - 1] = T(0.0);
      for (int a = 0; a < dim; ++a) {
        const double aq = accel[((size_t)a * vol.n + q) * nc + c];
        s[1 + a] = u[0] * aq;
        s[nv - 1] = s[nv - 1] + u[1 + a] * aq;
      }
      for (int v = 0; v < nv; ++v)
        for (int j = 0; j < N; ++j)
          out[((size_t)v * N + j) * stride + c] += s[v] * (phi_vol[(size_t)q * N + j] * vol.w[q]);
    }
  }

  // dw/dt of one cell (the same terms as rhs, gathered from the cell's side:
  // every face of the cell, and each fine sub-face of a side with a finer
  // neighbour, is evaluated at its own Gauss points).  Output [v][l].
  void rhs_one(const double* W, int c, double* out) const {
    const int nc = mesh.ncells;
    std::vector<double> V((size_t)nv * N, 0.0), S((size_t)nv * N, 0.0);
    double u[5], f[5], uc[5], un[5], F[5], tmp[64];
    for (int q = 0; q < vol.n; ++q) {
      eval(W, c, &phi_vol[(size_t)q * N], u);
      for (int a = 0; a < dim; ++a) {
        euler_flux(dim, gamma, u, a, f);
        for (int v = 0; v < nv; ++v)
          for (int j = 0; j < N; ++j)
            V[(size_t)v * N + j] += f[v] * (dphi_vol[((size_t)a * vol.n + q) * N + j] * vol.w[q]);
      }
    }
    const double sub_w = std::ldexp(1.0, -(dim - 1));
    for (int a = 0; a < dim; ++a)
      for (int s = 0; s < 2; ++s) {
        const int nb = mesh.nbr[(size_t)(2 * a + s) * nc + c];
        const double sc = s ? 1.0 : -1.0;
        // list of (own variant, neighbour cell, neighbour variant, weight factor)
        std::vector<std::array<int, 3>> parts;
        std::vector<double> wf;
        if (nb == -1) {
          parts.push_back({0, -1, 0});
          wf.push_back(1.0);
        } else if (nb <= -2) {
          const auto& kids = mesh.node_children[-(nb + 2)];
          for (int quad = 0; quad < (1 << (dim - 1)); ++quad) {
            int ch = s ? 0 : (1 << a);  // the layer of the node touching this side
            for (int i = 0; i < dim - 1; ++i)
              if ((quad >> i) & 1) ch |= 1 << tang(a, i);
            parts.push_back({1 + quad, kids[ch], 0});
            wf.push_back(sub_w);
          }
        } else if (mesh.level[nb] == mesh.level[c]) {
          parts.push_back({0, nb, 0});
          wf.push_back(1.0);
        } else {
          int quad = 0;
          for (int i = 0; i < dim - 1; ++i) quad |= (mesh.coord[c][tang(a, i)] & 1) << i;
          parts.push_back({0, nb, 1 + quad});
          wf.push_back(1.0);
        }
        for (size_t p = 0; p < parts.size(); ++p) {
          const int own_var = parts[p][0], n = parts[p][1], n_var = parts[p][2];
          for (int q = 0; q < nfq; ++q) {
            for (int l = 0; l < N; ++l) tmp[l] = pf(a, s, own_var, q, l);
            eval(W, c, tmp, uc);
            if (n < 0) {
              for (int v = 0; v < nv; ++v) un[v] = uc[v];
            } else {
              for (int l = 0; l < N; ++l) tmp[l] = pf(a, 1 - s, n_var, q, l);
              eval(W, n, tmp, un);
            }
            if (s == 1) hllc(dim, gamma, uc, un, a, F);
            else hllc(dim, gamma, un, uc, a, F);
            for (int v = 0; v < nv; ++v)
              for (int j = 0; j < N; ++j)
                S[(size_t)v * N + j] += F[v] * (sc * pf(a, s, own_var, q, j) * fw[q] * wf[p]);
          }
        }
      }
    const double pre = std::ldexp(1.0, 1 - dim) / mesh.dx(c);
    for (size_t i = 0; i < V.size(); ++i) out[i] = pre * (V[i] - S[i]);
    if (!accel.empty()) {
      std::vector<double> G((size_t)nv * N * nc, 0.0);
      source_moments(W, c, G.data(), nc);
      for (int v = 0; v < nv; ++v)
        for (int j = 0; j < N; ++j) out[(size_t)v * N + j] += std::ldexp(1.0, -dim) * G[((size_t)v * N + j) * nc + c];
    }
  }

  // Timestep (eq. time_step; eq. time_step_pos when the positivity limiter
  // is on), from the cell-mean state, minimum over all cells.
  double compute_dt(const double* W) const {
    double fac = cfl / (2.0 * k + 1.0);
    if (positivity) fac = cfl * std::min(1.0 / (2.0 * k + 1.0), lw[0] / 2.0);
    double dt = 1e300;
    double u[5];
    for (int c = 0; c < mesh.ncells; ++c) {
      for (int v = 0; v < nv; ++v) u[v] = W[idx(v, 0, c)];
      const double p = pressure(dim, gamma, u);
      const double cs = std::sqrt(gamma * p / u[0]);
      double sum = 0.0;
      for (int a = 0; a < dim; ++a) sum += (std::fabs(u[1 + a] / u[0]) + cs) / mesh.dx(c);
      dt = std::min(dt, fac / sum);
      if (!accel.empty()) {
        // gravity bound (Sec. 2.5): c / (sqrt(2 gamma (gamma - 1)) |grad Phi|),
        // with the largest |a| over the cell's volume points
        double amax = 0.0;
        for (int q = 0; q < vol.n; ++q) {
          double a2 = 0.0;
          for (int a = 0; a < dim; ++a) {
            const double aq = accel[((size_t)a * vol.n + q) * mesh.ncells + c];
            a2 += aq * aq;
          }
          amax = std::max(amax, std::sqrt(a2));
        }
        if (amax > 0.0) dt = std::min(dt, cs / (std::sqrt(2.0 * gamma * (gamma - 1.0)) * amax));
      }
    }
    return dt;
  }

  // minmod and its TVB-bounded form (Secs. 3.1, 3.3); a zero argument makes
  // the signs unequal, giving 0; the bound is |a| <= Mtilde * dx
  static double minmod(double a, double b, double c) {
    if (a > 0 && b > 0 && c > 0) return std::min(a, std::min(b, c));
    if (a < 0 && b < 0 && c < 0) return -std::min(-a, std::min(-b, -c));
    return 0.0;
  }
  double minmodB(double a, double b, double c, double dx) const {
    if (std::fabs(a) <= Mtilde * dx) return a;
    return minmod(a, b, c);
  }

  // Mean of a neighbour over the same-size region next to cell c across side
  // (a, s), taken from state W (Sec. 4.4): equal level -> its mean; finer
  // (a node) -> mean of the 2^d children (first row of the node weights of
  // eq. deref_weights); coarser -> first row of the refinement projection
  // onto the matching sub-volume; no neighbour -> the cell's own mean.
  void neighbour_mean(const double* W, int c, int a, int s, double* out) const {
    const int nc = mesh.ncells;
    const int nb = mesh.nbr[(size_t)(2 * a + s) * nc + c];
    if (nb == -1) {
      for (int v = 0; v < nv; ++v) out[v] = W[idx(v, 0, c)];
    } else if (nb <= -2) {
      const auto& kids = mesh.node_children[-(nb + 2)];
      for (int v = 0; v < nv; ++v) {
        double sum = 0.0;
        for (int ch : kids) sum += W[idx(v, 0, ch)];
        out[v] = sum / (double)kids.size();
      }
    } else if (mesh.level[nb] == mesh.level[c]) {
      for (int v = 0; v < nv; ++v) out[v] = W[idx(v, 0, nb)];
    } else {
      std::array<int, 3> p = mesh.coord[c];
      p[a] += s ? 1 : -1;
      const int ext = mesh.n[a] << mesh.level[c];
      p[a] = (p[a] + ext) % ext;
      int ch = 0;
      for (int b = 0; b < dim; ++b) ch |= (p[b] & 1) << b;
      for (int v = 0; v < nv; ++v) {
        double sum = 0.0;
        for (int l = 0; l < N; ++l) sum += Pref[((size_t)ch * N + 0) * N + l] * W[idx(v, l, nb)];
        out[v] = sum;
      }
    }
  }

  // Slope limiter (Secs. 3.1-3.3): characteristic (or component-wise)
  // minmodB of sqrt(3) * slope against beta * mean differences.  If any
  // limited value differs from its input, the linear weights become R c~
  // and every weight of degree >= 2 is set to zero.  All inputs are taken
  // from the state before limiting.
  void slope_limit(double* W) const {
    if (limiter == LIM_NONE || k == 0) return;
    const std::vector<double> W0(W, W + size());
    std::vector<double> cellw((size_t)nv * N);
    for (int c = 0; c < mesh.ncells; ++c) {
      if (!slope_limit_cell(W0.data(), c, cellw.data())) continue;
      for (int v = 0; v < nv; ++v)
        for (int l = 0; l < N; ++l) W[idx(v, l, c)] = cellw[(size_t)v * N + l];
    }
  }

  // Slope limiting of cell c with inputs from W0; writes the cell's weights
  // [v][l] to out and returns true if they changed.
  bool slope_limit_cell(const double* W0, int c, double* out) const {
    for (int v = 0; v < nv; ++v)
      for (int l = 0; l < N; ++l) out[(size_t)v * N + l] = W0[idx(v, l, c)];
    if (limiter == LIM_NONE || k == 0) return false;
    const double s3 = std::sqrt(3.0);
    double mean[5];
    for (int v = 0; v < nv; ++v) mean[v] = W0[idx(v, 0, c)];
    bool changed = false;
    double ct[3][5];
    double Rm[3][25];
    for (int a = 0; a < dim; ++a) {
      double L[25], R[25];
      if (limiter == LIM_CHARACTERISTIC) {
        eigen_matrices(dim, gamma, mean, a, L, R);
      } else {
        for (int i = 0; i < nv * nv; ++i) L[i] = R[i] = 0.0;
        for (int i = 0; i < nv; ++i) L[i * nv + i] = R[i * nv + i] = 1.0;
      }
      for (int i = 0; i < nv * nv; ++i) Rm[a][i] = R[i];
      double mm[5], mp[5];
      neighbour_mean(W0, c, a, 0, mm);
      neighbour_mean(W0, c, a, 1, mp);
      for (int i = 0; i < nv; ++i) {
        double cs = 0.0, dm = 0.0, dp = 0.0;
        for (int v = 0; v < nv; ++v) {
          cs += L[i * nv + v] * W0[idx(v, 1 + a, c)];
          dm += L[i * nv + v] * (mean[v] - mm[v]);
          dp += L[i * nv + v] * (mp[v] - mean[v]);
        }
        const double arg = s3 * cs;
        const double lim = minmodB(arg, beta * dm, beta * dp, mesh.dx(c));
        if (lim != arg) changed = true;
        ct[a][i] = lim / s3;
      }
    }
    if (!changed) return false;
    for (int a = 0; a < dim; ++a)
      for (int v = 0; v < nv; ++v) {
        double s = 0.0;
        for (int i = 0; i < nv; ++i) s += Rm[a][v * nv + i] * ct[a][i];
        out[(size_t)v * N + 1 + a] = s;
      }
    for (int l = 0; l < N; ++l)
      if (basis.degree(l) >= 2)
        for (int v = 0; v < nv; ++v) out[(size_t)v * N + l] = 0.0;
    return true;
  }

  // Positivity limiter (Sec. 3.4, after Zhang & Shu 2010).  Points: the set S
  // plus, for cells with finer neighbours, the Gauss points of the fine
  // sub-faces (Sec. 4.4).  theta_1 scales the higher density weights so that
  // rho >= eps at all points; theta_2 = min tau scales all higher weights.
  // Reading of eq. p_positivity: tau solves p(ubar + tau (u - ubar)) = eps,
  // a quadratic in tau; the stable closed-form root is refined by two
  // Newton-Raphson steps.
  std::vector<std::array<double, 3>> positivity_points(int c) const {
    std::vector<std::array<double, 3>> pts = Spts;
    for (int a = 0; a < dim; ++a)
      for (int s = 0; s < 2; ++s) {
        const int nb = mesh.nbr[(size_t)(2 * a + s) * mesh.ncells + c];
        if (nb > -2) continue;
        for (int v = 1; v < nvariant; ++v)
          for (int q = 0; q < nfq; ++q) {
            double xi[3];
            face_point(a, s, v, q, xi);
            pts.push_back({xi[0], xi[1], xi[2]});
          }
      }
    return pts;
  }

  double solve_tau(const double* ub, const double* u) const {
    const double g1 = gamma - 1.0;
    double dl[5];
    for (int v = 0; v < nv; ++v) dl[v] = u[v] - ub[v];
    const int iE = dim + 1;
    double mm = 0, md = 0, dd = 0;
    for (int a = 0; a < dim; ++a) {
      mm += ub[1 + a] * ub[1 + a];
      md += ub[1 + a] * dl[1 + a];
      dd += dl[1 + a] * dl[1 + a];
    }
    // g(tau) = (gamma-1) (E rho - |m|^2/2) - eps rho along the segment
    const double qa = g1 * (dl[iE] * dl[0] - 0.5 * dd);
    const double qb = g1 * (ub[iE] * dl[0] + ub[0] * dl[iE] - md) - eps * dl[0];
    const double qc = g1 * (ub[iE] * ub[0] - 0.5 * mm) - eps * ub[0];
    if (qc <= 0.0) return 0.0;  // the mean itself is not admissible
    double tau;
    if (std::fabs(qa) <= 1e-14 * (std::fabs(qb) + std::fabs(qc))) {
      tau = -qc / qb;
    } else {
      const double disc = std::max(qb * qb - 4.0 * qa * qc, 0.0);
      const double qq = -0.5 * (qb + std::copysign(std::sqrt(disc), qb));
      const double r1 = qq / qa, r2 = qc / qq;
      const bool ok1 = r1 >= 0.0 && r1 <= 1.0, ok2 = r2 >= 0.0 && r2 <= 1.0;
      if (ok1 && ok2) tau = std::min(r1, r2);
      else if (ok1) tau = r1;
      else if (ok2) tau = r2;
      else tau = std::fabs(r1 - 0.5) < std::fabs(r2 - 0.5) ? r1 : r2;
    }
    for (int it = 0; it < 2; ++it) {
      const double g = (qa * tau + qb) * tau + qc;
      const double dg = 2.0 * qa * tau + qb;
      if (dg != 0.0) tau -= g / dg;
    }
    return std::min(std::max(tau, 0.0), 1.0);
  }

  void positivity_limit(double* W) const {
    if (!positivity) return;
    std::vector<double> cellw((size_t)nv * N);
    for (int c = 0; c < mesh.ncells; ++c) {
      for (int v = 0; v < nv; ++v)
        for (int l = 0; l < N; ++l) cellw[(size_t)v * N + l] = W[idx(v, l, c)];
      positivity_limit_cell(c, cellw.data());
      for (int v = 0; v < nv; ++v)
        for (int l = 0; l < N; ++l) W[idx(v, l, c)] = cellw[(size_t)v * N + l];
    }
  }

  // positivity limiting of the weights w[v][l] of cell c, in place
  void positivity_limit_cell(int c, double* w) const {
    if (!positivity) return;
    const auto pts = positivity_points(c);
    double u[5], ub[5];
    for (int v = 0; v < nv; ++v) ub[v] = w[(size_t)v * N];
    std::vector<double> row(N);
    auto at = [&](const std::array<double, 3>& x) {
      for (int l = 0; l < N; ++l) row[l] = basis.phi(l, x.data());
      for (int v = 0; v < nv; ++v) {
        double s = 0.0;
        for (int l = 0; l < N; ++l) s += w[(size_t)v * N + l] * row[l];
        u[v] = s;
      }
    };
    double rmin = 1e300;
    for (const auto& x : pts) {
      at(x);
      rmin = std::min(rmin, u[0]);
    }
    double th1 = 1.0;
    if (rmin < eps) th1 = std::min(std::fabs((ub[0] - eps) / (ub[0] - rmin)), 1.0);
    if (th1 < 1.0)
      for (int l = 1; l < N; ++l) w[l] *= th1;
    double th2 = 1.0;
    for (const auto& x : pts) {
      at(x);
      if (pressure(dim, gamma, u) >= eps) continue;
      th2 = std::min(th2, solve_tau(ub, u));
    }
    if (th2 < 1.0)
      for (int v = 0; v < nv; ++v)
        for (int l = 1; l < N; ++l) w[(size_t)v * N + l] *= th2;
  }

  // slope then positivity limiting of one cell (inputs from W), -> out[v][l]
  void limit_one(const double* W, int c, double* out) const {
    slope_limit_cell(W, c, out);
    positivity_limit_cell(c, out);
  }

  void limit(double* W) const {
    slope_limit(W);
    positivity_limit(W);
  }

  // dw/dt of every cell in the gather form: rhs_one per cell, the cells
  // shared among `threads` OpenMP threads.  Each cell writes only its own
  // weights, so the loop has no races and its result does not depend on the
  // thread count (the scatter form `rhs` adds each face term to both
  // neighbours and cannot be split over cells; the two forms sum the same
  // terms in a different order, so they agree to rounding).
  void rhs_parallel(const double* W, double* dW) const {
    const int nc = mesh.ncells;
#pragma omp parallel num_threads(threads)
    {
      std::vector<double> out((size_t)nv * N);
#pragma omp for schedule(static)
      for (int c = 0; c < nc; ++c) {
        rhs_one(W, c, out.data());
        for (int v = 0; v < nv; ++v)
          for (int j = 0; j < N; ++j) dW[idx(v, j, c)] = out[(size_t)v * N + j];
      }
    }
  }

  // One time step (Sec. 4.5, steps 5a-5b); dt <= 0 takes the CFL timestep.
  // With threads > 1 the right-hand side is the gather form on that many
  // threads (timing of the oracle on all host cores); otherwise the scatter
  // form `rhs`.
  double rk_step(double* W, double dt) const {
    if (dt <= 0.0) dt = compute_dt(W);
    std::vector<double> w(W, W + size());
    const bool lim = (limiter != LIM_NONE && k > 0) || positivity;
    rk_butcher<double>(
        tb, w, dt,
        [&](const std::vector<double>& U, std::vector<double>& K) {
          if (threads > 1) rhs_parallel(U.data(), K.data());
          else rhs(U.data(), K.data());
        },
        lim ? std::function<void(std::vector<double>&)>([&](std::vector<double>& U) { limit(U.data()); })
            : std::function<void(std::vector<double>&)>());
    std::copy(w.begin(), w.end(), W);
    return dt;
  }

  // Forward-mode derivative of one unlimited step with a frozen dt:
  // JV = (d w_new / d w) V.
  void rk_step_jvp(const double* W, const double* Vd, double dt, double* Wout, double* JV) const {
    std::vector<Dual> w(size());
    for (size_t i = 0; i < w.size(); ++i) w[i] = Dual(W[i], Vd[i]);
    rk_butcher<Dual>(
        tb, w, dt, [&](const std::vector<Dual>& U, std::vector<Dual>& K) { rhs(U.data(), K.data()); },
        std::function<void(std::vector<Dual>&)>());
    for (size_t i = 0; i < w.size(); ++i) {
      Wout[i] = w[i].v;
      JV[i] = w[i].d;
    }
  }

  // L2 projection of point values onto the basis (Sec. 2.3):
  // w_j = 2^-d sum_q u(xi_q) phi_j(xi_q) w_q, u given as [v][q][cell].
  void project(const double* uq, double* W) const {
    const int nc = mesh.ncells;
    for (int c = 0; c < nc; ++c)
      for (int v = 0; v < nv; ++v)
        for (int j = 0; j < N; ++j) {
          double s = 0.0;
          for (int q = 0; q < vol.n; ++q)
            s += uq[((size_t)v * vol.n + q) * nc + c] * phi_vol[(size_t)q * N + j] * vol.w[q];
          W[idx(v, j, c)] = std::ldexp(s, -dim);
        }
  }

  // physical coordinates of the points of a rule in every cell, [a][q][cell]
  void rule_points(const TensorRule& r, double* xyz) const {
    const int nc = mesh.ncells;
    for (int c = 0; c < nc; ++c)
      for (int q = 0; q < r.n; ++q)
        for (int a = 0; a < dim; ++a)
          xyz[((size_t)a * r.n + q) * nc + c] = mesh.center(c, a) + 0.5 * mesh.dx(c) * r.xi[q][a];
  }

  // sum over cells of |K| w_1 (conserved totals)
  void totals(const double* W, double* out) const {
    for (int v = 0; v < nv; ++v) {
      double s = 0.0;
      for (int c = 0; c < mesh.ncells; ++c) s += std::pow(mesh.dx(c), dim) * W[idx(v, 0, c)];
      out[v] = s;
    }
  }

  // L1 density error (eq. L1_norm) with a (k+3)^d Gauss rule per cell;
  // rho_exact given at the rule's points, [q][cell]
  double l1_density(const double* W, const double* rho_exact) const {
    const int nc = mesh.ncells;
    double vol_total = 1.0;
    for (int a = 0; a < dim; ++a) vol_total *= mesh.hi[a] - mesh.lo[a];
    double s = 0.0;
    std::vector<double> row(N);
    for (int c = 0; c < nc; ++c) {
      double cell = 0.0;
      for (int q = 0; q < l1rule.n; ++q) {
        double rho = 0.0;
        for (int l = 0; l < N; ++l) rho += W[idx(0, l, c)] * basis.phi(l, l1rule.xi[q].data());
        cell += std::fabs(rho - rho_exact[(size_t)q * nc + c]) * l1rule.w[q];
      }
      s += std::pow(0.5 * mesh.dx(c), dim) * cell;
    }
    return s / vol_total;
  }

  // ---- mesh adaptation of the two-level mesh (Secs. 4.1, 4.3, 4.4) ----
  // Base cells in lexicographic order; first[b] = first cell of base cell b,
  // node_of[b] = its node index or -1 when b is a leaf.
  void base_maps(std::vector<int>& first, std::vector<int>& node_of) const {
    const int nb = mesh.n[0] * mesh.n[1] * mesh.n[2];
    first.assign(nb + 1, 0);
    node_of.assign(nb, -1);
    std::map<std::array<int, 3>, int> nodes;
    for (int m = 0; m < mesh.nnodes; ++m) nodes[mesh.node_coord[m]] = m;
    for (int b = 0; b < nb; ++b) {
      const std::array<int, 3> p = {b % mesh.n[0], (b / mesh.n[0]) % mesh.n[1], b / (mesh.n[0] * mesh.n[1])};
      auto it = nodes.find(p);
      if (it != nodes.end()) node_of[b] = it->second;
      first[b + 1] = first[b] + (it != nodes.end() ? (1 << dim) : 1);
    }
  }

  // New refinement of every base cell: the criterion of eq. cell_ref on a
  // leaf (the largest density slope weight |w_rho,1+a| above alpha w_t), of
  // eq. node_ref on a node (its node weights' largest slope above w_t /
  // alpha), then one buffer layer: a base cell is refined when it or any base
  // cell around it (sharing a face, edge or corner; periodic axes wrap)
  // meets its criterion.
  std::vector<int> adapt_flags(const double* W, double w_t, double alpha) const {
    std::vector<int> first, node_of;
    base_maps(first, node_of);
    const int nb = (int)node_of.size();
    std::vector<double> Wn((size_t)nv * N * std::max(mesh.nnodes, 1));
    if (mesh.nnodes > 0) node_weights(W, Wn.data());
    std::vector<int> crit(nb, 0);
    for (int b = 0; b < nb; ++b) {
      double slope = 0.0;
      for (int a = 0; a < dim; ++a) {
        const double wa = node_of[b] < 0 ? W[idx(0, 1 + a, first[b])]
                                         : Wn[(size_t)(1 + a) * mesh.nnodes + node_of[b]];
        slope = std::max(slope, std::fabs(wa));
      }
      crit[b] = node_of[b] < 0 ? (slope > alpha * w_t) : (slope > w_t / alpha);
    }
    std::vector<int> flags(nb, 0);
    const int* n = mesh.n;
    for (int b = 0; b < nb; ++b) {
      const int p[3] = {b % n[0], (b / n[0]) % n[1], b / (n[0] * n[1])};
      int any = 0;
      for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int d[3] = {dx, dy, dz};
            int q[3];
            bool inside = true;
            for (int a = 0; a < 3; ++a) {
              q[a] = p[a] + d[a];
              if (q[a] < 0 || q[a] >= n[a]) {
                if (a < dim && mesh.bc[a] == BC_PERIODIC) q[a] = (q[a] + n[a]) % n[a];
                else inside = false;
              }
            }
            if (inside) any |= crit[q[0] + n[0] * (q[1] + n[1] * q[2])];
          }
      flags[b] = any;
    }
    return flags;
  }

  // The state on this mesh from the state Wold on `old` (the same base grid):
  // unchanged cells copied, a refined leaf projected onto its children with
  // the refinement matrices (eq. ref_weights), a derefined node's children
  // merged with the transposed matrices (eq. deref_weights).
  void adapt_project(const Problem& old, const double* Wold, double* W) const {
    std::vector<int> f0, n0, f1, n1;
    old.base_maps(f0, n0);
    base_maps(f1, n1);
    const int nch = 1 << dim;
    for (size_t b = 0; b < n1.size(); ++b)
      for (int v = 0; v < nv; ++v) {
        if ((n0[b] < 0) == (n1[b] < 0)) {  // unchanged: copy every cell of the base cell
          for (int k = 0; k < f1[b + 1] - f1[b]; ++k)
            for (int l = 0; l < N; ++l) W[idx(v, l, f1[b] + k)] = Wold[old.idx(v, l, f0[b] + k)];
        } else if (n1[b] >= 0) {  // refine: w^c = P_c w
          for (int ch = 0; ch < nch; ++ch)
            for (int j = 0; j < N; ++j) {
              double s = 0.0;
              for (int l = 0; l < N; ++l) s += Pref[((size_t)ch * N + j) * N + l] * Wold[old.idx(v, l, f0[b])];
              W[idx(v, j, f1[b] + ch)] = s;
            }
        } else {  // derefine: w = 2^-d sum_c P_c^T w^c
          for (int j = 0; j < N; ++j) {
            double s = 0.0;
            for (int ch = 0; ch < nch; ++ch)
              for (int l = 0; l < N; ++l) s += Pref[((size_t)ch * N + l) * N + j] * Wold[old.idx(v, l, f0[b] + ch)];
            W[idx(v, j, f1[b])] = std::ldexp(s, -dim);
          }
        }
      }
  }

  // node weights w_node = 2^-d sum_c P_c^T w^c (eq. deref_weights)
  void node_weights(const double* W, double* Wn) const {
    const int nn = mesh.nnodes;
    for (int m = 0; m < nn; ++m)
      for (int v = 0; v < nv; ++v)
        for (int j = 0; j < N; ++j) {
          double s = 0.0;
          for (int ch = 0; ch < (1 << dim); ++ch) {
            const int c = mesh.node_children[m][ch];
            for (int l = 0; l < N; ++l) s += Pref[((size_t)ch * N + l) * N + j] * W[idx(v, l, c)];
          }
          Wn[((size_t)v * N + j) * nn + m] = std::ldexp(s, -dim);
        }
  }
};

}  // namespace orc
