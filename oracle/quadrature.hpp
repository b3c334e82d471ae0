// Oracle (test infrastructure only): Legendre polynomials, Gauss-Legendre and
// Gauss-Lobatto-Legendre rules, and the modal basis of the DG scheme.
//
// Plain FP64 code written from the paper (Appendices A, B and C; Sec. 2.2,
// eqs. set_basis_functions and nof_basis_functions).  Only tests/, the
// package smoke check and the CPU-baseline leg of bench.py may use it.
#pragma once
#include <array>
#include <cmath>
#include <vector>

namespace orc {

// P_0..P_n and their derivatives at x (Appendix A).  The polynomials follow
// Bonnet's recursion (m+1) P_{m+1} = (2m+1) x P_m - m P_{m-1}; the
// derivatives use P'_{m+1} = P'_{m-1} + (2m+1) P_m, which also holds at x=+-1.
inline void legendre_all(int n, double x, double* P, double* dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  if (n >= 1) {
    P[1] = x;
    dP[1] = 1.0;
  }
  for (int m = 1; m < n; ++m) {
    P[m + 1] = ((2.0 * m + 1.0) * x * P[m] - m * P[m - 1]) / (m + 1.0);
    dP[m + 1] = dP[m - 1] + (2.0 * m + 1.0) * P[m];
  }
}

inline double legendre(int n, double x) {
  double P[32], dP[32];
  legendre_all(n, x, P, dP);
  return P[n];
}

inline double legendre_deriv(int n, double x) {
  double P[32], dP[32];
  legendre_all(n, x, P, dP);
  return dP[n];
}

// n-point Gauss-Legendre rule on [-1,1] (Appendix B): Newton-Raphson on P_n
// from Lether's initial guess, weights 2 / ((1 - x^2) P_n'(x)^2).
// Nodes are returned in ascending order.
inline void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  std::vector<double> P(n + 2), dP(n + 2);
  for (int q = 1; q <= n; ++q) {
    const double nn = n;
    double xi = (1.0 - 1.0 / (8.0 * nn * nn) + 1.0 / (8.0 * nn * nn * nn)) *
                std::cos(M_PI * (4.0 * q - 1.0) / (4.0 * nn + 2.0));
    for (int it = 0; it < 100; ++it) {
      legendre_all(n, xi, P.data(), dP.data());
      const double step = P[n] / dP[n];
      xi -= step;
      if (std::fabs(step) < 1e-15) break;
    }
    // one more step once the update is at round-off level
    legendre_all(n, xi, P.data(), dP.data());
    xi -= P[n] / dP[n];
    legendre_all(n, xi, P.data(), dP.data());
    // Lether's guess runs from the largest root (q=1) down to the smallest
    x[n - q] = xi;
    w[n - q] = 2.0 / ((1.0 - xi * xi) * dP[n] * dP[n]);
  }
}

// n-point Gauss-Lobatto-Legendre rule (Appendix C): nodes are the roots of
// (1 - x^2) P'_{n-1}(x); interior weights 2 / (n (n-1) P_{n-1}(x)^2); the two
// end weights are equal and all weights sum to 2.  Requires n >= 2.
inline void gauss_lobatto(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const int m = n - 1;  // interior nodes are the roots of P'_m
  std::vector<double> P(m + 2), dP(m + 2);
  x[0] = -1.0;
  x[n - 1] = 1.0;
  for (int q = 1; q <= n - 2; ++q) {
    // start from the Chebyshev-Lobatto point and run Newton on P'_m; the
    // second derivative comes from Legendre's equation (eq. legendre_dgl):
    // (1 - x^2) P'' = 2 x P' - m (m+1) P
    double xi = -std::cos(M_PI * q / (double)m);
    for (int it = 0; it < 100; ++it) {
      legendre_all(m, xi, P.data(), dP.data());
      const double d2 = (2.0 * xi * dP[m] - m * (m + 1.0) * P[m]) / (1.0 - xi * xi);
      const double step = dP[m] / d2;
      xi -= step;
      if (std::fabs(step) < 1e-15) break;
    }
    legendre_all(m, xi, P.data(), dP.data());
    xi -= dP[m] * (1.0 - xi * xi) / (2.0 * xi * dP[m] - m * (m + 1.0) * P[m]);
    x[q] = xi;
  }
  double interior = 0.0;
  for (int q = 1; q <= n - 2; ++q) {
    legendre_all(m, x[q], P.data(), dP.data());
    w[q] = 2.0 / (n * (n - 1.0) * P[m] * P[m]);
    interior += w[q];
  }
  w[0] = w[n - 1] = 0.5 * (2.0 - interior);
}

// Modal basis (eq. set_basis_functions): products of scaled Legendre
// polynomials sqrt(2n+1) P_n with total degree <= k.  Ordering (a layout
// convention; the paper fixes only phi_1 = 1 and phi_2..phi_4 = x, y, z
// slopes): by total degree, then by the x exponent descending, then by the
// y exponent descending.
struct Basis {
  int dim = 0, k = 0, N = 0;
  bool tensor = false;
  std::vector<std::array<int, 3>> e;

  Basis() = default;
  // total degree <= k (the paper's basis, eq. set_basis_functions), or, with
  // tensor set, every exponent <= k (the tensor-product space Q_k).  Either
  // way the order is by total degree, then the x exponent descending, then
  // the y exponent descending, so phi_1 = 1 and phi_2.. phi_(1+dim) are the
  // linear functions x, y (, z).
  Basis(int dim_, int k_, bool tensor_ = false) : dim(dim_), k(k_), tensor(tensor_) {
    const int gmax = tensor ? dim * k : k;
    for (int g = 0; g <= gmax; ++g) {
      if (dim == 2) {
        for (int nx = g; nx >= 0; --nx) {
          const int ny = g - nx;
          if (nx <= k && ny <= k) e.push_back({nx, ny, 0});
        }
      } else {
        for (int nx = g; nx >= 0; --nx)
          for (int ny = g - nx; ny >= 0; --ny) {
            const int nz = g - nx - ny;
            if (nx <= k && ny <= k && nz <= k) e.push_back({nx, ny, nz});
          }
      }
    }
    N = (int)e.size();
  }

  static double scaled(int n, double x) { return std::sqrt(2.0 * n + 1.0) * legendre(n, x); }
  static double scaled_deriv(int n, double x) {
    return std::sqrt(2.0 * n + 1.0) * legendre_deriv(n, x);
  }

  // phi_l(xi)
  double phi(int l, const double* xi) const {
    double v = 1.0;
    for (int a = 0; a < dim; ++a) v *= scaled(e[l][a], xi[a]);
    return v;
  }
  // d phi_l / d xi_a
  double dphi(int l, int a, const double* xi) const {
    double v = 1.0;
    for (int b = 0; b < dim; ++b)
      v *= (b == a) ? scaled_deriv(e[l][b], xi[b]) : scaled(e[l][b], xi[b]);
    return v;
  }
  // degree of phi_l
  int degree(int l) const { return e[l][0] + e[l][1] + e[l][2]; }
};

// Number of basis functions (eq. nof_basis_functions and its 2D analogue).
inline int n_basis(int dim, int k) {
  return dim == 3 ? (k + 1) * (k + 2) * (k + 3) / 6 : (k + 1) * (k + 2) / 2;
}

// Tensor-product rule on [-1,1]^dim from a 1D rule (Appendix B); point index
// runs with the first axis fastest.
struct TensorRule {
  int dim = 0, n1 = 0, n = 0;
  std::vector<std::array<double, 3>> xi;
  std::vector<double> w;
  TensorRule() = default;
  TensorRule(int dim_, const std::vector<double>& x1, const std::vector<double>& w1) : dim(dim_) {
    n1 = (int)x1.size();
    int nz = dim == 3 ? n1 : 1;
    for (int iz = 0; iz < nz; ++iz)
      for (int iy = 0; iy < n1; ++iy)
        for (int ix = 0; ix < n1; ++ix) {
          xi.push_back({x1[ix], x1[iy], dim == 3 ? x1[iz] : 0.0});
          w.push_back(w1[ix] * w1[iy] * (dim == 3 ? w1[iz] : 1.0));
        }
    n = (int)w.size();
  }
};

}  // namespace orc
