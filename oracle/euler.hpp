// Oracle (test infrastructure only): ideal-gas Euler equations, the HLLC
// numerical flux and the characteristic eigenvector matrices.  Templated on
// the scalar so that the same plain formulas run on doubles and on forward-
// mode dual numbers (used to form exact Jacobian-vector products).
//
// Sources: Sec. 2.1 (eqs. euler, state_vector, flux_vectors, eos); the HLLC
// solver named in Sec. 2.4 (Toro's textbook form, written from the
// mathematics); Appendix E (eigenvector matrices).
#pragma once
#include <cmath>

namespace orc {

// ---------------------------------------------------------------------------
// Dual number: value and one directional derivative.
struct Dual {
  double v = 0.0, d = 0.0;
  Dual() = default;
  Dual(double x) : v(x), d(0.0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
  Dual& operator+=(const Dual& o) { v += o.v; d += o.d; return *this; }
  Dual& operator-=(const Dual& o) { v -= o.v; d -= o.d; return *this; }
  Dual& operator*=(const Dual& o) { d = d * o.v + v * o.d; v *= o.v; return *this; }
};
inline Dual operator+(Dual a, const Dual& b) { return a += b; }
inline Dual operator-(Dual a, const Dual& b) { return a -= b; }
inline Dual operator-(const Dual& a) { return Dual(-a.v, -a.d); }
inline Dual operator*(const Dual& a, const Dual& b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(const Dual& a, const Dual& b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual sqrt(const Dual& a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline Dual fabs(const Dual& a) { return a.v >= 0.0 ? a : -a; }
inline bool operator<(const Dual& a, const Dual& b) { return a.v < b.v; }
inline bool operator<=(const Dual& a, const Dual& b) { return a.v <= b.v; }
inline bool operator>(const Dual& a, const Dual& b) { return a.v > b.v; }
inline bool operator>=(const Dual& a, const Dual& b) { return a.v >= b.v; }

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
using std::fabs;
using std::sqrt;
template <class T> inline T tmin(const T& a, const T& b) { return b < a ? b : a; }
template <class T> inline T tmax(const T& a, const T& b) { return a < b ? b : a; }

// ---------------------------------------------------------------------------
// State u = (rho, rho v_1..rho v_dim, rho e) with nv = dim + 2 components.

// pressure from the ideal-gas law p = (gamma-1) rho u_int (eq. eos), with
// rho e = rho u_int + rho v^2 / 2 (eq. state_vector)
template <class T>
inline T pressure(int dim, double gamma, const T* u) {
  T kin = T(0.0);
  for (int a = 0; a < dim; ++a) kin += u[1 + a] * u[1 + a];
  kin = 0.5 * kin / u[0];
  return (gamma - 1.0) * (u[dim + 1] - kin);
}

// flux vector f_a(u) (eq. flux_vectors)
template <class T>
inline void euler_flux(int dim, double gamma, const T* u, int a, T* f) {
  const T rho = u[0];
  const T va = u[1 + a] / rho;
  const T p = pressure(dim, gamma, u);
  f[0] = u[1 + a];
  for (int b = 0; b < dim; ++b) f[1 + b] = u[1 + b] * va;
  f[1 + a] += p;
  f[dim + 1] = (u[dim + 1] + p) * va;
}

// HLLC flux across a face with normal +e_a between the left (minus side)
// state uL and the right (plus side) state uR.  Wave speeds after Davis,
// S_L = min(vL - cL, vR - cR), S_R = max(vL + cL, vR + cR); contact speed
// S*; star states and the four-case selection of the textbook HLLC solver.
// The case S* = 0 takes the left star state.
template <class T>
inline void hllc(int dim, double gamma, const T* uL, const T* uR, int a, T* F) {
  const int nv = dim + 2;
  const T rL = uL[0], rR = uR[0];
  const T vL = uL[1 + a] / rL, vR = uR[1 + a] / rR;
  const T pL = pressure(dim, gamma, uL), pR = pressure(dim, gamma, uR);
  const T cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
  const T SL = tmin(vL - cL, vR - cR);
  const T SR = tmax(vL + cL, vR + cR);
  const T Sstar = (pR - pL + rL * vL * (SL - vL) - rR * vR * (SR - vR)) /
                  (rL * (SL - vL) - rR * (SR - vR));
  T fL[5], fR[5];
  euler_flux(dim, gamma, uL, a, fL);
  euler_flux(dim, gamma, uR, a, fR);
  auto star = [&](const T* u, const T& r, const T& v, const T& p, const T& S, T* us) {
    const T fac = r * (S - v) / (S - Sstar);
    us[0] = fac;
    for (int b = 0; b < dim; ++b) us[1 + b] = fac * (u[1 + b] / r);
    us[1 + a] = fac * Sstar;
    us[dim + 1] = fac * (u[dim + 1] / r + (Sstar - v) * (Sstar + p / (r * (S - v))));
  };
  T us[5];
  if (SL >= T(0.0)) {
    for (int i = 0; i < nv; ++i) F[i] = fL[i];
  } else if (Sstar >= T(0.0)) {
    star(uL, rL, vL, pL, SL, us);
    for (int i = 0; i < nv; ++i) F[i] = fL[i] + SL * (us[i] - uL[i]);
  } else if (SR > T(0.0)) {
    star(uR, rR, vR, pR, SR, us);
    for (int i = 0; i < nv; ++i) F[i] = fR[i] + SR * (us[i] - uR[i]);
  } else {
    for (int i = 0; i < nv; ++i) F[i] = fR[i];
  }
}

// ---------------------------------------------------------------------------
// Appendix E: right (columns = eigenvectors) and left eigenvector matrices of
// the flux Jacobian in direction a, evaluated at the state u.  3D matrices as
// printed, with k = (v1^2 + v2^2 + v3^2)/2 and the y and z back-transforms
// taken as R_y and R_z.  In 2D the z velocity and the second shear wave are
// absent: the 4x4 matrices keep rows/columns (rho, m1, m2, E) and the first
// four waves.  Matrices are row-major nv x nv.
inline void eigen_matrices(int dim, double gamma, const double* u, int a, double* L, double* R) {
  const double rho = u[0];
  double v[3] = {0, 0, 0};
  for (int b = 0; b < dim; ++b) v[b] = u[1 + b] / rho;
  const double p = pressure(dim, gamma, u);
  const double c = std::sqrt(gamma * p / rho);
  const double kin = 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const double g1 = gamma - 1.0;
  const double h = c * c / g1 + kin;
  const double phi = g1 * kin;
  const double be = 1.0 / (2.0 * c * c);
  double R5[5][5], L5[5][5];
  const double v1 = v[0], v2 = v[1], v3 = v[2];
  if (a == 0) {
    const double Rx[5][5] = {{1, 1, 1, 0, 0},
                             {v1 - c, v1, v1 + c, 0, 0},
                             {v2, v2, v2, -1, 0},
                             {v3, v3, v3, 0, 1},
                             {h - c * v1, kin, h + c * v1, -v2, v3}};
    const double Lx[5][5] = {
        {be * (phi + c * v1), -be * (g1 * v1 + c), -be * g1 * v2, -be * g1 * v3, be * g1},
        {1 - 2 * be * phi, 2 * be * g1 * v1, 2 * be * g1 * v2, 2 * be * g1 * v3, -2 * be * g1},
        {be * (phi - c * v1), -be * (g1 * v1 - c), -be * g1 * v2, -be * g1 * v3, be * g1},
        {v2, 0, -1, 0, 0},
        {-v3, 0, 0, 1, 0}};
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) { R5[i][j] = Rx[i][j]; L5[i][j] = Lx[i][j]; }
  } else if (a == 1) {
    const double Ry[5][5] = {{1, 1, 1, 0, 0},
                             {v1, v1, v1, 1, 0},
                             {v2 - c, v2, v2 + c, 0, 0},
                             {v3, v3, v3, 0, -1},
                             {h - c * v2, kin, h + c * v2, v1, -v3}};
    const double Ly[5][5] = {
        {be * (phi + c * v2), -be * g1 * v1, -be * (g1 * v2 + c), -be * g1 * v3, be * g1},
        {1 - 2 * be * phi, 2 * be * g1 * v1, 2 * be * g1 * v2, 2 * be * g1 * v3, -2 * be * g1},
        {be * (phi - c * v2), -be * g1 * v1, -be * (g1 * v2 - c), -be * g1 * v3, be * g1},
        {-v1, 1, 0, 0, 0},
        {v3, 0, 0, -1, 0}};
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) { R5[i][j] = Ry[i][j]; L5[i][j] = Ly[i][j]; }
  } else {
    const double Rz[5][5] = {{1, 1, 1, 0, 0},
                             {v1, v1, v1, -1, 0},
                             {v2, v2, v2, 0, 1},
                             {v3 - c, v3, v3 + c, 0, 0},
                             {h - c * v3, kin, h + c * v3, -v1, v2}};
    const double Lz[5][5] = {
        {be * (phi + c * v3), -be * g1 * v1, -be * g1 * v2, -be * (g1 * v3 + c), be * g1},
        {1 - 2 * be * phi, 2 * be * g1 * v1, 2 * be * g1 * v2, 2 * be * g1 * v3, -2 * be * g1},
        {be * (phi - c * v3), -be * g1 * v1, -be * g1 * v2, -be * (g1 * v3 - c), be * g1},
        {v1, -1, 0, 0, 0},
        {-v2, 0, 1, 0, 0}};
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) { R5[i][j] = Rz[i][j]; L5[i][j] = Lz[i][j]; }
  }
  if (dim == 3) {
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) { R[i * 5 + j] = R5[i][j]; L[i * 5 + j] = L5[i][j]; }
  } else {
    const int var[4] = {0, 1, 2, 4};  // (rho, m1, m2, E) inside the 3D state
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        R[i * 4 + j] = R5[var[i]][j];  // rows: variables, columns: waves 0..3
        L[i * 4 + j] = L5[i][var[j]];  // rows: waves 0..3, columns: variables
      }
  }
}

}  // namespace orc
