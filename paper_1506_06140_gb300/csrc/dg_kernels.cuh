// sm_103a kernels of the DG right-hand side and RK stage (paper Sec. 2.4,
// eqs. dg_term2 / dg_term3 / spatial_discretisation; Appendix D), the slope
// and positivity limiters (Secs. 3.2-3.4, 4.4), the timestep (Sec. 2.5), and
// the projection / reduction helpers.  Templated on the arithmetic type and
// on (DIM, K) so that every loop over basis functions and quadrature points
// is unrolled at compile time.
//
// Layout: state W[var][coef][cell] (cell fastest, so a warp reading 32
// consecutive cells of one coefficient row issues one coalesced request);
// face fluxes F[var][face point][face]; all tables in a per-handle buffer
// (see Shape<> for offsets).
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "dg_convert.cuh"
#include "dg_internal.h"
#include "dg_physics.cuh"
#include "dg_stage.cuh"
#include "dg_adjoint.cuh"
#include "dg_direct.cuh"
#include "dg_tc.cuh"

namespace dgi {

// ===========================================================================
// Host: tables (basis values at the quadrature points, Appendices A-C)

inline void host_legendre(int n, double x, double* P, double* dP) {
  // P_{m+1} = ((2m+1) x P_m - m P_{m-1}) / (m+1);  P'_{m+1} = (m+1) P_m + x P'_m
  P[0] = 1.0;
  dP[0] = 0.0;
  for (int m = 0; m < n; ++m) {
    P[m + 1] = (m == 0) ? x : ((2.0 * m + 1.0) * x * P[m] - m * P[m - 1]) / (m + 1.0);
    dP[m + 1] = (m + 1.0) * P[m] + x * dP[m];
  }
}

template <int DIM, int K, int B = 0>
struct HostBasis {
  using S = Shape<DIM, K, B>;
  int e[S::N][3];
  // by total degree, then the x exponent descending, then y descending;
  // every exponent <= K for the tensor-product basis (B = 1)
  HostBasis() {
    int n = 0;
    for (int g = 0; g <= (B ? DIM * K : K); ++g) {
      if (DIM == 2) {
        for (int nx = g; nx >= 0; --nx) {
          if (nx > K || g - nx > K) continue;
          e[n][0] = nx; e[n][1] = g - nx; e[n][2] = 0; ++n;
        }
      } else {
        for (int nx = g; nx >= 0; --nx)
          for (int ny = g - nx; ny >= 0; --ny) {
            if (nx > K || ny > K || g - nx - ny > K) continue;
            e[n][0] = nx; e[n][1] = ny; e[n][2] = g - nx - ny; ++n;
          }
      }
    }
  }
  // scaled Legendre sqrt(2n+1) P_n and its derivative
  static void sl(int n, double x, double& v, double& d) {
    double P[16], dP[16];
    host_legendre(n, x, P, dP);
    const double s = std::sqrt(2.0 * n + 1.0);
    v = s * P[n];
    d = s * dP[n];
  }
  double phi(int l, const double* xi) const {
    double r = 1.0;
    for (int a = 0; a < DIM; ++a) {
      double v, d;
      sl(e[l][a], xi[a], v, d);
      r *= v;
    }
    return r;
  }
  double dphi(int l, int a, const double* xi) const {
    double r = 1.0;
    for (int b = 0; b < DIM; ++b) {
      double v, d;
      sl(e[l][b], xi[b], v, d);
      r *= (b == a) ? d : v;
    }
    return r;
  }
  int degree(int l) const { return e[l][0] + e[l][1] + e[l][2]; }
};

// point q of face (dir, s) in the cell frame; variant 0 = whole face,
// 1 + quad = the sub-face 'quad' (bit i = upper half along tangential axis i)
template <int DIM, int K>
inline void face_point(int dir, int s, int variant, int q, const std::vector<double>& gx,
                       double* xi, double* w, const std::vector<double>& gw) {
  xi[0] = xi[1] = xi[2] = 0.0;
  xi[dir] = s ? 1.0 : -1.0;
  *w = 1.0;
  int t = 0, qq = q;
  for (int b = 0; b < DIM; ++b) {
    if (b == dir) continue;
    const int i = qq % (K + 1);
    qq /= (K + 1);
    double eta = gx[i];
    if (variant > 0) eta = 0.5 * (eta + (((variant - 1) >> t) & 1 ? 1.0 : -1.0));
    xi[b] = eta;
    *w *= gw[i];
    ++t;
  }
}

template <int DIM, int K, int BA = 0>
void fill_tables(std::vector<double>& T, const std::vector<double>& gx,
                 const std::vector<double>& gw, const std::vector<double>& g3x,
                 const std::vector<double>& g3w, const std::vector<double>& lx) {
  using S = Shape<DIM, K, BA>;
  HostBasis<DIM, K, BA> B;
  T.assign(S::TAB_SIZE, 0.0);
  const double two_d = std::ldexp(1.0, DIM);
  // volume rule, x fastest
  for (int q = 0; q < S::Q; ++q) {
    double xi[3] = {0, 0, 0}, w = 1.0;
    int qq = q;
    for (int a = 0; a < DIM; ++a) {
      xi[a] = gx[qq % S::K1];
      w *= gw[qq % S::K1];
      qq /= S::K1;
    }
    for (int a = 0; a < 3; ++a) T[S::OFF_XI + q * 3 + a] = xi[a];
    for (int l = 0; l < S::N; ++l) {
      T[S::OFF_PHI + q * S::N + l] = B.phi(l, xi);
      T[S::OFF_PROJ + q * S::N + l] = B.phi(l, xi) * w / two_d;
      for (int a = 0; a < DIM; ++a) T[S::OFF_DPHIW + (a * S::Q + q) * S::N + l] = B.dphi(l, a, xi) * w;
    }
  }
  // faces
  const double sub_w = std::ldexp(1.0, -(DIM - 1));
  for (int side = 0; side < S::NSIDE; ++side)
    for (int var = 0; var < S::NVAR; ++var)
      for (int q = 0; q < S::QF; ++q) {
        double xi[3], w;
        face_point<DIM, K>(side >> 1, side & 1, var, q, gx, xi, &w, gw);
        for (int l = 0; l < S::N; ++l) {
          const int idx = ((side * S::NVAR + var) * S::QF + q) * S::N + l;
          T[S::OFF_PHIF + idx] = B.phi(l, xi);
          T[S::OFF_PHIFW + idx] = B.phi(l, xi) * w * (var > 0 ? sub_w : 1.0);
        }
      }
  // refinement matrices (P_c)_{j,l} = 2^-d int phi_j(eta) phi_l((eta + o_c)/2) d eta
  for (int ch = 0; ch < S::NCH; ++ch)
    for (int q = 0; q < S::Q; ++q) {
      const double* eta = &T[S::OFF_XI + q * 3];
      double w = 1.0;
      int qq = q;
      for (int a = 0; a < DIM; ++a) { w *= gw[qq % S::K1]; qq /= S::K1; }
      double xc[3] = {0, 0, 0};
      for (int a = 0; a < DIM; ++a) xc[a] = 0.5 * (eta[a] + (((ch >> a) & 1) ? 1.0 : -1.0));
      for (int j = 0; j < S::N; ++j)
        for (int l = 0; l < S::N; ++l)
          T[S::OFF_PREF + (ch * S::N + j) * S::N + l] += B.phi(j, eta) * B.phi(l, xc) * w / two_d;
    }
  // positivity set S: Lobatto along axis a, Gauss along the others
  for (int a = 0; a < DIM; ++a)
    for (int r = 0; r < S::M; ++r)
      for (int tq = 0; tq < S::QF; ++tq) {
        double xi[3] = {0, 0, 0};
        xi[a] = lx[r];
        int qq = tq;
        for (int b = 0; b < DIM; ++b) {
          if (b == a) continue;
          xi[b] = gx[qq % S::K1];
          qq /= S::K1;
        }
        const int i = (a * S::M + r) * S::QF + tq;
        for (int l = 0; l < S::N; ++l) T[S::OFF_SPHI + i * S::N + l] = B.phi(l, xi);
      }
  // (k+3)^d rule for the L1 error
  for (int q = 0; q < S::Q1; ++q) {
    double xi[3] = {0, 0, 0}, w = 1.0;
    int qq = q;
    for (int a = 0; a < DIM; ++a) {
      xi[a] = g3x[qq % S::K3];
      w *= g3w[qq % S::K3];
      qq /= S::K3;
    }
    for (int a = 0; a < 3; ++a) T[S::OFF_XI1 + q * 3 + a] = xi[a];
    T[S::OFF_L1W + q] = w;
    for (int l = 0; l < S::N; ++l) T[S::OFF_L1PHI + q * S::N + l] = B.phi(l, xi);
  }
  for (int l = 0; l < S::N; ++l) T[S::OFF_DEG + l] = B.degree(l);
  for (int l = 0; l < S::N; ++l) {
    double m = 1.0;
    for (int a = 0; a < DIM; ++a) m *= std::sqrt(2.0 * B.e[l][a] + 1.0);
    T[S::OFF_PMAX + l] = m;  // max of |phi_l| over [-1,1]^d (attained at a corner)
  }
  // 1D tables (layout of Tab1D<double>)
  Tab1D<double> t1{};
  for (int a = 0; a <= K; ++a)
    for (int i = 0; i <= K; ++i) {
      double v, d;
      HostBasis<DIM, K>::sl(a, gx[i], v, d);
      t1.P[a][i] = v;
      t1.PW[a][i] = v * gw[i];
      t1.DW[a][i] = d * gw[i];
      for (int h = 0; h < 2; ++h) {
        double vh, dh;
        HostBasis<DIM, K>::sl(a, 0.5 * (gx[i] + (h ? 1.0 : -1.0)), vh, dh);
        t1.PH[h][a][i] = vh;
        t1.PWH[h][a][i] = vh * gw[i];
      }
    }
  for (int a = 0; a <= K; ++a)
    for (int s = 0; s < 2; ++s) {
      double v, d;
      HostBasis<DIM, K>::sl(a, s ? 1.0 : -1.0, v, d);
      t1.PE[s][a] = v;
    }
  for (int i = 0; i <= K; ++i) t1.W[i] = gw[i];
  // half-interval maps: (1/2) sum_i P~_a(half node i) P~_b(x_i) w_i, exact for
  // a + b <= 2k (the (k+1)-point rule), zero above the diagonal
  for (int h = 0; h < 2; ++h)
    for (int a = 0; a <= K; ++a)
      for (int b = 0; b <= a; ++b) {
        double s = 0.0;
        for (int i = 0; i <= K; ++i) s += t1.PH[h][a][i] * t1.P[b][i] * gw[i];
        t1.TH[h][a][b] = 0.5 * s;
      }
  static_assert(sizeof(Tab1D<double>) == 156 * sizeof(double), "Tab1D layout");
  std::memcpy(&T[S::OFF_1D], &t1, sizeof(t1));
}

// ===========================================================================
// Device helpers

template <typename real>
__device__ __forceinline__ real ld(const real* p) { return __ldg(p); }

__device__ __forceinline__ double cell_dx(const MeshDev& m, int c) {
  const double base = m.dx_prob ? m.dx_prob[m.prob[c]] : m.dx0;
  return ldexp(base, -(int)m.level[c]);
}

// ===========================================================================
// Limiters (Secs. 3.2-3.4 and 4.4), one thread per cell, FP64 arithmetic.
// Inputs come from Uin (state before limiting), the result goes to Uout.

template <typename real, int DIM, int K>
__device__ __forceinline__ void nb_mean(const LimitArgs<real>& a, int c, int dir, int s, int nb,
                                        const real* own, real* out) {
  using S = Shape<DIM, K>;
  const int nc = a.m.ncells;
  if (nb == -1) {
    for (int v = 0; v < S::NV; ++v) out[v] = own[v];
  } else if (nb <= -2) {
    const int* kids = a.m.node_children + (size_t)(-(nb + 2)) * S::NCH;
    for (int v = 0; v < S::NV; ++v) {
      real sum = real(0);
      for (int ch = 0; ch < S::NCH; ++ch) sum += a.Uin[(size_t)(v * S::N) * nc + kids[ch]];
      out[v] = sum / real(S::NCH);
    }
  } else if (a.m.level[nb] == a.m.level[c]) {
    for (int v = 0; v < S::NV; ++v) out[v] = a.Uin[(size_t)(v * S::N) * nc + nb];
  } else {
    // coarser neighbour: mean of its polynomial over the same-size region
    int ch = 0;
    for (int b = 0; b < DIM; ++b) {
      int pb = a.m.coord[(size_t)b * nc + c];
      if (b == dir) {
        const int ext = a.m.n[b] << a.m.level[c];
        pb = (pb + (s ? 1 : -1) + ext) % ext;
      }
      ch |= (pb & 1) << b;
    }
    const double* row = a.tab64 + S::OFF_PREF + (size_t)(ch * S::N + 0) * S::N;
    for (int v = 0; v < S::NV; ++v) {
      real sum = real(0);
      for (int l = 0; l < S::N; ++l) sum += real(row[l]) * a.Uin[(size_t)(v * S::N + l) * nc + nb];
      out[v] = sum;
    }
  }
}

template <typename T>
__device__ __forceinline__ T minmod3(T a, T b, T c) {
  if (a > T(0) && b > T(0) && c > T(0)) return rmin(a, rmin(b, c));
  if (a < T(0) && b < T(0) && c < T(0)) return rmax(a, rmax(b, c));
  return T(0);
}

// Root tau in [0,1] of p(ubar + tau (u - ubar)) = eps: multiplying by the
// density gives the quadratic qa tau^2 + qb tau + qc = 0; stable closed-form
// root, then two Newton-Raphson steps (Sec. 3.4).
template <int DIM>
__device__ double positivity_tau(const double* ub, const double* u, double gamma, double eps) {
  const double g1 = gamma - 1.0;
  double dr = u[0] - ub[0], dE = u[DIM + 1] - ub[DIM + 1];
  double mm = 0.0, md = 0.0, dd = 0.0;
  for (int b = 0; b < DIM; ++b) {
    const double dm = u[1 + b] - ub[1 + b];
    mm += ub[1 + b] * ub[1 + b];
    md += ub[1 + b] * dm;
    dd += dm * dm;
  }
  const double qa = g1 * (dE * dr - 0.5 * dd);
  const double qb = g1 * (ub[DIM + 1] * dr + ub[0] * dE - md) - eps * dr;
  const double qc = g1 * (ub[DIM + 1] * ub[0] - 0.5 * mm) - eps * ub[0];
  if (qc <= 0.0) return 0.0;
  double tau;
  if (fabs(qa) <= 1e-14 * (fabs(qb) + fabs(qc))) {
    tau = -qc / qb;
  } else {
    const double disc = fmax(qb * qb - 4.0 * qa * qc, 0.0);
    const double qq = -0.5 * (qb + copysign(sqrt(disc), qb));
    const double r1 = qq / qa, r2 = qc / qq;
    const bool ok1 = r1 >= 0.0 && r1 <= 1.0, ok2 = r2 >= 0.0 && r2 <= 1.0;
    if (ok1 && ok2) tau = fmin(r1, r2);
    else if (ok1) tau = r1;
    else if (ok2) tau = r2;
    else tau = fabs(r1 - 0.5) < fabs(r2 - 0.5) ? r1 : r2;
  }
  for (int it = 0; it < 2; ++it) {
    const double g = (qa * tau + qb) * tau + qc;
    const double dg = 2.0 * qa * tau + qb;
    if (dg != 0.0) tau -= g / dg;
  }
  return fmin(fmax(tau, 0.0), 1.0);
}

// slope-limiter parameters: 1 component-wise, 2 characteristic (Secs. 3.2-3.3)
struct LimParams {
  int limiter;
  double beta, Mtilde;
};

// characteristic (or component-wise) slopes of direction A, limited, in the
// precision `real`: ct = minmodB(sqrt(3) L w_(1+A), beta L (ubar - u_minus),
// beta L (u_plus - ubar)) / sqrt(3)
template <typename real, int DIM, int K, int A>
__device__ __forceinline__ bool limit_direction(const LimParams& a, const CharState<real, DIM>& st,
                                                const real (&w)[DIM + 2][Shape<DIM, K>::N],
                                                const real* mean, const real* mm, const real* mp, real dx,
                                                real* ct) {
  constexpr int NV = DIM + 2;
  real x[NV], cs[NV], dm[NV], dp[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) x[v] = w[v][1 + A];
  if (a.limiter == 2) {
    char_L<real, DIM, A>(st, x, cs);
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = mean[v] - mm[v];
    char_L<real, DIM, A>(st, x, dm);
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = mp[v] - mean[v];
    char_L<real, DIM, A>(st, x, dp);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      cs[v] = x[v];
      dm[v] = mean[v] - mm[v];
      dp[v] = mp[v] - mean[v];
    }
  }
  const real s3 = real(1.7320508075688772);  // sqrt(3)
  const real beta = real(a.beta), mdx = real(a.Mtilde) * dx;
  bool changed = false;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const real arg = s3 * cs[i];
    const real lim = (fabs(arg) <= mdx) ? arg : minmod3<real>(arg, beta * dm[i], beta * dp[i]);
    changed = changed || (lim != arg);
    ct[i] = lim / s3;
  }
  return changed;
}

template <typename real, int DIM, int K, int A>
__device__ __forceinline__ void unlimit_direction(const LimParams& a, const CharState<real, DIM>& st,
                                                  const real* ct, real (&w)[DIM + 2][Shape<DIM, K>::N]) {
  constexpr int NV = DIM + 2;
  real x[NV];
  if (a.limiter == 2) {
    char_R<real, DIM, A>(st, ct, x);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = ct[v];
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) w[v][1 + A] = x[v];
}

// Positivity test of one cell at the point set of the positivity limiter
// (the set S of eq. union_quad_points, plus the fine sub-face points of every
// side with a finer neighbour), in FP32.  A point value is a sum of N <= 20
// products of FP32-rounded weights and table entries: its error is at most
// (N + 3) 2^-24 < 2e-6 times the sum A of the absolute products, so
// rho >= u_0 - 2e-6 A_0 and likewise for |m_a| and E; the kinetic term
// |m|_up^2 / (2 rho_lo) is rounded by at most 6 ulp (factor 1 + 1e-6) and the
// pressure difference by 3 ulp of |E_lo| + kin (margin 1e-6).  True when
// density and pressure clear rho_min and p_min at every point.  The margins are tight
// enough for cold flows (p / E ~ 1e-5, Keplerian disc).
template <int DIM, int K>
__device__ bool points_clear_fp32(const MeshDev& m, const float* tab32, float rho_min, float p_min, double gamma,
                                  const float (&wf)[Shape<DIM, K>::NV][Shape<DIM, K>::N], int c) {
  using S = Shape<DIM, K>;
  constexpr int NV = S::NV, N = S::N;
  static_assert(N <= 20, "the rounding margins assume at most 20 basis functions");
  const int nc = m.ncells;
  unsigned finer = 0;
  if (m.nnodes > 0)
    for (int sd = 0; sd < S::NSIDE; ++sd)
      if (m.nbr[(size_t)sd * nc + c] <= -2) finer |= 1u << sd;
  const float g1 = (float)(gamma - 1.0);
  const int npts = S::NSP + __popc(finer) * S::NSUB * S::QF;
  for (int ip = 0; ip < npts; ++ip) {
    const float* ph;
    if (ip < S::NSP) {
      ph = tab32 + S::OFF_SPHI + (size_t)ip * N;
    } else {
      int r = ip - S::NSP, sd = 0;
      for (; sd < S::NSIDE; ++sd) {
        if (!((finer >> sd) & 1)) continue;
        if (r < S::NSUB * S::QF) break;
        r -= S::NSUB * S::QF;
      }
      ph = tab32 + S::OFF_PHIF + (size_t)((sd * S::NVAR + 1 + r / S::QF) * S::QF + r % S::QF) * N;
    }
    float u[NV], A[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float s = 0.0f, t = 0.0f;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        const float x = wf[v][l] * ph[l];
        s += x;
        t += fabsf(x);
      }
      u[v] = s;
      A[v] = t;
    }
    const float rho_lo = u[0] - 2e-6f * A[0];
    if (!(rho_lo >= rho_min)) return false;
    float m2 = 0.0f;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      const float mu = fabsf(u[1 + b]) + 2e-6f * A[1 + b];
      m2 += mu * mu;
    }
    const float e_lo = u[DIM + 1] - 2e-6f * A[DIM + 1];
    const float kin = 0.5f * m2 / rho_lo * (1.0f + 1e-6f);
    const float p_lo = g1 * (e_lo - kin);
    if (!(p_lo >= p_min + 1e-6f * g1 * (fabsf(e_lo) + kin))) return false;
  }
  return true;
}

// One thread per cell.  The slope limiter runs in the state's precision (in
// FP32 for an FP64 state when fp32_slopes is set: a cell it leaves alone
// keeps its FP64 weights bit for bit); the positivity limiter's final
// decisions in FP64 behind exact FP32 prechecks.
template <typename real, int DIM, int K>
__device__ __forceinline__ void limit_body(const LimitArgs<real>& a, int bid) {
  using S = Shape<DIM, K>;
  constexpr int NV = S::NV, N = S::N;
  const int c = bid * blockDim.x + threadIdx.x;
  const int nc = a.m.ncells;
  if (c >= nc) return;
  real w[NV][N];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int l = 0; l < N; ++l) w[v][l] = a.Uin[(size_t)(v * N + l) * nc + c];
  real mean[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) mean[v] = w[v][0];
  {
    // mean pressure > 0 <=> rho (E - |m|^2 / (2 rho)) > 0 for rho > 0 (no division)
    real m2 = real(0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) m2 += mean[1 + b] * mean[1 + b];
    const real rp = mean[DIM + 1] * mean[0] - real(0.5) * m2;
    if (!(mean[0] > real(0)) || !(rp > real(0))) atomicOr(a.status, 1 << DG_ERR_NONPHYSICAL_BIT);
  }
  if constexpr (K > 0) {
    if (a.limiter != 0) {
      const LimParams lp{a.limiter, a.beta, a.Mtilde};
      // neighbour means of all sides first: the index loads, then the mean
      // loads, each batch independent
      int nbs[2 * DIM];
#pragma unroll
      for (int sd = 0; sd < 2 * DIM; ++sd) nbs[sd] = a.m.nbr[(size_t)sd * nc + c];
      real nbm[2 * DIM][NV];
#pragma unroll
      for (int sd = 0; sd < 2 * DIM; ++sd) nb_mean<real, DIM, K>(a, c, sd >> 1, sd & 1, nbs[sd], mean, nbm[sd]);
      bool done = false;
      if constexpr (sizeof(real) == 8) {
        if (a.fp32_slopes) {
          // the same limiter on the FP32-rounded weights and means
          float wf[NV][N], mf[NV], nf[2 * DIM][NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            mf[v] = f32_round(mean[v]);
#pragma unroll
            for (int l = 0; l < N; ++l) wf[v][l] = f32_round(w[v][l]);
#pragma unroll
            for (int sd = 0; sd < 2 * DIM; ++sd) nf[sd][v] = f32_round(nbm[sd][v]);
          }
          const float dxf = (float)cell_dx(a.m, c);
          const CharState<float, DIM> st =
              a.limiter == 2 ? char_state<float, DIM>(mf, (float)a.gamma) : CharState<float, DIM>{};
          float ct[DIM][NV];
          bool changed = limit_direction<float, DIM, K, 0>(lp, st, wf, mf, nf[0], nf[1], dxf, ct[0]);
          changed = limit_direction<float, DIM, K, 1>(lp, st, wf, mf, nf[2], nf[3], dxf, ct[1]) || changed;
          if constexpr (DIM == 3)
            changed = limit_direction<float, DIM, K, DIM - 1>(lp, st, wf, mf, nf[4], nf[5], dxf, ct[DIM - 1]) || changed;
          if (changed) {
            if (a.counts) atomicAdd(a.counts, 1ull);
            unlimit_direction<float, DIM, K, 0>(lp, st, ct[0], wf);
            unlimit_direction<float, DIM, K, 1>(lp, st, ct[1], wf);
            if constexpr (DIM == 3) unlimit_direction<float, DIM, K, DIM - 1>(lp, st, ct[DIM - 1], wf);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
#pragma unroll
              for (int b = 0; b < DIM; ++b) w[v][1 + b] = f64_exact(wf[v][1 + b]);
#pragma unroll
              for (int l = DIM + 1; l < N; ++l) w[v][l] = real(0);
            }
          }
          done = true;
        }
      }
      if (!done) {
        const real dx = (real)cell_dx(a.m, c);
        const CharState<real, DIM> st =
            a.limiter == 2 ? char_state<real, DIM>(mean, real(a.gamma)) : CharState<real, DIM>{};
        real ct[DIM][NV];
        bool changed = limit_direction<real, DIM, K, 0>(lp, st, w, mean, nbm[0], nbm[1], dx, ct[0]);
        changed = limit_direction<real, DIM, K, 1>(lp, st, w, mean, nbm[2], nbm[3], dx, ct[1]) || changed;
        if constexpr (DIM == 3)
          changed = limit_direction<real, DIM, K, DIM - 1>(lp, st, w, mean, nbm[4], nbm[5], dx, ct[DIM - 1]) || changed;
        if (changed) {
          if (a.counts) atomicAdd(a.counts, 1ull);
          unlimit_direction<real, DIM, K, 0>(lp, st, ct[0], w);
          unlimit_direction<real, DIM, K, 1>(lp, st, ct[1], w);
          if constexpr (DIM == 3) unlimit_direction<real, DIM, K, DIM - 1>(lp, st, ct[DIM - 1], w);
          // the degree of phi_l is >= 2 exactly for l > DIM (total-degree order)
#pragma unroll
          for (int l = DIM + 1; l < N; ++l)
#pragma unroll
            for (int v = 0; v < NV; ++v) w[v][l] = real(0);
        }
      }
    }
  }
  bool need_positivity = a.positivity && K > 0 && a.tab32;
  if (need_positivity) {
    // Exact shortcuts in FP32 (for either state precision), so that only
    // cells that may need theta < 1 reach the FP64 pass:
    // 1. |phi_l| <= prod sqrt(2e+1) on [-1,1]^d gives rho(x) >= rho_bar -
    //    sum_{l>=1} |w_rho,l| phi_max_l and p(x) >= (gamma-1) (E_low -
    //    |m|_up^2 / (2 rho_low)) over the whole cell; margins 1e-5 cover the
    //    FP32 rounding of these sums of <= 20 terms (< 2e-6);
    // 2. failing that, the values at the limiter's own points.
    float wf[NV][N];
    bool in_range = true;  // FP64 weights below 2^100 in magnitude (else: the FP64 pass decides)
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int l = 0; l < N; ++l) {
        if constexpr (sizeof(real) == 8) {
          wf[v][l] = f32_round(w[v][l]);
          const unsigned e = ((unsigned)(__double_as_longlong(w[v][l]) >> 52)) & 0x7FFu;
          in_range = in_range && e < 1023u + 100u;
        } else {
          wf[v][l] = (float)w[v][l];
        }
      }
    if (in_range) {
      float lo[NV], up[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float r = 0.0f;
#pragma unroll
        for (int l = 1; l < N; ++l) r += fabsf(wf[v][l]) * a.tab32[S::OFF_PMAX + l];
        r *= 1.0f + 1e-5f;
        lo[v] = wf[v][0] - r - 1e-6f * fabsf(wf[v][0]);
        up[v] = (fabsf(wf[v][0]) + r) * (1.0f + 1e-5f);
      }
      // thresholds: twice the positivity pass's floors (eps; for an FP32 state
      // also the rounding scale 2^-20 of the absolute weight sums, see
      // positivity_kernel), so a cell that clears them is left alone there
      float rho_min = 2.0f * (float)a.eps, p_min = rho_min;
      if constexpr (sizeof(real) == 4) {
        float ar = fabsf(wf[0][0]), ae = fabsf(wf[NV - 1][0]);
#pragma unroll
        for (int l = 1; l < N; ++l) {
          ar += fabsf(wf[0][l]) * a.tab32[S::OFF_PMAX + l];
          ae += fabsf(wf[NV - 1][l]) * a.tab32[S::OFF_PMAX + l];
        }
        rho_min = fmaxf(rho_min, 2.0f * 0x1p-20f * 1.01f * ar);
        p_min = fmaxf(p_min, 2.0f * (float)(a.gamma - 1.0) * 0x1p-20f * 1.01f * ae);
      }
      if (lo[0] >= rho_min) {
        float m2 = 0.0f;
#pragma unroll
        for (int b = 0; b < DIM; ++b) m2 += up[1 + b] * up[1 + b];
        const float kin = 0.5f * m2 / lo[0];
        const float p_low = (float)(a.gamma - 1.0) * (lo[DIM + 1] - kin);
        if (p_low >= p_min + 1e-5f * (fabsf(lo[DIM + 1]) + kin)) need_positivity = false;
      }
      if (need_positivity && points_clear_fp32<DIM, K>(a.m, a.tab32, rho_min, p_min, a.gamma, wf, c))
        need_positivity = false;
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int l = 0; l < N; ++l) a.Uout[(size_t)(v * N + l) * nc + c] = w[v][l];
  // cells whose bound does not clear eps get the point search in a second pass
  if (need_positivity) a.queue[atomicAdd(a.queue_len, 1)] = c;
}

template <typename real, int DIM, int K>
__global__ void __launch_bounds__(128, sizeof(real) == 4 && DIM == 3 ? 4 : 1) limit_kernel(const LimitArgs<real> a) {
  pdl_wait();
  limit_body<real, DIM, K>(a, blockIdx.x);
}

// Positivity limiter of Sec. 3.4 (with the hanging-face points of Sec. 4.4)
// for the queued cells, in FP64: theta_1 on the density, then theta_2 from
// the pressure root tau of every point below eps.  One warp per queued cell,
// its lanes over the points; theta_1 and theta_2 are minima over the points,
// so the result does not depend on how the points are shared out.  Reads and
// writes Uout.
__device__ __forceinline__ double warp_min(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// blocks bid of nblk striding over the queue
template <typename real, int DIM, int K>
__device__ __forceinline__ void positivity_body(const LimitArgs<real>& a, int bid, int nblk) {
  using S = Shape<DIM, K>;
  constexpr int NV = S::NV, N = S::N;
  const int nc = a.m.ncells;
  const double* tab = a.tab64;
  const int len = *a.queue_len;
  if (a.counts && bid == 0 && threadIdx.x == 0) atomicAdd(a.counts + 2, (unsigned long long)len);
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  // warp-uniform loop: every lane of a warp takes the same cells
  for (int i = bid * wpb + (threadIdx.x >> 5); i < len; i += nblk * wpb) {
    const int c = a.queue[i];
    real w[NV][N];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int l = 0; l < N; ++l) w[v][l] = a.Uout[(size_t)(v * N + l) * nc + c];
    double mean64[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) mean64[v] = (double)w[v][0];
    // floors of density and pressure at the points: eps; for an FP32 state
    // the limited weights are stored rounded to FP32, which moves point
    // values by up to 2^-24 of the absolute weight sums (and the kinetic
    // energy at a near-vacuum point far more), so the floors also keep a
    // distance 2^-20 of those sums, at most half the mean
    double eps_r = a.eps, eps_p = a.eps;
    if constexpr (sizeof(real) == 4) {
      double ar = fabs(mean64[0]), ae = fabs(mean64[NV - 1]), m2 = 0.0;
#pragma unroll
      for (int l = 1; l < N; ++l) {
        ar += fabs((double)w[0][l]) * tab[S::OFF_PMAX + l];
        ae += fabs((double)w[NV - 1][l]) * tab[S::OFF_PMAX + l];
      }
#pragma unroll
      for (int b = 0; b < DIM; ++b) m2 += mean64[1 + b] * mean64[1 + b];
      const double pbar = (a.gamma - 1.0) * (mean64[NV - 1] - 0.5 * m2 / mean64[0]);
      eps_r = fmax(eps_r, fmin(0x1p-20 * ar, 0.5 * mean64[0]));
      eps_p = fmax(eps_p, fmin((a.gamma - 1.0) * 0x1p-20 * ae, 0.5 * pbar));
    }
    // points: the union set S, plus fine sub-face points on sides with a finer neighbour
    unsigned finer = 0;
    if (a.m.nnodes > 0)
      for (int sd = 0; sd < S::NSIDE; ++sd)
        if (a.m.nbr[(size_t)sd * nc + c] <= -2) finer |= 1u << sd;
    const int npts = S::NSP + __popc(finer) * S::NSUB * S::QF;
    auto point_row = [&](int ip) -> const double* {
      if (ip < S::NSP) return tab + S::OFF_SPHI + (size_t)ip * N;
      int r = ip - S::NSP;
      int sd = 0;
      for (; sd < S::NSIDE; ++sd) {
        if (!((finer >> sd) & 1)) continue;
        if (r < S::NSUB * S::QF) break;
        r -= S::NSUB * S::QF;
      }
      const int var = 1 + r / S::QF, q = r % S::QF;
      return tab + S::OFF_PHIF + (size_t)((sd * S::NVAR + var) * S::QF + q) * N;
    };
    double rmin = 1e300;
    for (int ip = lane; ip < npts; ip += 32) {
      const double* ph = point_row(ip);
      double rho = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) rho += (double)w[0][l] * ph[l];
      rmin = fmin(rmin, rho);
    }
    rmin = warp_min(rmin);
    if (rmin < eps_r) {
      const double th1 = fmin(fabs((mean64[0] - eps_r) / (mean64[0] - rmin)), 1.0);
#pragma unroll
      for (int l = 1; l < N; ++l) w[0][l] = (real)((double)w[0][l] * th1);
    }
    double th2 = 1.0;
    for (int ip = lane; ip < npts; ip += 32) {
      const double* ph = point_row(ip);
      double u[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double sum = 0.0;
#pragma unroll
        for (int l = 0; l < N; ++l) sum += (double)w[v][l] * ph[l];
        u[v] = sum;
      }
      double m2 = 0.0;
#pragma unroll
      for (int b = 0; b < DIM; ++b) m2 += u[1 + b] * u[1 + b];
      const double pr = (a.gamma - 1.0) * (u[DIM + 1] - 0.5 * m2 / u[0]);
      if (pr >= eps_p) continue;
      th2 = fmin(th2, positivity_tau<DIM>(mean64, u, a.gamma, eps_p));
    }
    th2 = warp_min(th2);
    if (lane == 0 && (rmin < eps_r || th2 < 1.0) && a.counts) atomicAdd(a.counts + 1, 1ull);
    if (th2 < 1.0) {
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int l = 1; l < N; ++l) w[v][l] = (real)((double)w[v][l] * th2);
    }
    if (rmin < eps_r || th2 < 1.0) {
      // the lanes share the stores
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int l = 0; l < N; ++l)
          if ((v * N + l) % 32 == lane) a.Uout[(size_t)(v * N + l) * nc + c] = w[v][l];
    }
  }
}

template <typename real, int DIM, int K>
__global__ void __launch_bounds__(128) positivity_kernel(const LimitArgs<real> a) {
  pdl_wait();
  positivity_body<real, DIM, K>(a, blockIdx.x, gridDim.x);
}

// ===========================================================================
// Auxiliary kernels

constexpr int RED_THREADS = 256;

// Block sum with warp shuffles in a fixed order (deterministic): a
// shuffle-down tree within each warp, then one over the warps' sums.  The
// result is valid in thread 0.
__device__ __forceinline__ double block_sum(double x, double* sh) {
  constexpr unsigned full = 0xffffffffu;
  constexpr int NW = RED_THREADS / 32;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(full, x, o);
  if (l == 0) sh[w] = x;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = l < NW ? sh[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(full, r, o);
  }
  __syncthreads();
  return r;
}

// Timestep (eq. time_step): dt = fac / max_K s_K with the signal speed
// s_K = sum_a (|v_a| + c) / dx_K of the cell mean; since correctly rounded
// division is monotone, fac / max s_K equals min_K fac / s_K exactly.  The
// maximum is accumulated as the bit pattern of a positive double.
// the work of block bid of nblk, THREADS threads per block
template <typename real, int DIM, int K, int THREADS, int B = 0>
__device__ __forceinline__ void dt_body(const AuxArgs<real>& a, int bid, int nblk) {
  using S = Shape<DIM, K, B>;
  const int c = bid * THREADS + threadIdx.x;
  const int nc = a.m.ncells;
  // the speeds are reduced in the state's precision and widened to FP64 at
  // the atomics (the widening is monotonic, so the maximum is the same)
  real speed = real(0);
  int pb = 0;
  if (c < nc) {
    // in the state's precision (an FP32 state's speed is FP32-accurate anyway)
    pb = cell_problem(a.m, c);
    real u[S::NV];
#pragma unroll
    for (int v = 0; v < S::NV; ++v) u[v] = a.W[(size_t)(v * S::N) * nc + c];
    const real gamma = real(a.gamma);
    const real rinv = real(1) / u[0];
    real m2 = real(0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) m2 += u[1 + b] * u[1 + b];
    const real p = (gamma - real(1)) * (u[DIM + 1] - real(0.5) * m2 * rinv);
    if (!(u[0] > real(0)) || !(p > real(0))) {
      atomicOr(a.status, 1 << DG_ERR_NONPHYSICAL_BIT);
    } else {
      const real cs = sqrt(gamma * p * rinv);
      real sum = real(0);
#pragma unroll
      for (int b = 0; b < DIM; ++b) sum += fabs(u[1 + b] * rinv) + cs;
      const real inv_dx = real(a.inv_dx_prob ? a.inv_dx_prob[pb] : a.inv_dx[0]);
      speed = sum * inv_dx * real(1 << a.m.level[c]);
      if (a.accel) {
        // gravity bound (Sec. 2.5) as a speed: dt_factor sqrt(2 gamma (gamma-1)) |a|_max / c,
        // |a| the largest over the cell's volume points
        real a2max = real(0);
#pragma unroll
        for (int q = 0; q < S::Q; ++q) {
          real a2 = real(0);
#pragma unroll
          for (int b = 0; b < DIM; ++b) {
            const real aq = a.accel[((size_t)b * S::Q + q) * nc + c];
            a2 += aq * aq;
          }
          a2max = fmax(a2max, a2);
        }
        speed = fmax(speed, real(a.grav_factor) * sqrt(a2max) / cs);
      }
    }
  } else {
    pb = -1;
  }
  // a warp whose cells belong to one problem reduces with shuffles; the block
  // then issues one atomic per run of warps with the same problem (a warp
  // spanning two problems falls back to one atomic per cell)
  __shared__ int sp[THREADS / 32];
  __shared__ real ss[THREADS / 32];
  const unsigned full = 0xffffffffu;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int p0 = __shfl_sync(full, pb, 0);
  if (p0 < 0) p0 = __reduce_max_sync(full, pb);  // lane 0 past the end: any valid lane's problem
  const bool uniform = __all_sync(full, pb == p0 || pb < 0);
  bool wrote = false;  // this thread issued a maximum atomic
  if (uniform) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) speed = fmax(speed, __shfl_xor_sync(full, speed, off));
  } else if (pb >= 0) {
    atomicMax(a.dt_bits + pb, (unsigned long long)__double_as_longlong((double)speed));
    wrote = true;
  }
  if (lane == 0) {
    sp[w] = uniform ? p0 : -1;
    ss[w] = speed;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int cur = -1;
    real m = real(0);
    for (int i = 0; i < THREADS / 32; ++i) {
      if (sp[i] != cur) {
        if (cur >= 0) atomicMax(a.dt_bits + cur, (unsigned long long)__double_as_longlong((double)m));
        cur = sp[i];
        m = real(0);
      }
      if (cur >= 0) m = fmax(m, ss[i]);
    }
    if (cur >= 0) atomicMax(a.dt_bits + cur, (unsigned long long)__double_as_longlong((double)m));
    wrote = true;
  }
  if (a.dt_out) {
    // every maximum this block issued is visible device-wide before the block
    // counts itself done (a fence by each thread that issued one); the last
    // block finishes the timestep and resets the maxima
    __shared__ int last;
    if (wrote) __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(a.dt_done, 1u) == (unsigned)nblk - 1u;
    __syncthreads();
    if (last) {
      __threadfence();
      const int np = a.m.nprob;
      for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const double speed = __longlong_as_double((long long)atomicExch(a.dt_bits + p, 0ull));
        const double v = speed > 0.0 ? a.dt_factor / speed : 0.0;
        a.dt_out[p] = v;
        if (a.dt_copy) a.dt_copy[p] = v;
      }
      if (threadIdx.x == 0) *a.dt_done = 0u;
    }
  }
}

template <typename real, int DIM, int K, int B = 0>
__global__ void __launch_bounds__(RED_THREADS) dt_kernel(const AuxArgs<real> a) {
  pdl_wait();
  dt_body<real, DIM, K, RED_THREADS, B>(a, blockIdx.x, gridDim.x);
}

template <typename real, int DIM, int K, int B = 0>
__global__ void __launch_bounds__(RED_THREADS) totals_kernel(const AuxArgs<real> a) {
  using S = Shape<DIM, K, B>;
  __shared__ double sh[RED_THREADS];
  const int c = blockIdx.x * RED_THREADS + threadIdx.x;
  const int nc = a.m.ncells;
  double vol = 0.0;
  if (c < nc) {
    const double dx = cell_dx(a.m, c);
    vol = DIM == 2 ? dx * dx : dx * dx * dx;
  }
  for (int v = 0; v < S::NV; ++v) {
    const double x = (c < nc) ? vol * (double)a.W[(size_t)(v * S::N) * nc + c] : 0.0;
    const double s = block_sum(x, sh);
    if (threadIdx.x == 0) a.partial[(size_t)blockIdx.x * S::NV + v] = s;
  }
}

template <typename real, int DIM, int K, int B = 0>
__global__ void __launch_bounds__(RED_THREADS) l1_kernel(const AuxArgs<real> a) {
  using S = Shape<DIM, K, B>;
  __shared__ double sh[RED_THREADS];
  const int c = blockIdx.x * RED_THREADS + threadIdx.x;
  const int nc = a.m.ncells;
  double cell = 0.0;
  if (c < nc) {
    double w[S::N];
    for (int l = 0; l < S::N; ++l) w[l] = (double)a.W[(size_t)l * nc + c];
    for (int q = 0; q < S::Q1; ++q) {
      const double* ph = a.tab64 + S::OFF_L1PHI + q * S::N;
      double rho = 0.0;
      for (int l = 0; l < S::N; ++l) rho += w[l] * ph[l];
      cell += fabs(rho - a.u[(size_t)q * nc + c]) * a.tab64[S::OFF_L1W + q];
    }
    const double hx = 0.5 * cell_dx(a.m, c);
    cell *= DIM == 2 ? hx * hx : hx * hx * hx;
  }
  const double s = block_sum(cell, sh);
  if (threadIdx.x == 0) a.partial[blockIdx.x] = s;
}

// partial[nblocks][nv] -> out[nv] (scaled), summed in block order
// one warp per variable: lane l sums blocks l, l+32, ... in order, then a
// fixed shuffle tree (deterministic)
static __global__ void reduce_partials_kernel(const double* partial, int nblocks, int nv, double scale,
                                       double* out) {
  const int v = blockIdx.x, l = threadIdx.x;
  if (v >= nv) return;
  double s = 0.0;
  for (int b = l; b < nblocks; b += 32) s += partial[(size_t)b * nv + v];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (l == 0) out[v] = s * scale;
}

template <typename real, int DIM, int K, int B = 0>
__global__ void project_kernel(const AuxArgs<real> a) {
  using S = Shape<DIM, K, B>;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int nc = a.m.ncells;
  if (c >= nc) return;
  for (int v = 0; v < S::NV; ++v) {
    double acc[S::N];
    for (int j = 0; j < S::N; ++j) acc[j] = 0.0;
    for (int q = 0; q < S::Q; ++q) {
      const double uq = a.u[((size_t)v * S::Q + q) * nc + c];
      for (int j = 0; j < S::N; ++j) acc[j] += uq * a.tab64[S::OFF_PROJ + q * S::N + j];
    }
    for (int j = 0; j < S::N; ++j) a.Wout[(size_t)(v * S::N + j) * nc + c] = (real)acc[j];
  }
}

template <typename real, int DIM, int K, int B = 0>
__global__ void points_kernel(const AuxArgs<real> a, int l1rule) {
  using S = Shape<DIM, K, B>;  // the table offsets depend on the basis size
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int nc = a.m.ncells;
  if (c >= nc) return;
  const int nq = l1rule ? S::Q1 : S::Q;
  const double* xi = a.tab64 + (l1rule ? S::OFF_XI1 : S::OFF_XI);
  const double dx = cell_dx(a.m, c);
  for (int d = 0; d < DIM; ++d) {
    const double lo = a.m.lo_prob ? a.m.lo_prob[3 * a.m.prob[c] + d] : a.m.lo[d];
    const double ctr = lo + ((double)a.m.coord[(size_t)d * nc + c] + 0.5) * dx;
    for (int q = 0; q < nq; ++q) a.out[((size_t)d * nq + q) * nc + c] = ctr + 0.5 * dx * xi[q * 3 + d];
  }
}

template <typename real, int DIM, int K>
__global__ void node_weights_kernel(const AuxArgs<real> a) {
  using S = Shape<DIM, K>;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int nn = a.m.nnodes, nc = a.m.ncells;
  if (m >= nn) return;
  const int* kids = a.m.node_children + (size_t)m * S::NCH;
  for (int v = 0; v < S::NV; ++v)
    for (int j = 0; j < S::N; ++j) {
      double s = 0.0;
      for (int ch = 0; ch < S::NCH; ++ch)
        for (int l = 0; l < S::N; ++l)
          s += a.tab64[S::OFF_PREF + (ch * S::N + l) * S::N + j] *
               (double)a.W[(size_t)(v * S::N + l) * nc + kids[ch]];
      a.Wout[(size_t)(v * S::N + j) * nn + m] = (real)(s / S::NCH);
    }
}

// ===========================================================================
// Launchers

template <typename real, int DIM, int K, int B = 0>
cudaError_t launch_face(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const StageArgs<real>*>(pa);
  using FT = FaceTile<real, DIM, K>;
  constexpr int NV = Shape<DIM, K>::NV;
  if (a.m.nfaces == 0) return cudaSuccess;
  const int fb = a.face_tile == 16 || a.face_tile == 64 ? a.face_tile : 32;
  const int grid = (a.m.nfaces + fb - 1) / fb;
  if (fb == 16) return launch_pdl(a.pdl, face_flux_kernel<real, DIM, K, 16, B>, grid, 16 * NV, FT::smem(16), s, a);
  if (fb == 64) return launch_pdl(a.pdl, face_flux_kernel<real, DIM, K, 64, B>, grid, 64 * NV, FT::smem(64), s, a);
  return launch_pdl(a.pdl, face_flux_kernel<real, DIM, K, 32, B>, grid, 32 * NV, FT::smem(32), s, a);
  return cudaGetLastError();
}

template <typename real, int DIM, int K, int B = 0>
cudaError_t launch_cell(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const StageArgs<real>*>(pa);
  using CT = CellTile<real, DIM, K>;
  constexpr int NV = Shape<DIM, K>::NV;
  if (a.m.ncells == 0) return cudaSuccess;
  const int tc = (a.cell_tile == 16 || a.cell_tile == 32 || a.cell_tile == 64) && a.cell_tile <= CT::TC_MAX
                     ? a.cell_tile
                     : CT::TC;
  if (a.accel) {  // gravity: the default tile only (not built for the tensor-product basis)
    if constexpr (B == 0) {
      cell_update_kernel<real, DIM, K, CT::TC, true><<<(a.m.ncells + CT::TC - 1) / CT::TC, CT::TC * NV,
                                                       CT::smem(CT::TC, true), s>>>(a);
      return cudaGetLastError();
    } else {
      return cudaErrorNotSupported;
    }
  }
  const int grid = (a.m.ncells + tc - 1) / tc;
  if (tc == 16) {
    return launch_pdl(a.pdl, cell_update_kernel<real, DIM, K, 16, false, B>, grid, 16 * NV, CT::smem(16), s, a);
  } else if (tc == 32) {
    if constexpr (CT::TC_MAX >= 32)
      return launch_pdl(a.pdl, cell_update_kernel<real, DIM, K, 32, false, B>, grid, 32 * NV, CT::smem(32), s, a);
  } else {
    if constexpr (CT::TC_MAX >= 64)
      return launch_pdl(a.pdl, cell_update_kernel<real, DIM, K, 64, false, B>, grid, 64 * NV, CT::smem(64), s, a);
  }
  return cudaGetLastError();
}

template <typename real>
__global__ void combine_kernel(const CombineArgs<real> a) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    real s = real(0);
    for (int r = 0; r < a.n_terms; ++r) s += a.c[r] * a.x[r][i];
    a.out[i] = s;
  }
}

template <typename real>
cudaError_t launch_combine(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const CombineArgs<real>*>(pa);
  if (a.n == 0) return cudaSuccess;
  const size_t blocks = std::min<size_t>((a.n + 255) / 256, (size_t)152 * 16);
  combine_kernel<real><<<(unsigned)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename real, int DIM, int K, int B = 0>
cudaError_t prepare_kernels() {
  if constexpr (B == 0) {
    cudaError_t e0 = prepare_adjoint_kernels<real, DIM, K>();
    if (e0 != cudaSuccess) return e0;
  }
  using CT = CellTile<real, DIM, K>;
  using FT = FaceTile<real, DIM, K>;
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(cell_update_kernel<real, DIM, K, 16, false, B>, attr, (int)CT::smem(16));
  if (e == cudaSuccess && CT::TC_MAX >= 32) {
    if constexpr (CT::TC_MAX >= 32)
      e = cudaFuncSetAttribute(cell_update_kernel<real, DIM, K, 32, false, B>, attr, (int)CT::smem(32));
  }
  if (e == cudaSuccess && CT::TC_MAX >= 64) {
    if constexpr (CT::TC_MAX >= 64)
      e = cudaFuncSetAttribute(cell_update_kernel<real, DIM, K, 64, false, B>, attr, (int)CT::smem(64));
  }
  if (e != cudaSuccess) return e;
  if constexpr (B == 0) {
    if ((e = cudaFuncSetAttribute(cell_update_kernel<real, DIM, K, CT::TC, true>, attr,
                                  (int)CT::smem(CT::TC, true))) != cudaSuccess)
      return e;
  }
  if ((e = cudaFuncSetAttribute(face_flux_kernel<real, DIM, K, 16, B>, attr, (int)FT::smem(16))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(face_flux_kernel<real, DIM, K, 32, B>, attr, (int)FT::smem(32))) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(face_flux_kernel<real, DIM, K, 64, B>, attr, (int)FT::smem(64));
}

template <typename real, int DIM, int K>
cudaError_t launch_limit(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const LimitArgs<real>*>(pa);
  if (a.m.ncells == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.queue_len, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if ((e = launch_pdl(a.pdl, limit_kernel<real, DIM, K>, (a.m.ncells + 127) / 128, 128, 0, s, a)) != cudaSuccess)
    return e;
  if (a.positivity && K > 0) {
    // the queue's length is known on the device only: a fixed grid strides over it
    const int blocks = (a.m.ncells + 127) / 128 < 608 ? (a.m.ncells + 127) / 128 : 608;
    cudaError_t e2 = launch_pdl(a.pdl, positivity_kernel<real, DIM, K>, blocks, 128, 0, s, a);
    if (e2 != cudaSuccess) return e2;
  }
  return cudaGetLastError();
}

template <typename real, int DIM, int K, int B = 0>
cudaError_t launch_project(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const AuxArgs<real>*>(pa);
  if (a.m.ncells == 0) return cudaSuccess;
  project_kernel<real, DIM, K, B><<<(a.m.ncells + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename real, int DIM, int K, int B = 0>
cudaError_t launch_points(const void* pa, int l1rule, cudaStream_t s) {
  const auto& a = *static_cast<const AuxArgs<real>*>(pa);
  if (a.m.ncells == 0) return cudaSuccess;
  points_kernel<real, DIM, K, B><<<(a.m.ncells + 127) / 128, 128, 0, s>>>(a, l1rule);
  return cudaGetLastError();
}

template <typename real, int DIM, int K, int B = 0>
cudaError_t launch_dt(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const AuxArgs<real>*>(pa);
  if (a.m.ncells == 0) return cudaSuccess;
  return launch_pdl(a.pdl, dt_kernel<real, DIM, K, B>, (a.m.ncells + RED_THREADS - 1) / RED_THREADS, RED_THREADS, 0, s,
                    a);  // per-problem max
  return cudaGetLastError();
}

template <typename real, int DIM, int K, int B = 0>
cudaError_t launch_totals(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const AuxArgs<real>*>(pa);
  using S = Shape<DIM, K, B>;
  const int nb = (a.m.ncells + RED_THREADS - 1) / RED_THREADS;
  if (nb > 0) totals_kernel<real, DIM, K, B><<<nb, RED_THREADS, 0, s>>>(a);
  reduce_partials_kernel<<<S::NV, 32, 0, s>>>(a.partial, nb, S::NV, 1.0, a.out);
  return cudaGetLastError();
}

template <typename real, int DIM, int K, int B = 0>
cudaError_t launch_l1(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const AuxArgs<real>*>(pa);
  const int nb = (a.m.ncells + RED_THREADS - 1) / RED_THREADS;
  if (nb > 0) l1_kernel<real, DIM, K, B><<<nb, RED_THREADS, 0, s>>>(a);
  reduce_partials_kernel<<<1, 32, 0, s>>>(a.partial, nb, 1, 1.0 / a.volume, a.out);
  return cudaGetLastError();
}

template <typename real, int DIM, int K>
cudaError_t launch_node_weights(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const AuxArgs<real>*>(pa);
  if (a.m.nnodes == 0) return cudaSuccess;
  node_weights_kernel<real, DIM, K><<<(a.m.nnodes + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dgi

#include "dg_fused.cuh"
#include "dg_persist.cuh"
#include "dg_x2.cuh"

namespace dgi {

template <typename real, int DIM, int K, int B = 0>
KernelSet make_kernel_set(int prec) {
  using S = Shape<DIM, K, B>;
  KernelSet ks;
  ks.dim = DIM;
  ks.k = K;
  ks.prec = prec;
  ks.basis = B;
  ks.N = S::N;
  ks.NV = S::NV;
  ks.Q = S::Q;
  ks.QF = S::QF;
  ks.Q1 = S::Q1;
  ks.NSUB = S::NSUB;
  ks.NSP = S::NSP;
  ks.M = S::M;
  ks.tab_size = S::TAB_SIZE;
  ks.off_pref = S::OFF_PREF;
  ks.fill_tables = &fill_tables<DIM, K, B>;
  ks.prepare = &prepare_kernels<real, DIM, K, B>;
  ks.cell_tile = CellTile<real, DIM, K>::TC;
  ks.cell_tile_max = CellTile<real, DIM, K>::TC_MAX;
  ks.face_tile = FaceTile<real, DIM, K>::FB;
  ks.face_tile_max = FaceTile<real, DIM, K>::FB_MAX;
  ks.face = &launch_face<real, DIM, K, B>;
  ks.cell = &launch_cell<real, DIM, K, B>;
  ks.project = &launch_project<real, DIM, K, B>;
  ks.points = &launch_points<real, DIM, K, B>;
  ks.dt = &launch_dt<real, DIM, K, B>;
  ks.totals = &launch_totals<real, DIM, K, B>;
  ks.l1 = &launch_l1<real, DIM, K, B>;
  ks.combine = &launch_combine<real>;
  // the tensor-product basis has the stage, timestep, projection and
  // diagnostic kernels only
  if constexpr (B == 0) {
    ks.limit = &launch_limit<real, DIM, K>;
    ks.node_weights = &launch_node_weights<real, DIM, K>;
    ks.adj_face = &launch_adj_face<real, DIM, K>;
    ks.adj_cell = &launch_adj_cell<real, DIM, K>;
    if constexpr (std::is_same<real, float>::value && DIM == 2) {
      ks.cell_x2 = &launch_cell_x2<K>;
      ks.cell_direct = &launch_cell_direct<DIM, K>;
      ks.fill_direct = &fill_direct_tables<DIM, K>;
    }
    if constexpr (DIM == 2) {
      ks.persist = &launch_persist<real, DIM, K>;
      ks.prepare_persist = &prepare_persist<real, DIM, K>;
      ks.stage_fused = &launch_stage_fused<real, K>;
      ks.prepare_fused = &prepare_stage_fused<real, K>;
    }
    if constexpr (std::is_same<real, float>::value && DIM == 2 && K >= 1 && K <= 3) {
      ks.cell_tc = &launch_cell_tc<K, false>;
      ks.prepare_tc = &prepare_cell_tc<K, false>;
      ks.fill_tc = &fill_tc_tables<K>;
    }
  }
  return ks;
}

}  // namespace dgi
