// Adjoint (transposed linearisation) of the DG time derivative, for the
// adjoint of one RK step with a frozen timestep.  Not in the paper: the
// derivative of the scheme of Sec. 2.4 with respect to the weights.
//
// dW/dt = pre (V - S) with V_j = sum_d sum_q f_d(u(q)) dphi_j/dxi_d(q) w_q and
// S_j the surface integral of the HLLC fluxes.  For a cotangent G on dW/dt:
//   volume : g_d(q) = pre sum_j G_j dphi_j/dxi_d(q) w_q,
//            ubar(q) = sum_d (df_d/du)^T g_d,   Ubar_l += sum_q ubar(q) phi_l(q);
//   faces  : Fbar(q) = w_q (pre_p t_p(q) - pre_m t_m(q)), t = trace of G,
//            ubar_-/+ = (dF/du_-/+)^T Fbar,     Ubar_l += sum_q ubar(q) phi_l(q)
// (the coarse side of a hanging face carries its sub-face weight 2^-(d-1)).
// The Jacobian-transpose products of the point flux and of HLLC are
// reverse-mode derivatives of the same formulas, written out by hand.
#pragma once
#include <cuda_runtime.h>

#include "dg_internal.h"
#include "dg_physics.cuh"
#include "dg_stage.cuh"

namespace dgi {

// Jacobian-transpose products of the fluxes by reverse-mode differentiation
// written out by hand: the forward formulas of euler_flux / hllc_flux are
// evaluated once, then their adjoints are accumulated in reverse order.

// out = sum_d (df_d/du)^T g_d at one point (f_d the Euler flux of eqs.
// flux_vectors and eos)
template <typename real, int DIM>
__device__ __forceinline__ void flux_vjp(const real* u, const real (*g)[DIM + 2], real g1,
                                         real* out) {
  constexpr int E = DIM + 1;
  const real rinv = recip(u[0]);
  real v[DIM], m2 = real(0);
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    v[b] = u[1 + b] * rinv;
    m2 += u[1 + b] * v[b];
  }
  const real p = g1 * (u[E] - real(0.5) * m2);
  const real H = u[E] + p;
  // forward, per direction a: f0 = m_a, f_(1+b) = m_b v_a + delta_ab p, f_E = H v_a
  real mb[DIM], vb[DIM];
#pragma unroll
  for (int b = 0; b < DIM; ++b) { mb[b] = real(0); vb[b] = real(0); }
  real pb = real(0), Eb = real(0);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const real* ga = g[a];
    mb[a] += ga[0];
    real s = real(0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      mb[b] += ga[1 + b] * v[a];
      s += ga[1 + b] * u[1 + b];
    }
    vb[a] += s + ga[E] * H;
    pb += ga[1 + a] + ga[E] * v[a];
    Eb += ga[E] * v[a];
  }
  // p = g1 (E - m2 / 2), m2 = sum_b m_b v_b, v_b = m_b / rho
  Eb += g1 * pb;
  const real m2b = real(-0.5) * g1 * pb;
  real rinvb = real(0);
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    mb[b] += m2b * v[b];
    vb[b] += m2b * u[1 + b];
    mb[b] += vb[b] * rinv;
    rinvb += vb[b] * u[1 + b];
  }
  out[0] = -rinvb * rinv * rinv;
#pragma unroll
  for (int b = 0; b < DIM; ++b) out[1 + b] = mb[b];
  out[E] = Eb;
}

// outL = (dF/duL)^T fbar, outR = (dF/duR)^T fbar for the HLLC flux in
// direction A (the construction of hllc_flux, branch by branch)
template <typename real, int DIM, int A>
__device__ __forceinline__ void hllc_vjp(const real* uL, const real* uR, real gamma,
                                         const real* fbar, real* outL, real* outR) {
  constexpr int NV = DIM + 2, E = DIM + 1;
  const real g1 = gamma - real(1);
  // ---- forward
  const real rL = uL[0], rR = uR[0];
  const real iL = recip(rL), iR = recip(rR);
  real kL = real(0), kR = real(0);
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    kL += uL[1 + b] * uL[1 + b];
    kR += uR[1 + b] * uR[1 + b];
  }
  const real pL = g1 * (uL[E] - real(0.5) * kL * iL);
  const real pR = g1 * (uR[E] - real(0.5) * kR * iR);
  const real vL = uL[1 + A] * iL, vR = uR[1 + A] * iR;
  const real XL = gamma * pL * iL, XR = gamma * pR * iR;
  const real cL = sqrt_pos(XL), cR = sqrt_pos(XR);
  const bool minR = (vR - cR) < (vL - cL);  // S_L from the right state
  const bool maxR = (vL + cL) < (vR + cR);  // S_R from the right state
  const real SL = minR ? vR - cR : vL - cL;
  const real SR = maxR ? vR + cR : vL + cL;
  const real dL = rL * (SL - vL), dR = rR * (SR - vR);
  const real num = pR - pL + vL * dL - vR * dR, den = dL - dR;
  const real iden = recip(den);
  const real Ss = num * iden;
  const bool left = (SL >= real(0)) || (Ss >= real(0));
  const bool star = left ? (SL < real(0)) : (SR > real(0));
  const real* u = left ? uL : uR;
  const real r = left ? rL : rR;
  const real ir = left ? iL : iR;
  const real v = left ? vL : vR;
  const real p = left ? pL : pR;
  const real S = left ? SL : SR;
  // ---- reverse: adjoints of the side-K quantities first
  real ub[NV];  // direct adjoint of u_K
#pragma unroll
  for (int i = 0; i < NV; ++i) ub[i] = real(0);
  real vb = real(0), pb = real(0), irb = real(0), rb = real(0), Sb = real(0), Ssb = real(0);
  if (star) {
    const real rsv = r * (S - v);
    const real Dn = S - Ss;
    const real irsv = recip(rsv), iDn = recip(Dn);
    const real fac = rsv * iDn;
    const real prs = p * irsv;
    const real Y = u[E] * ir + (Ss - v) * (Ss + prs);
    real us[NV];
    us[0] = fac;
#pragma unroll
    for (int b = 0; b < DIM; ++b) us[1 + b] = fac * (u[1 + b] * ir);
    us[1 + A] = fac * Ss;
    us[E] = fac * Y;
    // F_i += S (us_i - u_i)
    real facb = real(0);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      Sb += fbar[i] * (us[i] - u[i]);
      ub[i] -= S * fbar[i];
    }
    facb += S * fbar[0];
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      if (b == A) continue;
      const real usb = S * fbar[1 + b];
      facb += usb * u[1 + b] * ir;
      ub[1 + b] += usb * fac * ir;
      irb += usb * fac * u[1 + b];
    }
    {
      const real usb = S * fbar[1 + A];
      facb += usb * Ss;
      Ssb += usb * fac;
    }
    {
      const real usb = S * fbar[E];
      facb += usb * Y;
      const real Yb = usb * fac;
      ub[E] += Yb * ir;
      irb += Yb * u[E];
      const real Ab = Yb * (Ss + prs), Bb = Yb * (Ss - v);
      Ssb += Ab + Bb;
      vb -= Ab;
      const real prsb = Bb;
      pb += prsb * irsv;
      real rsvb = -prsb * prs * irsv;
      // fac = rsv / Dn, Dn = S - Ss
      rsvb += facb * iDn;
      const real Dnb = -facb * fac * iDn;
      Sb += Dnb;
      Ssb -= Dnb;
      // rsv = r (S - v)
      rb += rsvb * (S - v);
      Sb += rsvb * r;
      vb -= rsvb * r;
    }
  }
  // physical flux of side K: F0 = m_A, F_(1+b) = m_b v + delta_Ab p, F_E = (E + p) v
  ub[1 + A] += fbar[0];
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    ub[1 + b] += fbar[1 + b] * v;
    vb += fbar[1 + b] * u[1 + b];
  }
  pb += fbar[1 + A] + fbar[E] * v;
  ub[E] += fbar[E] * v;
  vb += fbar[E] * (u[E] + p);
  // ---- per-side accumulators
  real bL[NV], bR[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    bL[i] = left ? ub[i] : real(0);
    bR[i] = left ? real(0) : ub[i];
  }
  real vLb = left ? vb : real(0), vRb = left ? real(0) : vb;
  real pLb = left ? pb : real(0), pRb = left ? real(0) : pb;
  real iLb = left ? irb : real(0), iRb = left ? real(0) : irb;
  bL[0] += left ? rb : real(0);
  bR[0] += left ? real(0) : rb;
  real SLb = left ? Sb : real(0), SRb = left ? real(0) : Sb;
  // S* = num / den
  const real numb = Ssb * iden;
  const real denb = -Ssb * Ss * iden;
  pRb += numb;
  pLb -= numb;
  vLb += numb * dL;
  real dLb = numb * vL + denb;
  vRb -= numb * dR;
  real dRb = -numb * vR - denb;
  // dL = rL (SL - vL), dR = rR (SR - vR)
  bL[0] += dLb * (SL - vL);
  SLb += dLb * rL;
  vLb -= dLb * rL;
  bR[0] += dRb * (SR - vR);
  SRb += dRb * rR;
  vRb -= dRb * rR;
  // SL = min(vL - cL, vR - cR), SR = max(vL + cL, vR + cR)
  real cLb = real(0), cRb = real(0);
  if (minR) { vRb += SLb; cRb -= SLb; } else { vLb += SLb; cLb -= SLb; }
  if (maxR) { vRb += SRb; cRb += SRb; } else { vLb += SRb; cLb += SRb; }
  // c = sqrt(gamma p i)
  {
    const real XLb = cLb * recip(real(2) * cL), XRb = cRb * recip(real(2) * cR);
    pLb += XLb * gamma * iL;
    iLb += XLb * gamma * pL;
    pRb += XRb * gamma * iR;
    iRb += XRb * gamma * pR;
  }
  // v = m_A i
  bL[1 + A] += vLb * iL;
  iLb += vLb * uL[1 + A];
  bR[1 + A] += vRb * iR;
  iRb += vRb * uR[1 + A];
  // p = g1 (E - k i / 2), k = |m|^2
  bL[E] += g1 * pLb;
  bR[E] += g1 * pRb;
  const real kLb = real(-0.5) * g1 * pLb * iL, kRb = real(-0.5) * g1 * pRb * iR;
  iLb += real(-0.5) * g1 * pLb * kL;
  iRb += real(-0.5) * g1 * pRb * kR;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    bL[1 + b] += real(2) * uL[1 + b] * kLb;
    bR[1 + b] += real(2) * uR[1 + b] * kRb;
  }
  // i = 1 / rho
  bL[0] -= iLb * iL * iL;
  bR[0] -= iRb * iR * iR;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    outL[i] = bL[i];
    outR[i] = bR[i];
  }
}

// point values of sum_l c_l prod_a TAB_a[e_a][i_a] with one table per axis
// (the factorised modal->nodal with the tables chosen per axis)
template <typename real, int DIM, int K>
__device__ __forceinline__ void modal_to_nodal_axes(const real (&T0)[4][4], const real (&T1)[4][4],
                                                    const real (&T2)[4][4], const real* w,
                                                    real* u) {
  constexpr int K1 = K + 1;
  if constexpr (DIM == 2) {
    real t[K1][K1];
#pragma unroll
    for (int a = 0; a <= K; ++a)
#pragma unroll
      for (int j = 0; j < K1; ++j) {
        real s = real(0);
#pragma unroll
        for (int b = 0; b <= K - a; ++b) s += w[bidx<2>(a, b, 0)] * T1[b][j];
        t[a][j] = s;
      }
#pragma unroll
    for (int j = 0; j < K1; ++j)
#pragma unroll
      for (int i = 0; i < K1; ++i) {
        real s = real(0);
#pragma unroll
        for (int a = 0; a <= K; ++a) s += T0[a][i] * t[a][j];
        u[i + K1 * j] = s;
      }
  } else {
    real t1[K1][K1][K1];
#pragma unroll
    for (int a = 0; a <= K; ++a)
#pragma unroll
      for (int b = 0; b <= K - a; ++b)
#pragma unroll
        for (int kz = 0; kz < K1; ++kz) {
          real s = real(0);
#pragma unroll
          for (int c = 0; c <= K - a - b; ++c) s += w[bidx<3>(a, b, c)] * T2[c][kz];
          t1[a][b][kz] = s;
        }
    real t2[K1][K1][K1];
#pragma unroll
    for (int a = 0; a <= K; ++a)
#pragma unroll
      for (int j = 0; j < K1; ++j)
#pragma unroll
        for (int kz = 0; kz < K1; ++kz) {
          real s = real(0);
#pragma unroll
          for (int b = 0; b <= K - a; ++b) s += t1[a][b][kz] * T1[b][j];
          t2[a][j][kz] = s;
        }
#pragma unroll
    for (int kz = 0; kz < K1; ++kz)
#pragma unroll
      for (int j = 0; j < K1; ++j)
#pragma unroll
        for (int i = 0; i < K1; ++i) {
          real s = real(0);
#pragma unroll
          for (int a = 0; a <= K; ++a) s += T0[a][i] * t2[a][j][kz];
          u[i + K1 * (j + K1 * kz)] = s;
        }
  }
}

// transpose of modal_to_nodal: c_l += sum_q u(q) phi_l(q)
template <typename real, int DIM, int K>
__device__ __forceinline__ void nodal_to_modal(const real (&P)[4][4], const real* u, real* c) {
  constexpr int K1 = K + 1;
  if constexpr (DIM == 2) {
#pragma unroll
    for (int a = 0; a <= K; ++a)
#pragma unroll
      for (int j = 0; j < K1; ++j) {
        real h = real(0);
#pragma unroll
        for (int i = 0; i < K1; ++i) h += u[i + K1 * j] * P[a][i];
#pragma unroll
        for (int b = 0; b <= K - a; ++b) c[bidx<2>(a, b, 0)] += h * P[b][j];
      }
  } else {
#pragma unroll
    for (int a = 0; a <= K; ++a) {
      real h1[K1][K1];  // [j][kz]
#pragma unroll
      for (int j = 0; j < K1; ++j)
#pragma unroll
        for (int kz = 0; kz < K1; ++kz) {
          real s = real(0);
#pragma unroll
          for (int i = 0; i < K1; ++i) s += u[i + K1 * (j + K1 * kz)] * P[a][i];
          h1[j][kz] = s;
        }
#pragma unroll
      for (int b = 0; b <= K - a; ++b)
#pragma unroll
        for (int kz = 0; kz < K1; ++kz) {
          real h2 = real(0);
#pragma unroll
          for (int j = 0; j < K1; ++j) h2 += h1[j][kz] * P[b][j];
#pragma unroll
          for (int c3 = 0; c3 <= K - a - b; ++c3) c[bidx<3>(a, b, c3)] += h2 * P[c3][kz];
        }
    }
  }
}

// transpose of face_trace: c_l += sum_q u(q) phi_l(face point q) (unweighted)
template <typename real, int DIM, int K, int DIR, int S>
__device__ __forceinline__ void trace_transpose(const Tab1D<real>& T, const real (&PT0)[4][4],
                                                const real (&PT1)[4][4], const real* uq,
                                                real* c) {
  constexpr int K1 = K + 1;
  if constexpr (DIM == 2) {
#pragma unroll
    for (int et = 0; et <= K; ++et) {
      real g = real(0);
#pragma unroll
      for (int q = 0; q < K1; ++q) g += uq[q] * PT0[et][q];
#pragma unroll
      for (int ed = 0; ed <= K - et; ++ed)
        c[DIR == 0 ? bidx<2>(ed, et, 0) : bidx<2>(et, ed, 0)] += T.PE[S][ed] * g;
    }
  } else {
    constexpr int A = DIR == 0 ? 1 : 0;
    constexpr int B = DIR == 2 ? 1 : 2;
    real H[K1][K1];
#pragma unroll
    for (int ea = 0; ea <= K; ++ea)
#pragma unroll
      for (int qb = 0; qb < K1; ++qb) {
        real s = real(0);
#pragma unroll
        for (int qa = 0; qa < K1; ++qa) s += uq[qa + K1 * qb] * PT0[ea][qa];
        H[ea][qb] = s;
      }
#pragma unroll
    for (int ea = 0; ea <= K; ++ea)
#pragma unroll
      for (int eb = 0; eb <= K - ea; ++eb) {
        real s = real(0);
#pragma unroll
        for (int qb = 0; qb < K1; ++qb) s += H[ea][qb] * PT1[eb][qb];
#pragma unroll
        for (int ed = 0; ed <= K - ea - eb; ++ed) {
          int e[3];
          e[DIR] = ed;
          e[A] = ea;
          e[B] = eb;
          c[bidx<3>(e[0], e[1], e[2])] += T.PE[S][ed] * s;
        }
      }
  }
}

// ===========================================================================
// Adjoint face kernel: FB faces x NV threads.
//   1. thread (face, var): traces of U and of G on both sides -> shared memory;
//   2. thread (face, point): Fbar, then ubar on both sides -> UB[side][var][point][face].

template <typename real, int DIM, int K>
struct AdjFaceTile {
  using S = Shape<DIM, K>;
  static constexpr int FB = 32;
  static constexpr int THREADS = FB * S::NV;
  static constexpr size_t SMEM = (size_t)4 * S::NV * S::QF * FB * sizeof(real);
};

template <typename real, int DIM, int K, int DIR>
__device__ __forceinline__ void trace_of(const AdjointArgs<real>& a, const real* X, int cell,
                                         int s, int var, int v, real* u) {
  using S = Shape<DIM, K>;
  const Tab1D<real>& T = a.t1;
  const int nc = a.m.ncells;
  real w[S::N];
#pragma unroll
  for (int l = 0; l < S::N; ++l) w[l] = X[(size_t)(v * S::N + l) * nc + cell];
  if (var == 0) {
    face_trace<real, DIM, K, DIR>(T, w, s, T.P, T.P, u);
  } else {
    const int h0 = (var - 1) & 1, h1 = ((var - 1) >> 1) & 1;
    face_trace<real, DIM, K, DIR>(T, w, s, T.PH[h0], T.PH[h1], u);
  }
}

template <typename real, int DIM, int K>
__global__ void __launch_bounds__(AdjFaceTile<real, DIM, K>::THREADS)
    adjoint_face_kernel(const AdjointArgs<real> a) {
  using S = Shape<DIM, K>;
  using FT = AdjFaceTile<real, DIM, K>;
  constexpr int FB = FT::FB, NV = S::NV, QF = S::QF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* sU = reinterpret_cast<real*>(smem_raw);  // [2][NV][QF][FB] traces of U
  real* sG = sU + 2 * NV * QF * FB;              // [2][NV][QF][FB] traces of G
  const int nf = a.m.nfaces, nc = a.m.ncells;
  const int fl = threadIdx.x % FB, v = threadIdx.x / FB;
  const int f = blockIdx.x * FB + fl;
  if (f < nf) {
    const unsigned info = a.m.finfo[f];
    const int dir = info & 3, vm = (info >> 2) & 7, vp = (info >> 5) & 7;
    const int cm = a.m.fm[f], cp = a.m.fp[f];
    auto tr = [&](const real* X, int cell, int s, int var, real* u) {
      if (dir == 0) trace_of<real, DIM, K, 0>(a, X, cell, s, var, v, u);
      else if (dir == 1) trace_of<real, DIM, K, 1>(a, X, cell, s, var, v, u);
      else if constexpr (DIM == 3) trace_of<real, DIM, K, DIM - 1>(a, X, cell, s, var, v, u);
    };
    real um[QF], up[QF], gm[QF], gp[QF];
#pragma unroll
    for (int q = 0; q < QF; ++q) { um[q] = up[q] = gm[q] = gp[q] = real(0); }
    if (cm >= 0) {
      tr(a.U, cm, 1, vm, um);
      tr(a.G, cm, 1, vm, gm);
    }
    if (cp >= 0) {
      tr(a.U, cp, 0, vp, up);
      tr(a.G, cp, 0, vp, gp);
    }
    if (cm < 0) {
#pragma unroll
      for (int q = 0; q < QF; ++q) um[q] = up[q];
    }
    if (cp < 0) {
#pragma unroll
      for (int q = 0; q < QF; ++q) up[q] = um[q];
    }
    // G traces scaled by the cell's prefactor and its integration weight
    auto pre_of = [&](int cell) {
      return a.pre_prob ? a.pre_prob[cell_problem(a.m, cell)] : a.pre[a.m.level[cell]];
    };
    const real pm = cm >= 0 ? pre_of(cm) * (vm ? real(1) / real(S::NSUB) : real(1)) : real(0);
    const real pp = cp >= 0 ? pre_of(cp) * (vp ? real(1) / real(S::NSUB) : real(1)) : real(0);
#pragma unroll
    for (int q = 0; q < QF; ++q) {
      sU[((0 * NV + v) * QF + q) * FB + fl] = um[q];
      sU[((1 * NV + v) * QF + q) * FB + fl] = up[q];
      sG[((0 * NV + v) * QF + q) * FB + fl] = pm * gm[q];
      sG[((1 * NV + v) * QF + q) * FB + fl] = pp * gp[q];
    }
  }
  __syncthreads();
  const real gamma = real(a.gamma);
  const Tab1D<real>& T = a.t1;
  for (int item = threadIdx.x; item < FB * QF; item += FT::THREADS) {
    const int ff = item % FB, q = item / FB;
    const int f2 = blockIdx.x * FB + ff;
    if (f2 >= nf) continue;
    const int d2 = a.m.finfo[f2] & 3;
    const int cm = a.m.fm[f2], cp = a.m.fp[f2];
    // face point weight (product of the tangential Gauss weights)
    real wq = real(1);
    {
      int qq = q;
#pragma unroll
      for (int t = 0; t < DIM - 1; ++t) {
        wq *= T.W[qq % (K + 1)];
        qq /= (K + 1);
      }
    }
    real uL[NV], uR[NV], fb[NV], bl[NV], br[NV];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) {
      uL[vv] = sU[((0 * NV + vv) * QF + q) * FB + ff];
      uR[vv] = sU[((1 * NV + vv) * QF + q) * FB + ff];
      // dW_minus/dt has -pre F phi w, dW_plus/dt has +pre F phi w
      fb[vv] = wq * (sG[((1 * NV + vv) * QF + q) * FB + ff] - sG[((0 * NV + vv) * QF + q) * FB + ff]);
    }
    if (d2 == 0) hllc_vjp<real, DIM, 0>(uL, uR, gamma, fb, bl, br);
    else if (d2 == 1) hllc_vjp<real, DIM, 1>(uL, uR, gamma, fb, bl, br);
    else hllc_vjp<real, DIM, DIM - 1>(uL, uR, gamma, fb, bl, br);
    // a mirrored side is the other side's own trace
    if (cm < 0) {
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) { br[vv] += bl[vv]; bl[vv] = real(0); }
    }
    if (cp < 0) {
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) { bl[vv] += br[vv]; br[vv] = real(0); }
    }
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) {
      a.FG[(((size_t)0 * NV + vv) * QF + q) * nf + f2] = bl[vv];
      a.FG[(((size_t)1 * NV + vv) * QF + q) * nf + f2] = br[vv];
    }
  }
  (void)nc;
}

// ===========================================================================
// Adjoint cell kernel: TC cells x NV threads.

template <typename real, int DIM, int K>
struct AdjCellTile {
  using S = Shape<DIM, K>;
  static constexpr size_t PER_CELL =
      (size_t)(S::NV * S::Q + DIM * S::NV * S::Q + S::NV * S::Q) * sizeof(real);
  static constexpr int TC = PER_CELL * 32 > 96 * 1024 ? 16 : 32;
  static constexpr int THREADS = TC * S::NV;
  static constexpr size_t SMEM = PER_CELL * TC;
};

template <typename real, int DIM, int K, int SD>
__device__ __forceinline__ void gather_face_adjoint(const AdjointArgs<real>& a, int c, int v,
                                                    unsigned coarse, real* acc) {
  using S = Shape<DIM, K>;
  constexpr int DIR = SD >> 1, SS = SD & 1;
  const Tab1D<real>& T = a.t1;
  const int nc = a.m.ncells, nf = a.m.nfaces;
  const int e0 = a.m.sface[(size_t)SD * nc + c];
  // the cell is the minus side (role 0) of faces on its + side, the plus side otherwise
  constexpr int ROLE = SS ? 0 : 1;
  real uq[S::QF];
  if (!((coarse >> SD) & 1)) {
#pragma unroll
    for (int q = 0; q < S::QF; ++q)
      uq[q] = a.FG[(((size_t)ROLE * S::NV + v) * S::QF + q) * nf + e0];
    trace_transpose<real, DIM, K, DIR, SS>(T, T.P, T.P, uq, acc);
  } else {
#pragma unroll
    for (int h = 0; h < S::NSUB; ++h) {
#pragma unroll
      for (int q = 0; q < S::QF; ++q)
        uq[q] = a.FG[(((size_t)ROLE * S::NV + v) * S::QF + q) * nf + e0 + h];
      trace_transpose<real, DIM, K, DIR, SS>(T, T.PH[h & 1], T.PH[(h >> 1) & 1], uq, acc);
    }
  }
}

template <typename real, int DIM, int K>
__global__ void __launch_bounds__(AdjCellTile<real, DIM, K>::THREADS)
    adjoint_cell_kernel(const AdjointArgs<real> a) {
  using S = Shape<DIM, K>;
  using CT = AdjCellTile<real, DIM, K>;
  constexpr int TC = CT::TC, NV = S::NV, Q = S::Q, N = S::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* sU = reinterpret_cast<real*>(smem_raw);  // [NV][Q][TC] nodal U
  real* sG = sU + NV * Q * TC;                   // [DIM][NV][Q][TC] nodal g_d
  real* sB = sG + DIM * NV * Q * TC;             // [NV][Q][TC] nodal ubar
  const int tc = threadIdx.x % TC, v = threadIdx.x / TC;
  const int nc = a.m.ncells;
  const int c = blockIdx.x * TC + tc;
  const bool valid = c < nc;
  const Tab1D<real>& T = a.t1;
  const real pre = !valid ? real(0)
                   : (a.pre_prob ? a.pre_prob[cell_problem(a.m, c)] : a.pre[a.m.level[c]]);
  {
    real w[N], u[Q];
#pragma unroll
    for (int l = 0; l < N; ++l)
      w[l] = valid ? a.U[(size_t)(v * N + l) * nc + c] : ((v == 0 && l == 0) ? real(1) : real(0));
    modal_to_nodal<real, DIM, K>(T, w, u);
#pragma unroll
    for (int q = 0; q < Q; ++q) sU[(v * Q + q) * TC + tc] = u[q];
#pragma unroll
    for (int l = 0; l < N; ++l) w[l] = valid ? pre * a.G[(size_t)(v * N + l) * nc + c] : real(0);
    // g_d(q) = sum_j G_j dphi_j/dxi_d(q) w_q: derivative table on axis d, weighted elsewhere
    modal_to_nodal_axes<real, DIM, K>(T.DW, T.PW, T.PW, w, u);
#pragma unroll
    for (int q = 0; q < Q; ++q) sG[((0 * NV + v) * Q + q) * TC + tc] = u[q];
    modal_to_nodal_axes<real, DIM, K>(T.PW, T.DW, T.PW, w, u);
#pragma unroll
    for (int q = 0; q < Q; ++q) sG[((1 * NV + v) * Q + q) * TC + tc] = u[q];
    if constexpr (DIM == 3) {
      modal_to_nodal_axes<real, DIM, K>(T.PW, T.PW, T.DW, w, u);
#pragma unroll
      for (int q = 0; q < Q; ++q) sG[((2 * NV + v) * Q + q) * TC + tc] = u[q];
    }
  }
  __syncthreads();
  const real g1 = real(a.gamma) - real(1);
  for (int q = v; q < Q; q += NV) {
    real u[NV], g[DIM][NV], b[NV];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) {
      u[vv] = sU[(vv * Q + q) * TC + tc];
#pragma unroll
      for (int d = 0; d < DIM; ++d) g[d][vv] = sG[((d * NV + vv) * Q + q) * TC + tc];
    }
    flux_vjp<real, DIM>(u, g, g1, b);
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) sB[(vv * Q + q) * TC + tc] = b[vv];
  }
  __syncthreads();
  if (!valid) return;
  real acc[N];
#pragma unroll
  for (int l = 0; l < N; ++l) acc[l] = real(0);
  {
    real b[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) b[q] = sB[(v * Q + q) * TC + tc];
    nodal_to_modal<real, DIM, K>(T.P, b, acc);
  }
  const unsigned coarse = a.m.scoarse[c];
  gather_face_adjoint<real, DIM, K, 0>(a, c, v, coarse, acc);
  gather_face_adjoint<real, DIM, K, 1>(a, c, v, coarse, acc);
  gather_face_adjoint<real, DIM, K, 2>(a, c, v, coarse, acc);
  gather_face_adjoint<real, DIM, K, 3>(a, c, v, coarse, acc);
  if constexpr (DIM == 3) {
    gather_face_adjoint<real, DIM, K, 2 * DIM - 2>(a, c, v, coarse, acc);
    gather_face_adjoint<real, DIM, K, 2 * DIM - 1>(a, c, v, coarse, acc);
  }
  const real sc = real(a.scale);
#pragma unroll
  for (int l = 0; l < N; ++l) a.acc[(size_t)(v * N + l) * nc + c] = sc * acc[l];
}

template <typename real, int DIM, int K>
cudaError_t prepare_adjoint_kernels() {
  cudaError_t e = cudaFuncSetAttribute(adjoint_cell_kernel<real, DIM, K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)AdjCellTile<real, DIM, K>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(adjoint_face_kernel<real, DIM, K>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)AdjFaceTile<real, DIM, K>::SMEM);
}

template <typename real, int DIM, int K>
cudaError_t launch_adj_face(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const AdjointArgs<real>*>(pa);
  using FT = AdjFaceTile<real, DIM, K>;
  if (a.m.nfaces == 0) return cudaSuccess;
  adjoint_face_kernel<real, DIM, K><<<(a.m.nfaces + FT::FB - 1) / FT::FB, FT::THREADS, FT::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <typename real, int DIM, int K>
cudaError_t launch_adj_cell(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const AdjointArgs<real>*>(pa);
  using CT = AdjCellTile<real, DIM, K>;
  if (a.m.ncells == 0) return cudaSuccess;
  adjoint_cell_kernel<real, DIM, K><<<(a.m.ncells + CT::TC - 1) / CT::TC, CT::THREADS, CT::SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dgi
