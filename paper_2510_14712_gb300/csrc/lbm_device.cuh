// lbm_device.cuh - per-node arithmetic of the non-ideal compressible LBM
// (Hosseini, Feinberg & Karlin, Sec. 3.2), shared by every kernel of the
// library.  Templated on the dimension D (2: D2Q9, 3: D3Q27) and on the
// arithmetic type `real` (double for the FP64 build, float otherwise).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm.h"

namespace lbm {

// Velocity i <-> (c_x, c_y[, c_z]) in {-1,0,1}^D, lexicographic with the last
// component fastest (Eq. D3Q27c): i = 9 (cx+1) + 3 (cy+1) + (cz+1) in 3-D and
// i = 3 (cx+1) + (cy+1) in 2-D.
template <int D> struct Lattice;
template <> struct Lattice<2> {
  static constexpr int Q = 9;
  __host__ __device__ static constexpr int c(int i, int a) {
    return a == 0 ? i / 3 - 1 : i % 3 - 1;
  }
};
template <> struct Lattice<3> {
  static constexpr int Q = 27;
  __host__ __device__ static constexpr int c(int i, int a) {
    return a == 0 ? i / 9 - 1 : (a == 1 ? (i / 3) % 3 - 1 : i % 3 - 1);
  }
};

// sum_i c_ia f_i (Eq. def_u) as a sum over mirror pairs: each direction with
// c_ia = +1 minus its mirror image in axis a.  Exactly zero for
// mirror-symmetric populations, so that a fluid at rest has u = 0 exactly and
// the upwind stencil takes its sgn(0) branch as in exact arithmetic.
template <int D, typename real> __device__ __forceinline__ void first_moment(const real* f, real* j) {
  using L = Lattice<D>;
  constexpr int stride0 = D == 3 ? 9 : 3, stride1 = D == 3 ? 3 : 1, stride2 = 1;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int st = a == 0 ? stride0 : (a == 1 ? stride1 : stride2);
    real acc = real(0);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      if (L::c(i, a) == 1) acc += f[i] - f[i - 2 * st];
    j[a] = acc;
  }
}

// Model constants in the arithmetic type.
template <typename real> struct Model {
  real a, b, R, cv;          // van der Waals (Eq. Pvdw) or Peng-Robinson constants, c_v (ideal part)
  real kappa;                // Korteweg capillarity (Eq. FK)
  real eta_over_mu;          // bulk / shear viscosity (Eq. corr_bulk)
  real mu;                   // shear viscosity (constant, Sec. 2)
  real k_over_mu;            // thermal conductivity / mu (Eq. qc)
  int kind;                  // LBM_EOS_VDW or LBM_EOS_PR
  real Tc, mpr;              // Peng-Robinson: T_c and the slope m of sqrt(alpha) in sqrt(T/T_c)
};

// The FP64 temperature inversion of Eq. lbm_temp used by the FP32 kernels when
// it is switched on (lbm_set_temperature_fp64): T = (E - |u|^2/2 + a rho) / c_v
// evaluated in FP64 from the FP32 moments, rounded once to FP32.  Returns T;
// e = E - |u|^2/2 (the specific internal energy) is rounded into `e`.  Most of
// FP32's error in T comes from E - |u|^2/2, so the subtraction is the part
// that needs the wider type, not only the division.
__host__ __device__ inline float vdw_temperature_fp64(double a, double inv_cv, float rho, float E, float u2, float& e) {
  const double ed = double(E) - 0.5 * double(u2);
  e = float(ed);
  return float((ed + a * double(rho)) * inv_cv);
}

// a / b correctly rounded, also in the FP32 kernel sets built with the
// reciprocal-based FP32 division (-prec-div=false): for the divisions of the
// moments by rho (Eqs. def_u, def_E), whose rounding the step amplifies most
// (the velocity by reciprocal doubles the FP32 error of u over 1000 steps of
// a Taylor-Green box in the oracle evaluated in float32)
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return a / b; }

template <typename real> __host__ __device__ inline real vdw_pressure(const Model<real>& m, real rho, real T) {
  return rho * m.R * T / (real(1) - m.b * rho) - m.a * rho * rho;          // Eq. Pvdw
}
template <typename real> __host__ __device__ inline real vdw_energy(const Model<real>& m, real rho, real T) {
  return m.cv * T - m.a * rho;                                             // Eq. de_vdW, integrated
}
template <typename real> __host__ __device__ inline real vdw_cs2(const Model<real>& m, real rho, real T) {
  const real s = real(1) / (real(1) - m.b * rho);
  return m.R * T * (real(1) + m.R / m.cv) * s * s - real(2) * m.a * rho;   // Eq. vdW_speed_of_sound
}

// ---- Peng-Robinson fluid (a general equation of state, Sec. 2) ----
//   P = rho R T / (1 - b rho) - a alpha(T) rho^2 / D(rho),  D = 1 + 2 b rho - b^2 rho^2,
//   alpha = s^2,  s = 1 + m (1 - sqrt(T / T_c)),
// with the caloric relation of the identity e = c_v T + int_0^rho (P - T dP/dT) / rho'^2:
//   e = c_v T + (T a alpha' - a alpha) L(rho) / (2 sqrt2 b),  L = ln((1 + (1+sqrt2) b rho) / (1 + (1-sqrt2) b rho)).
// Since T alpha' - alpha = -(1 + m) s, e = c_v T + A sqrt(T) + B0 with
//   A = a c (1 + m) m / sqrt(T_c),  B0 = -a c (1 + m)^2,  c = L / (2 sqrt2 b):
// a quadratic in sqrt(T), inverted below in closed form.
template <typename real> __host__ __device__ inline real pr_c(const Model<real>& m, real rho) {
  const real r2 = real(1.4142135623730951);
  return log((real(1) + (real(1) + r2) * m.b * rho) / (real(1) + (real(1) - r2) * m.b * rho)) / (real(2) * r2 * m.b);
}
template <typename real> __host__ __device__ inline real pr_s(const Model<real>& m, real T) {
  return real(1) + m.mpr * (real(1) - sqrt(T / m.Tc));
}
template <typename real> __host__ __device__ inline real pr_pressure(const Model<real>& m, real rho, real T) {
  const real s = pr_s(m, T), D = real(1) + real(2) * m.b * rho - m.b * m.b * rho * rho;
  return rho * m.R * T / (real(1) - m.b * rho) - m.a * s * s * rho * rho / D;
}
template <typename real> __host__ __device__ inline real pr_energy(const Model<real>& m, real rho, real T) {
  return m.cv * T - m.a * pr_c(m, rho) * (real(1) + m.mpr) * pr_s(m, T);
}
// (dP/dT)_rho, (dP/drho)_T, c_v(rho, T) and Eq. speed_of_sound
template <typename real> __host__ __device__ inline real pr_dPdT(const Model<real>& m, real rho, real T) {
  const real s = pr_s(m, T), D = real(1) + real(2) * m.b * rho - m.b * m.b * rho * rho;
  const real dal = -m.mpr * s / sqrt(T * m.Tc);
  return rho * m.R / (real(1) - m.b * rho) - m.a * dal * rho * rho / D;
}
template <typename real> __host__ __device__ inline real pr_cv(const Model<real>& m, real rho, real T) {
  const real s = pr_s(m, T);
  const real d2al = real(0.5) * m.mpr / T * (m.mpr / m.Tc + s / sqrt(T * m.Tc));
  return m.cv + T * m.a * d2al * pr_c(m, rho);
}
template <typename real> __host__ __device__ inline real pr_cs2(const Model<real>& m, real rho, real T) {
  const real s = pr_s(m, T), D = real(1) + real(2) * m.b * rho - m.b * m.b * rho * rho;
  const real x = real(1) - m.b * rho;
  const real dPdr = m.R * T / (x * x) - m.a * s * s * real(2) * rho * (real(1) + m.b * rho) / (D * D);
  const real dPdT = pr_dPdT(m, rho, T);
  return dPdr + T * dPdT * dPdT / (rho * rho * pr_cv(m, rho, T));
}
// T from (rho, e): the positive root of c_v y^2 + A y + (B0 - e) = 0, y = sqrt(T), in
// the form without cancellation, y = 2 (e - B0) / (A + sqrt(A^2 + 4 c_v (e - B0))): every
// term is positive, so the arithmetic precision of the kernel (FP32 or FP64) gives T to
// a few of its ulps
template <typename real> __host__ __device__ inline real pr_temperature(const Model<real>& m, real rho, real e) {
  const real c = pr_c(m, rho), k = m.mpr;
  const real A = m.a * c * (real(1) + k) * k / sqrt(m.Tc), B0 = -m.a * c * (real(1) + k) * (real(1) + k);
  const real q = e - B0;
  const real y = real(2) * q / (A + sqrt(A * A + real(4) * m.cv * q));
  return y * y;
}
// The same root with e given in FP64 (the FP64 temperature inversion of the
// FP32 kernels): q = e - B0 is formed in FP64 and rounded once; the root of
// positive terms is then evaluated in FP32.
__host__ __device__ inline float pr_temperature_q(const Model<float>& m, float rho, double e) {
  const float c = pr_c(m, rho), k = m.mpr;
  const float A = m.a * c * (1.0f + k) * k / sqrtf(m.Tc), B0 = -m.a * c * (1.0f + k) * (1.0f + k);
  const float q = float(e - double(B0));
  const float y = 2.0f * q / (A + sqrtf(A * A + 4.0f * m.cv * q));
  return y * y;
}
__host__ __device__ inline double pr_temperature_q(const Model<double>& m, double rho, double e) {
  return pr_temperature(m, rho, e);
}

// ---- the fluid of a handle (Model::kind): van der Waals or Peng-Robinson ----
template <typename real> __host__ __device__ inline real eos_pressure(const Model<real>& m, real rho, real T) {
  return m.kind == LBM_EOS_PR ? pr_pressure(m, rho, T) : vdw_pressure(m, rho, T);
}
template <typename real> __host__ __device__ inline real eos_energy(const Model<real>& m, real rho, real T) {
  return m.kind == LBM_EOS_PR ? pr_energy(m, rho, T) : vdw_energy(m, rho, T);
}
template <typename real> __host__ __device__ inline real eos_cs2(const Model<real>& m, real rho, real T) {
  return m.kind == LBM_EOS_PR ? pr_cs2(m, rho, T) : vdw_cs2(m, rho, T);
}
// T from rho and the specific internal energy e (Eq. lbm_temp for van der Waals)
template <typename real> __host__ __device__ inline real eos_temperature(const Model<real>& m, real rho, real e) {
  return m.kind == LBM_EOS_PR ? pr_temperature(m, rho, e) : (e + m.a * rho) / m.cv;
}
// the coefficients of grad s = c_T grad T - c_rho grad rho: c_v(rho, T)/T and (dP/dT)_rho / rho^2
template <typename real>
__host__ __device__ inline void eos_entropy_coefs(const Model<real>& m, real rho, real T, real& cT, real& cR) {
  if (m.kind == LBM_EOS_PR) {
    cT = pr_cv(m, rho, T) / T;
    cR = pr_dPdT(m, rho, T) / (rho * rho);
  } else {
    cR = m.R / (rho * (real(1) - m.b * rho));
    cT = m.cv / T;
  }
}

// Eq. phi: Psi(c; xi, zeta) = 1 - zeta (c = 0), (zeta + c xi)/2 (c = +-1).
// The three values for c = -1, 0, +1 of one axis.
template <typename real> struct Axis3 {
  real v[3];
  __host__ __device__ real operator[](int c) const { return v[c + 1]; }
};
template <typename real> __host__ __device__ inline Axis3<real> psi3(real xi, real zeta) {
  Axis3<real> t;
  t.v[0] = real(0.5) * (zeta - xi);
  t.v[1] = real(1) - zeta;
  t.v[2] = real(0.5) * (zeta + xi);
  return t;
}
// Psi(O, O^2) with O = theta d/du + u (Eq. Oa) applied to u^2/2, the part of
// the generating function E = e + u^2/2 (Eq. Egen) that depends on u_a:
//   O(u^2/2)   = theta u + u^3/2                   =: A
//   O^2(u^2/2) = theta^2 + 5/2 theta u^2 + u^4/2   =: B
//   factor     = u^2/2 - B (c = 0),  (B + c A)/2 (c = +-1).
template <typename real> __host__ __device__ inline Axis3<real> chi3(real u, real theta) {
  const real u2 = u * u;
  const real A = u * (theta + real(0.5) * u2);
  const real B = theta * theta + u2 * (real(2.5) * theta + real(0.5) * u2);
  Axis3<real> t;
  t.v[0] = real(0.5) * (B - A);
  t.v[1] = real(0.5) * u2 - B;
  t.v[2] = real(0.5) * (B + A);
  return t;
}

// Equilibria at one state for all i (Fig. FlowChart, "Initialize"):
// f^eq = rho prod_a Psi(c_ia; u_a, theta + u_a^2)                          (Eq. LBMeq)
// g^eq = rho [ e prod_a psi_a + sum_b chi_b prod_{a != b} psi_a ]         (Eq. LBMeqG)
template <int D, typename real>
__host__ __device__ inline void equilibria(const Model<real>& m, real rho, const real* u, real T, real* feq, real* geq) {
  using L = Lattice<D>;
  const real P = eos_pressure(m, rho, T);
  const real theta = P / rho;
  const real e = eos_energy(m, rho, T);
  Axis3<real> ps[D], ch[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    ps[a] = psi3(u[a], theta + u[a] * u[a]);
    ch[a] = chi3(u[a], theta);
  }
  // unrolled: table indices are compile-time, the tables stay in registers
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    real prod = real(1);
#pragma unroll
    for (int a = 0; a < D; ++a) prod *= ps[a][L::c(i, a)];
    real acc = e * prod;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      real t = ch[b][L::c(i, b)];
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a != b) t *= ps[a][L::c(i, a)];
      acc += t;
    }
    feq[i] = rho * prod;
    geq[i] = rho * acc;
  }
}

// Fields of one node needed by its neighbours' stencils.
template <int D, typename real> struct NodeFields {
  real u[D], T, h, Lam[D];
};

// Inputs of the collision at one node besides the populations.  T, P, c_s^2
// come from the thermodynamic closure of the node (exact vdW or learned) and
// e is the specific internal energy.
template <int D, typename real> struct NodeState {
  real rho, u[D], F[D], T, P, cs2, e;
  // shock capturing (Sec. 4.4): numerical mu, eta, k added to the constant ones
  bool sc;
  real mu_num, eta_num, k_num;
  real div_u;            // central divergence of u
  real gradT[D], gradh[D];
  real dLam[D];          // upwind derivative of Lambda_a along a (Sec. 3.2)
};

enum : unsigned { FLAG_NONFINITE = 1u, FLAG_NEGATIVE = 2u, FLAG_THETA = 4u, FLAG_PRESSURE = 8u };

// The attractors and relaxation factors of one node (Eqs. LBMeq, LBMstar,
// LBMeqG, LBMgstar, beta_main), as per-axis tables, so that each population
// can be relaxed on its own (Eqs. fLBGK, gLBGK): the kernels stream the f and
// the g populations through one direction at a time.
template <int D, typename real> struct Attractors {
  real rho, e, e_s, twobeta, omb;
  real qc[D];
  Axis3<real> pe[D], pf[D], pg[D], ce[D], cg[D];
  unsigned flags;

  __device__ __forceinline__ void setup(const Model<real>& m, const NodeState<D, real>& s) {
    rho = s.rho;
    const real T = s.T;
    const real inv_rho = real(1) / rho;
    const real P = s.P;
    const real theta = P * inv_rho;                                        // Eq. theta
    e = s.e;
    const real cs2 = s.cs2;
    real eta_over_mu = m.eta_over_mu, mu = m.mu, k_over_mu = m.k_over_mu;
    if (s.sc) {                                                            // {mu, eta, k} + {..}^num
      const real mu_e = m.mu + s.mu_num;
      eta_over_mu = (m.eta_over_mu * m.mu + s.eta_num) / mu_e;
      k_over_mu = (m.k_over_mu * m.mu + s.k_num) / mu_e;
      mu = mu_e;
    }
    const real alpha = real(D + 2) / real(D) - rho * cs2 / P - eta_over_mu;     // Eq. corr_bulk
    const real tau = mu / P;                                               // tau = mu / P
    const real beta = real(1) / (real(2) * tau + real(1));                 // Eq. beta_main
    twobeta = real(2) * beta;
    omb = real(1) - beta;
    // shifted state (Eqs. sh_vel_1, sh_temp_1, sh_T_1, qc_1; delta t = 1)
    real us[D], FF = real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      us[a] = s.u[a] + s.F[a] * inv_rho;
      FF += s.F[a] * s.F[a];
    }
    const real theta_s = theta + alpha * theta * s.div_u;
    // T* = T - |F|^2 / (2 rho^2 c_v): with e linear in T at fixed rho this is
    // e* = e - |F|^2 / (2 rho^2)
    e_s = e - FF * real(0.5) * inv_rho * inv_rho;
#pragma unroll
    for (int a = 0; a < D; ++a) qc[a] = P * (s.gradh[a] - k_over_mu * s.gradT[a]);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const real Phi = -s.dLam[a] * inv_rho;                               // Eq. correction
      pe[a] = psi3(s.u[a], theta + s.u[a] * s.u[a]);                       // Eqs. def_xi_eq, def_zeta_eq
      pf[a] = psi3(us[a], theta_s + us[a] * us[a] + Phi);                  // Eqs. xistar, zetastar
      pg[a] = psi3(us[a], theta_s + us[a] * us[a]);                        // g*: no Phi
      ce[a] = chi3(s.u[a], theta);
      cg[a] = chi3(us[a], theta_s);
    }
    flags = 0;
    if (!(isfinite(rho) && isfinite(T))) flags |= FLAG_NONFINITE;
    if (!(rho > real(0)) || !(T > real(0))) flags |= FLAG_NEGATIVE;
    if (theta >= real(1.0 / 3.0)) flags |= FLAG_THETA;
    if (!(P > real(0))) flags |= FLAG_PRESSURE;
  }

  // f_i + 2 beta (f_i^eq - f_i) + (1 - beta)(f_i^* - f_i^eq)      (Eq. fLBGK)
  // (I is a compile-time constant after loop unrolling)
  __device__ __forceinline__ real relax_f(int I, real f) const {
    using L = Lattice<D>;
    real fe = rho, fs = rho;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      fe *= pe[a][L::c(I, a)];
      fs *= pf[a][L::c(I, a)];
    }
    return relax(f, fe, fs - fe);
  }

  // p + 2 beta (p^eq - p) + (1 - beta) d, d = p^* - p^eq: the form of Eqs.
  // fLBGK / gLBGK whose terms are differences of nearly equal populations, so
  // that each rounding is relative to a small quantity (expanding it into
  // (1 - 2 beta) p + (3 beta - 1) p^eq + (1 - beta) p^* rounds three terms of
  // the size of p and, near beta = 1, cancels two of them)
  __device__ __forceinline__ real relax(real p, real pe_, real d) const {
    return fma(omb, d, fma(twobeta, pe_ - p, p));
  }

  // g_i + 2 beta (g_i^eq - g_i) + (1 - beta)(g_i^* - g_i^eq)      (Eq. gLBGK)
  __device__ __forceinline__ real relax_g(int I, real g) const {
    using L = Lattice<D>;
    real ge = e, gs = e_s, pe_all = real(1), pg_all = real(1);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      pe_all *= pe[a][L::c(I, a)];
      pg_all *= pg[a][L::c(I, a)];
    }
    ge *= pe_all;
    gs *= pg_all;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      real te = ce[b][L::c(I, b)], tg = cg[b][L::c(I, b)];
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a != b) {
          te *= pe[a][L::c(I, a)];
          tg *= pg[a][L::c(I, a)];
        }
      ge += te;
      gs += tg;
    }
    ge *= rho;
    gs *= rho;
    int nz = 0;
    real cq = real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      nz += L::c(I, a) != 0;
      cq += real(L::c(I, a)) * qc[a];
    }
    if (nz == 1) gs += real(0.5) * cq;                                     // Eq. LBMgstar, |c_i|^2 = 1
    return relax(g, ge, gs - ge);
  }
};

// Relaxation of all Q populations of one kind with products shared between
// directions.  Directions are grouped by their components on the first D-1
// axes ("lower" axes: x, and y in 3-D); for each group the products over the
// lower axes are formed once and the three directions of the group differ
// only in the factor of the last axis.  The update of Eqs. fLBGK / gLBGK is
// Attractors::relax of p, p^eq and p^* - p^eq.
// load(i) / store(i, v) move population i.
template <int D, typename real> struct FactoredRelax {
  using L = Lattice<D>;
  static constexpr int NG = D == 3 ? 9 : 3;          // groups of lower-axis components

  template <class Load, class Store>
  __device__ __forceinline__ static void f_pass(const Attractors<D, real>& at, Load load, Store store) {
#pragma unroll
    for (int gi = 0; gi < NG; ++gi) {
      const int cx = D == 3 ? gi / 3 - 1 : gi - 1;
      const int cy = D == 3 ? gi % 3 - 1 : 0;
      real fe2 = at.rho * at.pe[0][cx], fs2 = at.rho * at.pf[0][cx];
      if (D == 3) {
        fe2 *= at.pe[1][cy];
        fs2 *= at.pf[1][cy];
      }
#pragma unroll
      for (int cl = -1; cl <= 1; ++cl) {
        const int i = 3 * gi + cl + 1;
        const real fe = fe2 * at.pe[D - 1][cl];
        const real d = fma(fs2, at.pf[D - 1][cl], -fe);                   // f^* - f^eq, one rounding
        const real f = load(i);
        store(i, at.relax(f, fe, d));
      }
    }
  }

  template <class Load, class Store>
  __device__ __forceinline__ static void g_pass(const Attractors<D, real>& at, Load load, Store store) {
#pragma unroll
    for (int gi = 0; gi < NG; ++gi) {
      const int cx = D == 3 ? gi / 3 - 1 : gi - 1;
      const int cy = D == 3 ? gi % 3 - 1 : 0;
      // A = prod_lower psi, B = sum_b chi_b prod_{lower, a != b} psi, C = e A + B
      real Ae = at.pe[0][cx], Be = at.ce[0][cx], As = at.pg[0][cx], Bs = at.cg[0][cx];
      if (D == 3) {
        Be = Be * at.pe[1][cy] + Ae * at.ce[1][cy];
        Ae = Ae * at.pe[1][cy];
        Bs = Bs * at.pg[1][cy] + As * at.cg[1][cy];
        As = As * at.pg[1][cy];
      }
      const real Ce = at.rho * (at.e * Ae + Be), Cs = at.rho * (at.e_s * As + Bs);
      Ae *= at.rho;
      As *= at.rho;
      const int nzl = (cx != 0) + (D == 3 ? (cy != 0) : 0);
#pragma unroll
      for (int cl = -1; cl <= 1; ++cl) {
        const int i = 3 * gi + cl + 1;
        const real ge = at.pe[D - 1][cl] * Ce + Ae * at.ce[D - 1][cl];      // Eq. LBMeqG
        // g^* - g^eq (Eq. LBMgstar) with g^* accumulated onto -g^eq
        real d = fma(at.pg[D - 1][cl], Cs, fma(As, at.cg[D - 1][cl], -ge));
        if (nzl + (cl != 0) == 1) {                                          // |c_i|^2 = 1
          const real cq = cl != 0 ? real(cl) * at.qc[D - 1]
                                  : (cx != 0 ? real(cx) * at.qc[0] : real(cy) * at.qc[D == 3 ? 1 : 0]);
          d += real(0.5) * cq;
        }
        const real g = load(i);
        store(i, at.relax(g, ge, d));
      }
    }
  }
};

// The collision of Eqs. fLBGK / gLBGK at one node.  f, g: the 2Q pulled
// (post-streaming) populations in, post-collision populations out.
// Returns the status bits of this node.
template <int D, typename real>
__device__ __forceinline__ unsigned collide_node(const Model<real>& m, const NodeState<D, real>& s, real* f, real* g) {
  Attractors<D, real> at;
  at.setup(m, s);
#pragma unroll
  for (int i = 0; i < Lattice<D>::Q; ++i) {
    f[i] = at.relax_f(i, f[i]);
    g[i] = at.relax_g(i, g[i]);
  }
  return at.flags;
}

}  // namespace lbm
