// lbm_fused.cuh - the fused single-pass time step.
//
// One kernel does, for every interior node, everything of Sec. 3.2 between
// reading the post-collision populations of the last step and writing the
// new ones: pull-stream, moments (Eqs. def_h, def_u, def_E), Korteweg force
// (Eq. FK), EOS and temperature (Eqs. Pvdw, lbm_temp), neighbour derivatives
// (central; upwind for Phi), shifted state, attractors and collision (Eqs.
// fLBGK, gLBGK).  The ghost layers of non-periodic x faces are refilled by
// the separate k_ghosts kernel afterwards.
//
// Decomposition.  The last axis ("march" axis m: z in 3-D, y in 2-D) is
// periodic.  The other axes are cut into column tiles of TX x TY nodes; a
// CTA walks along m through a contiguous range of (column, plane) work items
// (persistent grid, one range per CTA, equal sizes).  Per plane p it
//   A. pulls f on the radius-3 L1 neighbourhood of the tile (R3) -> rho(p),
//      and f, g on radius 1 (R1) -> j(p), S(p)              [ring of 3 planes]
//   B. Laplacian of rho of plane p-1 on R2                  [ring of 3 planes]
//   C. F, u, E, T, P, theta, h, Lambda of plane p-2 on R1   [ring of 3 planes]
//   D. derivatives and collision of plane p-3 on the tile, pulling its 2Q
//      populations again (they were read three planes earlier: L2 hits).
// The 3-plane lag is the z-extent of the dependency cone: the collision at z
// needs u at z+-1, which needs F at z+-1, which needs lap rho at z+-2, which
// needs rho at z+-3.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

template <int D, int TX, int TY> struct FusedGeom {
  static constexpr int NT = TX * TY;                 // threads per CTA
  static constexpr int HY3 = D == 3 ? 3 : 0, HY2 = D == 3 ? 2 : 0, HY1 = D == 3 ? 1 : 0;
  static constexpr int BX3 = TX + 6, BY3 = TY + 2 * HY3, N3 = BX3 * BY3;
  static constexpr int BX2 = TX + 4, BY2 = TY + 2 * HY2, N2 = BX2 * BY2;
  static constexpr int BX1 = TX + 2, BY1 = TY + 2 * HY1, N1 = BX1 * BY1;
  static constexpr int NMOM = D + 1;                 // j_0..j_{D-1}, S
  static constexpr int NPRIM = 3 * D + 4;            // rho, u[D], T, h, Lam[D], F[D]
  static constexpr int P_RHO = 0, P_U = 1, P_T = 1 + D, P_H = 2 + D, P_LAM = 3 + D, P_F = 3 + 2 * D;
  template <typename real> static constexpr size_t smem_bytes() {
    return sizeof(real) * size_t(3 * N3 + 3 * NMOM * N1 + 3 * N2 + 3 * NPRIM * N1);
  }
};

// v mod n in [0, n) for any integer v
__device__ __forceinline__ int modp(int v, int n) {
  const int r = v % n;
  return r < 0 ? r + n : r;
}

// distance outside the tile along one in-plane axis (0 inside)
__device__ __forceinline__ int outside(int l, int h, int T) {
  const int v = l - h;
  return v < 0 ? -v : (v >= T ? v - T + 1 : 0);
}

// MINB: CTAs per SM the register allocation must allow (2 keeps one CTA's
// memory phase overlapping the other's collision)
template <int D, typename S, typename real, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB)
k_step_fused(Params p, const typename Store<S>::T* __restrict__ A, typename Store<S>::T* __restrict__ B,
             unsigned* err, int ncolx, int ncoly, int nseg) {
  using L = Lattice<D>;
  using G = FusedGeom<D, TX, TY>;
  constexpr int Q = L::Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* s_rho = reinterpret_cast<real*>(smem_raw);            // [3][N3]
  real* s_mom = s_rho + 3 * G::N3;                            // [3][NMOM][N1]
  real* s_lap = s_mom + 3 * G::NMOM * G::N1;                  // [3][N2]
  real* s_prm = s_lap + 3 * G::N2;                            // [3][NPRIM][N1]

  const Model<real> m = model_of<real>(p);
  const int tid = threadIdx.x;
  const int Nm = D == 3 ? p.Nz : p.Ny;                        // march extent
  const int Ny_in = D == 3 ? p.Ny : 1;                        // in-plane y extent
  const long long mstride = D == 3 ? (long long)p.Ny * p.pitch : (long long)p.pitch;
  const int xmin = p.periodic_x ? -0x40000000 : -3, xmax = p.periodic_x ? 0x40000000 : p.Nx + 2;
  unsigned flags = 0;

  // Work items are (column, z-segment) pairs, ordered segment-major so that
  // the CTAs resident together cover neighbouring columns at the same planes
  // and their halos are L2 hits.  nseg segments split the march axis.
  const int ncol = ncolx * ncoly;
  const long long nitems = (long long)ncol * nseg;
  for (long long it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int col = int(it % ncol);
    const int seg = int(it / ncol);
    const int mb = int((long long)Nm * seg / nseg), me = int((long long)Nm * (seg + 1) / nseg);
    const int x0 = (col % ncolx) * TX;
    const int y0 = D == 3 ? (col / ncolx) * TY : 0;

    for (int pl = mb - 3; pl <= me + 2; ++pl) {
      // ---------------- A: moments of plane pl --------------------------------
      {
        const int slot = (pl + 6) % 3;
        const int mp = modp(pl, Nm);
        long long mo[3];                                      // source plane offsets, c_m = -1, 0, +1
#pragma unroll
        for (int c = -1; c <= 1; ++c) mo[c + 1] = (long long)wrap(mp - c, Nm) * mstride;
        for (int k = tid; k < G::N3; k += G::NT) {
          const int lx = k % G::BX3, ly = k / G::BX3;
          const int ox = outside(lx, 3, TX), oy = D == 3 ? outside(ly, G::HY3, TY) : 0;
          if (ox + oy > 3) continue;
          int gx = x0 + lx - 3;
          if (gx < xmin || gx > xmax) continue;
          const int gy = modp(y0 + ly - G::HY3, Ny_in);
          const bool r1 = ox + oy <= 1;
          long long xo[3], yo[3];
#pragma unroll
          for (int c = -1; c <= 1; ++c) {
            xo[c + 1] = p.periodic_x ? modp(gx - c, p.Nx) : gx + p.G - c;
            yo[c + 1] = D == 3 ? (long long)modp(gy - c, Ny_in) * p.pitch : 0;
          }
          real f[Q];
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const int cx = L::c(i, 0), cy = D == 3 ? L::c(i, 1) : 0, cm = L::c(i, D - 1);
            f[i] = Store<S>::template ld<real>(A, i * p.plane + mo[cm + 1] + yo[cy + 1] + xo[cx + 1], p.ref[i]);
          }
          real rho = 0;
#pragma unroll
          for (int i = 0; i < Q; ++i) rho += f[i];
          s_rho[slot * G::N3 + k] = rho;
          if (r1) {
            const int k1 = (ly - (G::HY3 - G::HY1)) * G::BX1 + (lx - 2);
            real j[D];
            first_moment<D, real>(f, j);
            real Se = 0;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
              const int cx = L::c(i, 0), cy = D == 3 ? L::c(i, 1) : 0, cm = L::c(i, D - 1);
              Se += Store<S>::template ld<real>(A, (Q + i) * p.plane + mo[cm + 1] + yo[cy + 1] + xo[cx + 1],
                                                p.ref[Q + i]);
            }
            real* dst = s_mom + (slot * G::NMOM) * G::N1 + k1;
#pragma unroll
            for (int a = 0; a < D; ++a) dst[a * G::N1] = j[a];
            dst[D * G::N1] = Se;
          }
        }
      }
      __syncthreads();

      // ---------------- B: Laplacian of rho, plane pl-1, on R2 ------------------
      if (pl - 1 >= mb - 2) {
        const int q = pl - 1;
        const int sc = (q + 6) % 3, sm = (q + 5) % 3, sp = (q + 7) % 3;
        for (int k = tid; k < G::N2; k += G::NT) {
          const int lx = k % G::BX2, ly = k / G::BX2;
          const int ox = outside(lx, 2, TX), oy = D == 3 ? outside(ly, G::HY2, TY) : 0;
          if (ox + oy > 2) continue;
          const int gx = x0 + lx - 2;
          if (gx < xmin + 1 || gx > xmax - 1) continue;
          const int k3 = (ly + (G::HY3 - G::HY2)) * G::BX3 + (lx + 1);
          const real* r = s_rho + sc * G::N3;
          const real c2 = real(2) * r[k3];
          real lap = (r[k3 + 1] + r[k3 - 1] - c2) + (s_rho[sp * G::N3 + k3] + s_rho[sm * G::N3 + k3] - c2);
          if (D == 3) lap += r[k3 + G::BX3] + r[k3 - G::BX3] - c2;
          s_lap[sc * G::N2 + k] = lap;
        }
      }
      __syncthreads();

      // ---------------- C: primitive fields, plane pl-2, on R1 ------------------
      if (pl - 2 >= mb - 1) {
        const int q = pl - 2;
        const int sc = (q + 6) % 3, sm = (q + 5) % 3, sp = (q + 7) % 3;
        for (int k = tid; k < G::N1; k += G::NT) {
          const int lx = k % G::BX1, ly = k / G::BX1;
          const int ox = outside(lx, 1, TX), oy = D == 3 ? outside(ly, G::HY1, TY) : 0;
          if (ox + oy > 1) continue;
          const int gx = x0 + lx - 1;
          if (gx < xmin + 2 || gx > xmax - 2) continue;
          const int k3 = (ly + (G::HY3 - G::HY1)) * G::BX3 + (lx + 2);
          const int k2 = (ly + (G::HY2 - G::HY1)) * G::BX2 + (lx + 1);
          const real rho = s_rho[sc * G::N3 + k3];
          const real* lp = s_lap + sc * G::N2;
          real F[D];
          F[0] = m.kappa * rho * real(0.5) * (lp[k2 + 1] - lp[k2 - 1]);                         // Eq. FK
          if (D == 3) F[1] = m.kappa * rho * real(0.5) * (lp[k2 + G::BX2] - lp[k2 - G::BX2]);
          F[D - 1] = m.kappa * rho * real(0.5) * (s_lap[sp * G::N2 + k2] - s_lap[sm * G::N2 + k2]);
          const real* mo = s_mom + (sc * G::NMOM) * G::N1 + k;
          real u[D], uF = 0, u2 = 0;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            u[a] = (mo[a * G::N1] + real(0.5) * F[a]) / rho;                                     // Eq. def_u
            uF += u[a] * F[a];
            u2 += u[a] * u[a];
          }
          const real E = (mo[D * G::N1] + real(0.5) * uF) / rho;                                // Eq. def_E
          const real T = (E - real(0.5) * u2 + m.a * rho) / m.cv;                                 // Eq. lbm_temp
          const real P = vdw_pressure(m, rho, T);
          const real theta = P / rho;
          real* pr = s_prm + (sc * G::NPRIM) * G::N1 + k;
          pr[G::P_RHO * G::N1] = rho;
          pr[G::P_T * G::N1] = T;
          pr[G::P_H * G::N1] = vdw_energy(m, rho, T) + theta;                                   // Eq. enthalpy
#pragma unroll
          for (int a = 0; a < D; ++a) {
            pr[(G::P_U + a) * G::N1] = u[a];
            pr[(G::P_LAM + a) * G::N1] = rho * u[a] * u[a] * u[a] + real(3) * rho * u[a] * (theta - real(1.0 / 3.0));
            pr[(G::P_F + a) * G::N1] = F[a];
          }
        }
      }
      __syncthreads();

      // ---------------- D: collide plane pl-3 on the tile --------------------------
      if (pl - 3 >= mb) {
        const int q = pl - 3;
        const int sc = (q + 6) % 3, sm = (q + 5) % 3, sp = (q + 7) % 3;
        const int lx = tid % TX, ly = tid / TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx < p.Nx && (D == 2 || gy < p.Ny)) {
          const int mq = modp(q, Nm);
          long long mo[3], xo[3], yo[3];
#pragma unroll
          for (int c = -1; c <= 1; ++c) {
            mo[c + 1] = (long long)wrap(mq - c, Nm) * mstride;
            xo[c + 1] = p.periodic_x ? modp(gx - c, p.Nx) : gx + p.G - c;
            yo[c + 1] = D == 3 ? (long long)modp(gy - c, p.Ny) * p.pitch : 0;
          }
          const int k1 = (ly + G::HY1) * G::BX1 + (lx + 1);
          const real* pc = s_prm + (sc * G::NPRIM) * G::N1;
          const real* pm = s_prm + (sm * G::NPRIM) * G::N1;
          const real* pp = s_prm + (sp * G::NPRIM) * G::N1;
          NodeState<D, real> s;
          s.rho = pc[G::P_RHO * G::N1 + k1];
          s.T = pc[G::P_T * G::N1 + k1];
          s.div_u = 0;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            s.u[a] = pc[(G::P_U + a) * G::N1 + k1];
            s.F[a] = pc[(G::P_F + a) * G::N1 + k1];
          }
          // neighbour accessors along axis a: (plane pointer, index) of -1 / +1
#pragma unroll
          for (int a = 0; a < D; ++a) {
            const real *bm, *bp;
            int km, kp;
            if (a == D - 1) { bm = pm; bp = pp; km = kp = k1; }
            else if (a == 0) { bm = bp = pc; km = k1 - 1; kp = k1 + 1; }
            else { bm = bp = pc; km = k1 - G::BX1; kp = k1 + G::BX1; }
            s.div_u += real(0.5) * (bp[(G::P_U + a) * G::N1 + kp] - bm[(G::P_U + a) * G::N1 + km]);
            s.gradT[a] = real(0.5) * (bp[G::P_T * G::N1 + kp] - bm[G::P_T * G::N1 + km]);
            s.gradh[a] = real(0.5) * (bp[G::P_H * G::N1 + kp] - bm[G::P_H * G::N1 + km]);
            const real lc = pc[(G::P_LAM + a) * G::N1 + k1];
            const real back = lc - bm[(G::P_LAM + a) * G::N1 + km];
            const real fwd = bp[(G::P_LAM + a) * G::N1 + kp] - lc;
            s.dLam[a] = s.u[a] > real(0) ? back : (s.u[a] < real(0) ? fwd : real(0.5) * (back + fwd));
          }
          Attractors<D, real> at;
          at.setup(m, s);
          flags |= at.flags;
          const long long o = mo[1] + yo[1] + xo[1];
          // f pass then g pass: one population set in flight at a time
          real v[Q];
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const int cx = L::c(i, 0), cy = D == 3 ? L::c(i, 1) : 0, cm = L::c(i, D - 1);
            v[i] = Store<S>::template ld_last<real>(A, i * p.plane + mo[cm + 1] + yo[cy + 1] + xo[cx + 1], p.ref[i]);
          }
#pragma unroll
          for (int i = 0; i < Q; ++i)
            Store<S>::template st_stream<real>(B, i * p.plane + o, at.relax_f(i, v[i]), p.ref[i]);
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const int cx = L::c(i, 0), cy = D == 3 ? L::c(i, 1) : 0, cm = L::c(i, D - 1);
            v[i] = Store<S>::template ld_last<real>(A, (Q + i) * p.plane + mo[cm + 1] + yo[cy + 1] + xo[cx + 1],
                                                   p.ref[Q + i]);
          }
#pragma unroll
          for (int i = 0; i < Q; ++i)
            Store<S>::template st_stream<real>(B, (Q + i) * p.plane + o, at.relax_g(i, v[i]), p.ref[Q + i]);
        }
      }
      // no barrier needed here: the next write to the primitive ring (stage C)
      // comes after the two barriers of stages A and B of the next plane
    }
    __syncthreads();   // rings are reused by the next segment
  }
  if (flags) atomicOr(err, flags);
}

}  // namespace lbm
