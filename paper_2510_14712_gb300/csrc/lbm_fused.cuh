// lbm_fused.cuh - the fused single-pass time step.
//
// One kernel does, for every interior node, everything of Sec. 3.2 between
// reading the post-collision populations of the last step and writing the
// new ones: pull-stream, moments (Eqs. def_h, def_u, def_E), Korteweg force
// (Eq. FK), closure: temperature, EOS, sound speed (Eqs. lbm_temp, Pvdw,
// vdW_speed_of_sound; exact or learned), neighbour derivatives
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
// needs rho at z+-3.  With kOptPair each stage handles two planes between its
// barriers (A: pl, pl+1; B: pl-1, pl; C: pl-2, pl-1; D: pl-3, pl-2), halving
// the barriers per node; the rings then hold four planes.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_mlp.cuh"

namespace lbm {

// EX: extra per-node fields of the primitive ring (2 when the closure's P and
// c_s^2 are stored for the collision instead of recomputed there).
// NP: planes per barrier interval (each stage handles NP planes between two
// barriers); the rings then hold R = NP + 2 planes and the centre ring CN =
// NP + 1.
template <int D, int TX, int TY, int EX = 0, int NP = 1> struct FusedGeom {
  static constexpr int NT = TX * TY;                 // threads per CTA
  static constexpr int R = NP + 2, CN = NP + 1;
  static constexpr int HY3 = D == 3 ? 3 : 0, HY2 = D == 3 ? 2 : 0, HY1 = D == 3 ? 1 : 0;
  static constexpr int BX3 = TX + 6, BY3 = TY + 2 * HY3, N3 = BX3 * BY3;
  static constexpr int BX2 = TX + 4, BY2 = TY + 2 * HY2, N2 = BX2 * BY2;
  static constexpr int BX1 = TX + 2, BY1 = TY + 2 * HY1, N1 = BX1 * BY1;
  static constexpr int NMOM = D + 1;                 // j_0..j_{D-1}, S
  // primitive ring on R1 (read at the node and its neighbours): u[D], T, h, Lam[D]
  static constexpr int NPRIM = 2 * D + 2;
  static constexpr int P_U = 0, P_T = D, P_H = D + 1, P_LAM = D + 2;
  // centre ring on the tile only (read at the node): rho, F[D] (, P, c_s^2), CN planes
  static constexpr int NCEN = 1 + D + EX;
  static constexpr int C_RHO = 0, C_F = 1, C_P = 1 + D, C_CS2 = 2 + D;
  // own density of the two R1 ghost columns next to wall faces (x = -1, Nx),
  // R planes: the density ring holds their mirror images instead
  static constexpr int NGOWN = R * 2 * BY1;
  // bytes of the rings, rounded up to 16 (a closure's table follows them)
  template <typename real> static constexpr size_t smem_bytes() {
    return (sizeof(real) * size_t(R * N3 + R * NMOM * N1 + R * N2 + R * NPRIM * N1 + CN * NCEN * NT + NGOWN) + 15) &
           ~size_t(15);
  }
};

// Thermodynamic closures used by stage C of the fused step: from rho, the
// specific total energy E and |u|^2 they give e = E - |u|^2/2 and
// (T, P, c_s^2).  kWarp: the closure is warp-collective (every lane calls it,
// `act` says whether the lane's node is real).  kExtra: fields the closure
// adds to the primitive ring.  kSmem: shared-memory table bytes it loads.
// load() runs once per CTA before the first work item.

// Exact van der Waals closure: Eqs. lbm_temp, Pvdw, vdW_speed_of_sound.
// T64 (FP32 arithmetic only): the temperature inversion of Eq. lbm_temp in
// FP64 (vdw_temperature_fp64), the mixed-precision form of the FP32 and
// FP16-deviation builds.
template <typename real, bool T64 = false> struct ExactClosure {
  static constexpr bool kPr = false;
  static constexpr bool kWarp = false;
  static constexpr int kExtra = 0;
  static constexpr size_t kSmem = 0;
  double a64 = 0.0, inv_cv64 = 0.0;
  __device__ __forceinline__ void load(const Params& p, unsigned char*) {
    if constexpr (T64) {
      a64 = p.a;
      inv_cv64 = 1.0 / p.cv;
    }
  }
  __device__ __forceinline__ void operator()(const Model<real>& m, real rho, real E, real u2, bool, real& T, real& P,
                                             real& cs2, real& e) const {
    if constexpr (T64 && sizeof(real) == 4) {
      T = vdw_temperature_fp64(a64, inv_cv64, rho, E, u2, e);
    } else {
      e = E - real(0.5) * u2;
      T = (e + m.a * rho) / m.cv;
    }
    P = vdw_pressure(m, rho, T);
    cs2 = vdw_cs2(m, rho, T);
  }
};

// Exact Peng-Robinson closure: T from the quadratic in sqrt(T) of its caloric
// relation, then P and c_s^2 of the fluid; stage D reads P and c_s^2 from the
// centre ring (kExtra = 2) and e = h - P/rho.  T64 (FP32 arithmetic only):
// e = E - |u|^2/2 and the root's argument e - B0 in FP64, rounded once; the
// root itself has only positive terms and stays in FP32.
template <typename real, bool T64 = false> struct PrClosure {
  static constexpr bool kPr = true;
  static constexpr bool kWarp = false;
  static constexpr int kExtra = 2;
  static constexpr size_t kSmem = 0;
  __device__ __forceinline__ void load(const Params&, unsigned char*) {}
  __device__ __forceinline__ void operator()(const Model<real>& m, real rho, real E, real u2, bool, real& T, real& P,
                                             real& cs2, real& e) const {
    if constexpr (T64 && sizeof(real) == 4) {
      const double ed = double(E) - 0.5 * double(u2);
      e = real(ed);
      T = pr_temperature_q(m, rho, ed);
    } else {
      e = E - real(0.5) * u2;
      T = pr_temperature(m, rho, e);
    }
    P = pr_pressure(m, rho, T);
    cs2 = pr_cs2(m, rho, T);
  }
};

// Learned closure: the network of lbm_mlp.cuh inside its training box, the
// exact closure outside it (range gate).  FP32 arithmetic only.
struct MlpClosure {
  static constexpr bool kPr = false;
  static constexpr bool kWarp = true;
  static constexpr int kExtra = 2;
  static constexpr size_t kSmem = sizeof(mlp::Image);
  const mlp::Image* w;
  __device__ __forceinline__ void load(const Params& p, unsigned char* smem) {
    mlp::Image* d = reinterpret_cast<mlp::Image*>(smem);
    mlp::load_image(static_cast<const mlp::Image*>(p.mlp), d);
    w = d;
  }
  __device__ __forceinline__ void operator()(const Model<float>& m, float rho, float E, float u2, bool act, float& T,
                                             float& P, float& cs2, float& e) const {
    e = E - 0.5f * u2;
    mlp::closure_warp(*w, m, rho, e, act, T, P, cs2);
  }
};

// v mod n in [0, n) for any integer v
__device__ __forceinline__ int modp(int v, int n) {
  const int r = v % n;
  return r < 0 ? r + n : r;
}

// v wrapped into [0, n); cheap form valid for -n <= v < 2n, exact form otherwise
template <bool SMALL> __device__ __forceinline__ int wrapc(int v, int n) {
  if (SMALL) return modp(v, n);
  v += v < 0 ? n : 0;
  return v >= n ? v - n : v;
}

// distance outside the tile along one in-plane axis (0 inside)
__device__ __forceinline__ int outside(int l, int h, int T) {
  const int v = l - h;
  return v < 0 ? -v : (v >= T ? v - T + 1 : 0);
}

// Options of the fused step (template bit mask).
//   kOptRows: stage A in row form (3-D; FP32 or FP16-deviation storage; Nx a
//     multiple of 4; not SMALL; no wall face, whose ghost columns take mirror
//     densities in the position form): the R3 box is cut into
//     rows of TX + 8 nodes that start 4 nodes left of the tile, and each row
//     into chunks of 4 nodes, one chunk per lane.  A lane reads the 4 values of
//     one direction with one 16-byte (FP16: 8-byte) load of the source row
//     (aligned: x0, Nx and the ghost width are multiples of 4, so a chunk
//     never straddles the periodic seam), and the value a node pulls from across the chunk edge
//     comes from the neighbouring lane by a shuffle.  Warps take groups of
//     whole rows: the f rows of the R3 box (rho; j on the R1 rows), then the
//     g rows of the R1 box (S).  Per node and direction the moments are summed
//     in the same order as the position form, so both give the same bits.
//     Stage D's in-plane pull offsets are computed once per work item (the
//     thread's node is the same on every plane).
//   kOptPair: two planes per barrier interval (stages A to D each handle two
//     planes between their barriers; rings of four planes).
constexpr int kOptRows = 1, kOptPair = 2;

// planes per barrier interval of option set OPT
template <int OPT> constexpr int planes_per_interval() { return (OPT & kOptPair) ? 2 : 1; }

// One (column, z-segment) work item of the fused step: all planes mb..me-1 of
// the column of TX x hy nodes at (x0, y0) (hy <= TY rows; 1 in 2-D), reading A
// and writing B.  Shared by the single-instance kernel and the batched
// persistent kernel.  SMALL: the box is narrower than a tile plus its halo in
// x or y, so coordinates need an exact modulo instead of a single conditional
// wrap.
template <int D, typename S, typename real, int TX, int TY, bool SMALL, class CL, int OPT = 0>
__device__ __forceinline__ void fused_column(const Params& p, const typename Store<S>::T* __restrict__ A,
                                             typename Store<S>::T* __restrict__ B, int x0, int y0, int hy, int mb,
                                             int me, unsigned char* smem_raw, unsigned& flags, const CL& closure) {
  using L = Lattice<D>;
  constexpr int NP = planes_per_interval<OPT>();
  using G = FusedGeom<D, TX, TY, CL::kExtra, NP>;
  constexpr int Q = L::Q;
  real* s_rho = reinterpret_cast<real*>(smem_raw);            // [R][N3]
  real* s_mom = s_rho + G::R * G::N3;                         // [R][NMOM][N1]
  real* s_lap = s_mom + G::R * G::NMOM * G::N1;               // [R][N2]
  real* s_prm = s_lap + G::R * G::N2;                         // [R][NPRIM][N1]
  real* s_cen = s_prm + G::R * G::NPRIM * G::N1;              // [CN][NCEN][NT]
  real* s_gown = s_cen + G::CN * G::NCEN * G::NT;             // [R][2][BY1]
  // ring slot of plane v >= -4
  auto rs = [](int v) { return G::R == 3 ? (v + 6) % 3 : (v + 8) & 3; };
  auto cs = [](int v) { return G::CN == 2 ? (v & 1) : (v + 6) % 3; };

  const Model<real> m = model_of<real>(p);
  const int tid = threadIdx.x;
  const int Nm = D == 3 ? p.Nz : p.Ny;                        // march extent
  const long long mstride = D == 3 ? (long long)p.Ny * p.pitch : (long long)p.pitch;
  const int xmin = p.periodic_x ? -0x40000000 : -3, xmax = p.periodic_x ? 0x40000000 : p.Nx + 2;
  // the column's R3 box reaches a ghost column of a wall face (block-uniform)
  const bool wtile = (p.bc_lo == LBM_BC_WALL && x0 < 3) || (p.bc_hi == LBM_BC_WALL && x0 + TX + 3 > p.Nx);
  using ST = typename Store<S>::T;
  // element offsets inside a population buffer fit 32 bits (checked at create)
  const unsigned plane32 = unsigned(p.plane), pitch32 = unsigned(p.pitch);

  constexpr bool kRows = (OPT & kOptRows) != 0 && D == 3 && !SMALL && sizeof(real) == 4;
  constexpr bool kItem = kRows;
  // stage D's in-plane pull offsets of this thread's node (kItem)
  unsigned dxc[3], dyr[3];
  if constexpr (kItem) {
    const int dgx = x0 + tid % TX, dgy = y0 + tid / TX;
#pragma unroll
    for (int c = -1; c <= 1; ++c) {
      dxc[c + 1] = unsigned(p.periodic_x ? wrapc<SMALL>(dgx - c, p.Nx) : dgx + p.G - c);
      dyr[c + 1] = D == 3 ? unsigned(wrapc<SMALL>(dgy - c, p.Ny)) * pitch32 : 0u;
    }
  }

  for (int pl = mb - 3; pl <= me + 2; pl += NP) {
    // ---------------- A: moments of planes pl .. pl+NP-1 ----------------------
    if constexpr (kRows) {
      constexpr int NCH = (TX + 8) / 4, RPW = 32 / NCH;
      static_assert(TX % 4 == 0 && RPW >= 1, "row form: TX + 8 nodes in 4-node chunks, at least one row per warp");
      // plane pointers and ring slots of the interval's planes (NP <= 2)
      const ST* PmA[3];
      const ST* PmB[3];
      int slotA = rs(pl), slotB = slotA;
      {
        const int mp = modp(pl, Nm);
#pragma unroll
        for (int c = -1; c <= 1; ++c) PmA[c + 1] = PmB[c + 1] = A + (long long)wrap(mp - c, Nm) * mstride;
      }
      if constexpr (NP > 1) {
        const int mp = modp(pl + 1, Nm);
        slotB = rs(pl + 1);
#pragma unroll
        for (int c = -1; c <= 1; ++c) PmB[c + 1] = A + (long long)wrap(mp - c, Nm) * mstride;
      }
      const int lane = tid & 31, rr = lane / NCH, ch = lane - rr * NCH;
      // Row groups of three kinds: f rows of the R1 box (rho and j), g rows of
      // the R1 box (S), and the four f rows of the R3 box outside it (rho
      // only).  Warps take groups in snake order (w, 2 nw - 1 - w, 2 nw + w,
      // ...), so that the warps given a second group hold the cheap ones.
      const int n1 = hy + 2 * G::HY1;                                   // rows of the R1 box
      const int g1 = (n1 + RPW - 1) / RPW, g3 = (4 + RPW - 1) / RPW;
      const int ngroups = 2 * g1 + g3, nw = G::NT / 32, w = tid >> 5;
      // padded x of the chunk's first node: wrapped when x is periodic; else
      // shifted by the ghost layers, and chunks past the last one a node of
      // the box pulls from (x = Nx + 3, inside the row since Nx and G are
      // multiples of 4) are moved into the row (their values are not used)
      int xs = x0 - 4 + 4 * ch;
      if (p.periodic_x) {
        xs += xs < 0 ? p.Nx : 0;
        xs -= xs >= p.Nx ? p.Nx : 0;
      } else {
        xs = min(xs + p.G, p.pitch - 4);
      }
      for (int k = 0;; ++k) {
        // group index over the NP planes of the interval
        const int gp = (k & 1) ? (k + 1) * nw - 1 - w : k * nw + w;
        if (gp >= NP * ngroups) break;
        static_assert(NP == 1 || NP == 2, "one or two planes per interval");
        const int sa = NP == 1 ? 0 : int(gp >= ngroups);
        const int pa = pl + sa, gi = gp - sa * ngroups;
        if (NP > 1 && pa > me + 2) continue;                            // warp-uniform
        const int slot = sa ? slotB : slotA;
        const ST* Pm[3] = {sa ? PmB[0] : PmA[0], sa ? PmB[1] : PmA[1], sa ? PmB[2] : PmA[2]};
        const int kind = gi < g1 ? 0 : (gi < 2 * g1 ? 1 : 2);          // warp-uniform
        const int r = (gi - (kind == 0 ? 0 : (kind == 1 ? g1 : 2 * g1))) * RPW + rr;
        const bool act = rr < RPW && r < (kind == 2 ? 4 : n1);
        // row of the R3 box
        const int ly = kind == 2 ? (r < 2 ? r : hy + 2 + r) : r + (G::HY3 - G::HY1);
        const int gy = y0 + ly - G::HY3;
        unsigned ro[3];
#pragma unroll
        for (int c = -1; c <= 1; ++c) ro[c + 1] = unsigned(wrapc<false>(act ? gy - c : y0, p.Ny)) * pitch32 + xs;
        // the four nodes' values of direction i, as pulled: element j of the
        // chunk, or of the chunk left / right of it (neighbouring lane)
        auto pulled = [&](const int i, const int ii, real* w) {
          const int cx = L::c(i, 0), cy = L::c(i, 1), cm = L::c(i, 2);
          const unsigned o = unsigned(ii) * plane32 + ro[cy + 1];
          // every lane loads (idle lanes read a valid chunk of row y0 whose
          // values no active lane takes), so the loads need no predicate
          real v[4];
          if (pop_ok(p, Pm[cm + 1], o, 4)) Store<S>::template ld4<real>(Pm[cm + 1], o, p.ref[ii], v);
          else v[0] = v[1] = v[2] = v[3] = real(0);
          if (cx == 1) {
            w[0] = __shfl_up_sync(0xffffffffu, v[3], 1);
            w[1] = v[0]; w[2] = v[1]; w[3] = v[2];
          } else if (cx == -1) {
            w[0] = v[1]; w[1] = v[2]; w[2] = v[3];
            w[3] = __shfl_down_sync(0xffffffffu, v[0], 1);
          } else {
            w[0] = v[0]; w[1] = v[1]; w[2] = v[2]; w[3] = v[3];
          }
        };
        if (kind == 0) {
          real rho[4], sp[D][4], sn[D][4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            rho[j] = real(0);
#pragma unroll
            for (int a = 0; a < D; ++a) sp[a][j] = sn[a][j] = real(0);
          }
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            real w[4];
            pulled(i, i, w);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              rho[j] += w[j];
#pragma unroll
              for (int a = 0; a < D; ++a) {
                if (L::c(i, a) == 1) sp[a][j] += w[j];
                if (L::c(i, a) == -1) sn[a][j] += w[j];
              }
            }
          }
          if (act) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int lx = 4 * ch + j - 1;                            // x index in the R3 box
              if (lx >= 0 && lx < G::BX3) s_rho[slot * G::N3 + ly * G::BX3 + lx] = rho[j];
              const int lx1 = lx - 2;                                   // x index in the R1 box
              if (lx1 >= 0 && lx1 < G::BX1) {
                real* dst = s_mom + (slot * G::NMOM) * G::N1 + (ly - (G::HY3 - G::HY1)) * G::BX1 + lx1;
#pragma unroll
                for (int a = 0; a < D; ++a) dst[a * G::N1] = sp[a][j] - sn[a][j];
              }
            }
          }
        } else if (kind == 2) {
          real rho[4] = {real(0), real(0), real(0), real(0)};
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            real w[4];
            pulled(i, i, w);
#pragma unroll
            for (int j = 0; j < 4; ++j) rho[j] += w[j];
          }
          if (act) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int lx = 4 * ch + j - 1;
              if (lx >= 0 && lx < G::BX3) s_rho[slot * G::N3 + ly * G::BX3 + lx] = rho[j];
            }
          }
        } else {
          real Se[4] = {real(0), real(0), real(0), real(0)};
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            real w[4];
            pulled(i, Q + i, w);
#pragma unroll
            for (int j = 0; j < 4; ++j) Se[j] += w[j];
          }
          if (act) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int lx1 = 4 * ch + j - 3;
              if (lx1 >= 0 && lx1 < G::BX1) s_mom[(slot * G::NMOM + D) * G::N1 + r * G::BX1 + lx1] = Se[j];
            }
          }
        }
      }
    } else
    // Position form.
    // Direction-outer loop over this thread's positions of the R3 box: three
    // per-plane base pointers and one 32-bit element offset per load
    // (direction * plane + row + column).  j_a is accumulated as (sum over
    // c_a = +1) minus (sum over c_a = -1), both in increasing direction order,
    // so the two halves are computed identically for mirror-symmetric
    // populations and j is then exactly zero (as the pairwise sum of Eq.
    // def_u).  Positions 0 .. KFULL*NT-1 are spread over all threads; the
    // remainder (fewer than NT) is done by the first threads only.
    for (int sa = 0; sa < NP; ++sa) {
      const int pa = pl + sa;
      if (NP > 1 && pa > me + 2) break;
      const int slot = rs(pa);
      const int mp = modp(pa, Nm);
      const ST* Pm[3];
#pragma unroll
      for (int c = -1; c <= 1; ++c) Pm[c + 1] = A + (long long)wrap(mp - c, Nm) * mstride;
      auto moments = [&](const int k) {
        const int lx = k % G::BX3, ly = k / G::BX3;
        const int ox = outside(lx, 3, TX), oy = D == 3 ? outside(ly, G::HY3, hy) : 0;
        const int gx = x0 + lx - 3;
        if (ox + oy > 3 || gx < xmin || gx > xmax) return;
        const bool in1 = ox + oy <= 1;
        const int gy = D == 3 ? wrapc<SMALL>(y0 + ly - G::HY3, p.Ny) : 0;
        unsigned xc[3], yr[3];
#pragma unroll
        for (int c = -1; c <= 1; ++c) {
          xc[c + 1] = unsigned(p.periodic_x ? wrapc<SMALL>(gx - c, p.Nx) : gx + p.G - c);
          yr[c + 1] = D == 3 ? unsigned(wrapc<SMALL>(gy - c, p.Ny)) * pitch32 : 0u;
        }
        real rho = real(0), sp[D], sn[D];
#pragma unroll
        for (int a = 0; a < D; ++a) sp[a] = sn[a] = real(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const int cx = L::c(i, 0), cy = D == 3 ? L::c(i, 1) : 0, cm = L::c(i, D - 1);
          const unsigned o = unsigned(i) * plane32 + yr[cy + 1] + xc[cx + 1];
          const real v = pop_ok(p, Pm[cm + 1], o) ? Store<S>::template ld<real>(Pm[cm + 1], o, p.ref[i]) : real(0);
          rho += v;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            if (L::c(i, a) == 1) sp[a] += v;
            if (L::c(i, a) == -1) sn[a] += v;
          }
        }
        const int gw = wtile ? wall_mirror(p, gx) : gx;
        if (gw != gx) {
          // ghost column of a wall face: the Laplacian reads the density of the
          // mirror image (pulled here the same way as at that node); stage C
          // reads the column's own density at x = -1 and x = Nx
          if (in1 && (gx == -1 || gx == p.Nx))
            s_gown[(slot * 2 + (gx < 0 ? 0 : 1)) * G::BY1 + ly - (G::HY3 - G::HY1)] = rho;
          rho = real(0);
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const int cx = L::c(i, 0), cy = D == 3 ? L::c(i, 1) : 0, cm = L::c(i, D - 1);
            const unsigned o = unsigned(i) * plane32 + yr[cy + 1] + unsigned(gw + p.G - cx);
            rho += pop_ok(p, Pm[cm + 1], o) ? Store<S>::template ld<real>(Pm[cm + 1], o, p.ref[i]) : real(0);
          }
        }
        s_rho[slot * G::N3 + k] = rho;
        if (in1) {
          real Se = real(0);
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const int cx = L::c(i, 0), cy = D == 3 ? L::c(i, 1) : 0, cm = L::c(i, D - 1);
            const unsigned o = unsigned(Q + i) * plane32 + yr[cy + 1] + xc[cx + 1];
            Se += pop_ok(p, Pm[cm + 1], o) ? Store<S>::template ld<real>(Pm[cm + 1], o, p.ref[Q + i]) : real(0);
          }
          const int k1 = (ly - (G::HY3 - G::HY1)) * G::BX1 + (lx - 2);
          real* dst = s_mom + (slot * G::NMOM) * G::N1 + k1;
#pragma unroll
          for (int a = 0; a < D; ++a) dst[a * G::N1] = sp[a] - sn[a];
          dst[D * G::N1] = Se;
        }
      };
      constexpr int KFULL = G::N3 / G::NT, KREM = G::N3 % G::NT;
#pragma unroll 1
      for (int jp = 0; jp < KFULL; ++jp) moments(tid + jp * G::NT);
      if (KREM > 0 && tid < KREM) moments(tid + KFULL * G::NT);
    }
    __syncthreads();

    // ---------------- B: Laplacian of rho, planes pl-1 .., on R2 --------------
    for (int sq = 0; sq < NP; ++sq) {
      const int q = pl - 1 + sq;
      if (q < mb - 2 || (NP > 1 && q > me + 1)) continue;
      const int sc = rs(q), sm = rs(q - 1), sp = rs(q + 1);
      const int n2 = G::BX2 * (hy + 2 * G::HY2);              // the band's rows of the R2 box
      for (int k = tid; k < n2; k += G::NT) {
        const int lx = k % G::BX2, ly = k / G::BX2;
        const int ox = outside(lx, 2, TX), oy = D == 3 ? outside(ly, G::HY2, hy) : 0;
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

    // ---------------- C: primitive fields, planes pl-2 .., on R1 --------------
    // The loop runs a warp-uniform number of times (warp-collective closures);
    // `act` marks the lanes whose position is a needed node.
    for (int sq = 0; sq < NP; ++sq) {
      const int q = pl - 2 + sq;
      if (q < mb - 1 || (NP > 1 && q > me)) continue;
      const int sc = rs(q), sm = rs(q - 1), sp = rs(q + 1);
      const int lane = tid & 31;
      const int n1 = G::BX1 * (hy + 2 * G::HY1);              // the band's rows of the R1 box
      for (int k0 = tid - lane; k0 < n1; k0 += G::NT) {
        const int k = k0 + lane;
        const int lx = k % G::BX1, ly = k / G::BX1;
        const int ox = outside(lx, 1, TX), oy = D == 3 ? outside(ly, G::HY1, hy) : 0;
        const int gx = x0 + lx - 1;
        const bool act = k < G::N1 && ox + oy <= 1 && gx >= xmin + 2 && gx <= xmax - 2;
        real rho = real(1), E = real(0), u2 = real(0), F[D], u[D];
#pragma unroll
        for (int a = 0; a < D; ++a) F[a] = u[a] = real(0);
        if (act) {
          const int k3 = (ly + (G::HY3 - G::HY1)) * G::BX3 + (lx + 2);
          const int k2 = (ly + (G::HY2 - G::HY1)) * G::BX2 + (lx + 1);
          rho = s_rho[sc * G::N3 + k3];
          if (wtile && wall_mirror(p, gx) != gx) rho = s_gown[(sc * 2 + (gx < 0 ? 0 : 1)) * G::BY1 + ly];
          const real* lp = s_lap + sc * G::N2;
          F[0] = m.kappa * rho * real(0.5) * (lp[k2 + 1] - lp[k2 - 1]);                         // Eq. FK
          if (D == 3) F[1] = m.kappa * rho * real(0.5) * (lp[k2 + G::BX2] - lp[k2 - G::BX2]);
          F[D - 1] = m.kappa * rho * real(0.5) * (s_lap[sp * G::N2 + k2] - s_lap[sm * G::N2 + k2]);
          const real* mo = s_mom + (sc * G::NMOM) * G::N1 + k;
          real uF = 0;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            u[a] = div_rn(mo[a * G::N1] + real(0.5) * F[a], rho);                              // Eq. def_u
            uF += u[a] * F[a];
            u2 += u[a] * u[a];
          }
          E = div_rn(mo[D * G::N1] + real(0.5) * uF, rho);                                    // Eq. def_E
        }
        // closure (rho, E, |u|^2) -> e, (T, P, c_s^2)
        real T = real(0), P = real(1), cs2 = real(0), e = real(0);
        if constexpr (CL::kWarp) closure(m, rho, E, u2, act, T, P, cs2, e);
        else if (act) closure(m, rho, E, u2, act, T, P, cs2, e);
        if (act) {
          const real theta = P / rho;
          real* pr = s_prm + (sc * G::NPRIM) * G::N1 + k;
          pr[G::P_T * G::N1] = T;
          pr[G::P_H * G::N1] = e + theta;                                                      // Eq. enthalpy
#pragma unroll
          for (int a = 0; a < D; ++a) {
            pr[(G::P_U + a) * G::N1] = u[a];
            pr[(G::P_LAM + a) * G::N1] = rho * u[a] * u[a] * u[a] + real(3) * rho * u[a] * (theta - real(1.0 / 3.0));
          }
          if (lx >= 1 && lx <= TX && ly >= G::HY1 && ly < G::HY1 + hy) {                       // a tile node
            if (p.sc_on && q >= mb && q < me) {
              // this step's rho, u, T for the shock-capturing coefficients of the next step
              const int tx = x0 + lx - 1, ty = D == 3 ? y0 + ly - G::HY1 : 0;
              if (tx < p.Nx && (D == 2 || ty < p.Ny)) {
                const int mq = modp(q, Nm);
                const long long o = (D == 3 ? ((long long)mq * p.Ny + ty) * p.pitch : (long long)mq * p.pitch) +
                                    tx + p.G;
                real* W = static_cast<real*>(p.sc_prims);
                W[o] = rho;
#pragma unroll
                for (int a = 0; a < D; ++a) W[(1 + a) * p.plane + o] = u[a];
                W[(1 + D) * p.plane + o] = T;
              }
            }
            real* ce = s_cen + (cs(q) * G::NCEN) * G::NT + (ly - G::HY1) * TX + (lx - 1);
            ce[G::C_RHO * G::NT] = rho;
#pragma unroll
            for (int a = 0; a < D; ++a) ce[(G::C_F + a) * G::NT] = F[a];
            if constexpr (CL::kExtra > 0) {
              ce[G::C_P * G::NT] = P;
              ce[G::C_CS2 * G::NT] = cs2;
            }
          }
        }
      }
    }
    __syncthreads();

    // ---------------- D: collide planes pl-3 .. on the tile ----------------------
    for (int sq = 0; sq < NP; ++sq) {
      const int q = pl - 3 + sq;
      if (q < mb || (NP > 1 && q >= me)) continue;
      const int sc = rs(q), sm = rs(q - 1), sp = rs(q + 1);
      const int lx = tid % TX, ly = tid / TX;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx < p.Nx && (D == 2 || (ly < hy && gy < p.Ny))) {
        const int mq = modp(q, Nm);
        const ST* Pm[3];
        unsigned xc[3], yr[3];
#pragma unroll
        for (int c = -1; c <= 1; ++c) {
          Pm[c + 1] = A + (long long)wrap(mq - c, Nm) * mstride;
          if constexpr (kItem) {
            xc[c + 1] = dxc[c + 1];
            yr[c + 1] = dyr[c + 1];
          } else {
            xc[c + 1] = unsigned(p.periodic_x ? wrapc<SMALL>(gx - c, p.Nx) : gx + p.G - c);
            yr[c + 1] = D == 3 ? unsigned(wrapc<SMALL>(gy - c, p.Ny)) * pitch32 : 0u;
          }
        }
        ST* Bq = B + (long long)mq * mstride;
        const int k1 = (ly + G::HY1) * G::BX1 + (lx + 1);
        const real* pc = s_prm + (sc * G::NPRIM) * G::N1;
        const real* pm = s_prm + (sm * G::NPRIM) * G::N1;
        const real* pp = s_prm + (sp * G::NPRIM) * G::N1;
        NodeState<D, real> s;
        const real* cc = s_cen + (cs(q) * G::NCEN) * G::NT + tid;
        s.rho = cc[G::C_RHO * G::NT];
        s.T = pc[G::P_T * G::N1 + k1];
        if constexpr (CL::kExtra > 0) {
          s.P = cc[G::C_P * G::NT];
          s.cs2 = cc[G::C_CS2 * G::NT];
          s.e = pc[G::P_H * G::N1 + k1] - s.P / s.rho;
        } else {
          s.P = vdw_pressure(m, s.rho, s.T);
          s.cs2 = vdw_cs2(m, s.rho, s.T);
          s.e = vdw_energy(m, s.rho, s.T);
        }
        s.sc = p.sc_on != 0;
        s.mu_num = s.eta_num = s.k_num = real(0);
        if (s.sc) {
          const long long o = (D == 3 ? ((long long)mq * p.Ny + gy) * p.pitch : (long long)mq * p.pitch) + gx + p.G;
          const real* V = static_cast<const real*>(p.sc_visc);
          s.mu_num = V[o];
          s.eta_num = V[p.plane + o];
          s.k_num = V[2 * p.plane + o];
        }
        s.div_u = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          s.u[a] = pc[(G::P_U + a) * G::N1 + k1];
          s.F[a] = cc[(G::C_F + a) * G::NT];
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
        const unsigned oc = yr[1] + xc[1];                  // own in-plane offset
        // f pass then g pass: one population set in flight at a time
        real v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const int cx = L::c(i, 0), cy = D == 3 ? L::c(i, 1) : 0, cm = L::c(i, D - 1);
          const unsigned o = unsigned(i) * plane32 + yr[cy + 1] + xc[cx + 1];
          v[i] = pop_ok(p, Pm[cm + 1], o) ? Store<S>::template ld_last<real>(Pm[cm + 1], o, p.ref[i]) : real(0);
        }
        FactoredRelax<D, real>::f_pass(at, [&](int i) { return v[i]; }, [&](int i, real x) {
          if (pop_ok(p, Bq, unsigned(i) * plane32 + oc))
            Store<S>::template st_stream<real>(Bq, unsigned(i) * plane32 + oc, x, p.ref[i]);
        });
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const int cx = L::c(i, 0), cy = D == 3 ? L::c(i, 1) : 0, cm = L::c(i, D - 1);
          const unsigned o = unsigned(Q + i) * plane32 + yr[cy + 1] + xc[cx + 1];
          v[i] = pop_ok(p, Pm[cm + 1], o) ? Store<S>::template ld_last<real>(Pm[cm + 1], o, p.ref[Q + i]) : real(0);
        }
        FactoredRelax<D, real>::g_pass(at, [&](int i) { return v[i]; }, [&](int i, real x) {
          if (pop_ok(p, Bq, unsigned(Q + i) * plane32 + oc))
            Store<S>::template st_stream<real>(Bq, unsigned(Q + i) * plane32 + oc, x, p.ref[Q + i]);
        });
      }
    }
    // no barrier needed here: the next write to the primitive ring (stage C)
    // comes after the two barriers of stages A and B of the next plane
  }
  __syncthreads();   // rings are reused by the next work item
}

// Single-instance step: work items are (column, z-segment) pairs, ordered
// segment-major so that the CTAs resident together cover neighbouring
// columns at the same planes and their halos are L2 hits.  Columns are TX
// nodes wide and, in 3-D, one of ncoly bands of y rows (at most TY rows each;
// the launch picks ncoly so that the columns spread evenly over the resident
// CTA slots).  MINB: CTAs per SM
// the register allocation must allow (2 keeps one CTA's memory phase
// overlapping the other's collision).
template <int D, typename S, typename real, int TX, int TY, int MINB, bool SMALL, class CL = ExactClosure<real>,
          int OPT = 0>
__global__ void __launch_bounds__(TX * TY, MINB)
k_step_fused(const __grid_constant__ Params p, const typename Store<S>::T* __restrict__ A,
             typename Store<S>::T* __restrict__ B, unsigned* err, int ncolx, int ncoly, int nseg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CL closure;
  closure.load(p, smem_raw + FusedGeom<D, TX, TY, CL::kExtra, planes_per_interval<OPT>()>::template smem_bytes<real>());
  if constexpr (CL::kSmem > 0) __syncthreads();
  unsigned flags = 0;
  const int Nm = D == 3 ? p.Nz : p.Ny;
  const int ncol = ncolx * ncoly;
  const long long nitems = (long long)ncol * nseg;
  for (long long it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int col = int(it % ncol);
    const int seg = int(it / ncol);
    const int mb = int((long long)Nm * seg / nseg), me = int((long long)Nm * (seg + 1) / nseg);
    const int x0 = (col % ncolx) * TX;
    // 3-D: ncoly bands of y rows, as even as integers allow (each at most TY rows)
    const int band = col / ncolx;
    const int y0 = D == 3 ? int((long long)p.Ny * band / ncoly) : 0;
    const int hy = D == 3 ? int((long long)p.Ny * (band + 1) / ncoly) - y0 : 1;
    fused_column<D, S, real, TX, TY, SMALL, CL, OPT>(p, A, B, x0, y0, hy, mb, me, smem_raw, flags, closure);
  }
  if (flags) atomicOr(err, flags);
}

// One instance of a batch: its parameters, its two population buffers and its
// column count along x (ncoly = 1 in 2-D; 3-D columns are ncolx per y-row).
struct BatchInstance {
  Params p;
  void* pop[2];
  int ncolx, ncoly;
  int pad[2];
};

// One work item of a batch step: instance, column, plane range.
struct BatchItem {
  int inst, col, mb, me;
};

// Batched step: one persistent launch over the work items of every instance
// (sorted longest first), taken dynamically from an atomic counter so that
// uneven instances balance.  `parity` selects which buffer of each instance is
// the source.  Fatal / warning bits go to the instance's word in `errs`.
// SMALL instances are handled by the exact-modulo variant of the column body.
template <int D, typename S, typename real, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB)
k_step_fused_batch(const BatchInstance* __restrict__ insts, const BatchItem* __restrict__ items, int nitems,
                   int parity, int* counter, unsigned* errs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  using ST = typename Store<S>::T;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const BatchItem w = items[it];
    const BatchInstance& bi = insts[w.inst];
    const Params& p = bi.p;
    const ST* A = reinterpret_cast<const ST*>(bi.pop[parity]);
    ST* B = reinterpret_cast<ST*>(bi.pop[parity ^ 1]);
    const int x0 = (w.col % bi.ncolx) * TX;
    const int y0 = D == 3 ? (w.col / bi.ncolx) * TY : 0;
    unsigned flags = 0;
    const bool small = (p.periodic_x && p.Nx < TX + 6) || (D == 3 && p.Ny < TY + 6);
    const ExactClosure<real> cl{};
    if (small) fused_column<D, S, real, TX, TY, true>(p, A, B, x0, y0, TY, w.mb, w.me, smem_raw, flags, cl);
    else fused_column<D, S, real, TX, TY, false>(p, A, B, x0, y0, TY, w.mb, w.me, smem_raw, flags, cl);
    if (flags) atomicOr(errs + w.inst, flags);
  }
}

// Batched ghost fill: block b refills the x ghost layers of instance b (if its
// x faces are not periodic), as k_ghosts does for one instance.
template <int D, typename S>
__global__ void k_ghosts_batch(const BatchInstance* __restrict__ insts, int parity) {
  using ST = typename Store<S>::T;
  const BatchInstance& bi = insts[blockIdx.x];
  const Params& p = bi.p;
  if (p.periodic_x) return;
  ST* Bp = reinterpret_cast<ST*>(bi.pop[parity ^ 1]);
  const long long n = 2LL * p.G * p.Ny * p.Nz;
  for (long long gid = threadIdx.x; gid < n; gid += blockDim.x) {
    const int g = int(gid % (2 * p.G));
    const long long r = gid / (2 * p.G);
    ghost_node<D, S>(p, Bp, g, int(r % p.Ny), int(r / p.Ny));
  }
}

}  // namespace lbm
