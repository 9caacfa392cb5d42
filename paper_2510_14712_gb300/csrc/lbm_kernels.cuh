// lbm_kernels.cuh - kernels of the library, templated on the dimension D,
// the storage type of the populations and the arithmetic type.
//
// Data layout in HBM (all kernels):
//   population p_i of node (x, y, z) at  base + i*plane + (z*Ny + y)*pitch + (x + G)
//   with G = 4 ghost layers per non-periodic x face (G = 0 when x is
//   periodic), pitch >= Nx + 2G rounded up to 32 elements, plane = Nz*Ny*pitch.
//   The buffer holds the post-collision populations of the last step (pull
//   scheme: node x reads p_i at x - c_i).
//
// The multi-pass step (this file) is: moments -> primitive fields -> collide
// -> ghost fill.  It keeps per-node moment and primitive fields in a scratch
// area of 2D+... planes; the fused single-pass kernel lives in lbm_fused.cuh.
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// storage traits: how one population value is kept in HBM
// ---------------------------------------------------------------------------
struct Fp16Dev {};  // tag: FP16 storage of p_i - p_i^ref

template <typename S> struct Store;
// ld/st: plain; ld_last: last read of the value in this step (evict-first);
// st_stream: streaming store of the new populations (evict-first).
template <> struct Store<double> {
  using T = double;
  template <typename real, typename I> __device__ static real ld(const T* p, I o, float) { return real(__ldg(p + o)); }
  template <typename real, typename I> __device__ static real ld_last(const T* p, I o, float) { return real(__ldcs(p + o)); }
  template <typename real, typename I> __device__ static void st(T* p, I o, real v, float) { p[o] = double(v); }
  template <typename real, typename I> __device__ static void st_stream(T* p, I o, real v, float) { __stcs(p + o, double(v)); }
};
template <> struct Store<float> {
  using T = float;
  template <typename real, typename I> __device__ static real ld(const T* p, I o, float) { return real(__ldg(p + o)); }
  template <typename real, typename I> __device__ static real ld_last(const T* p, I o, float) { return real(__ldcs(p + o)); }
  template <typename real, typename I> __device__ static void st(T* p, I o, real v, float) { p[o] = float(v); }
  template <typename real, typename I> __device__ static void st_stream(T* p, I o, real v, float) { __stcs(p + o, float(v)); }
  // four consecutive values p[o .. o+3], o a multiple of 4 (one 16-byte load)
  template <typename real, typename I> __device__ static void ld4(const T* p, I o, float, real* v) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p + o));
    v[0] = real(q.x); v[1] = real(q.y); v[2] = real(q.z); v[3] = real(q.w);
  }
};
template <> struct Store<Fp16Dev> {
  using T = __half;
  template <typename real, typename I> __device__ static real ld(const T* p, I o, float ref) {
    return real(__half2float(__ldg(p + o)) + ref);
  }
  template <typename real, typename I> __device__ static real ld_last(const T* p, I o, float ref) {
    return real(__half2float(__ldcs(p + o)) + ref);
  }
  template <typename real, typename I> __device__ static void st(T* p, I o, real v, float ref) {
    p[o] = __float2half_rn(float(v) - ref);
  }
  template <typename real, typename I> __device__ static void st_stream(T* p, I o, real v, float ref) {
    __stcs(p + o, __float2half_rn(float(v) - ref));
  }
  // four consecutive values p[o .. o+3], o a multiple of 4 (one 8-byte load)
  template <typename real, typename I> __device__ static void ld4(const T* p, I o, float ref, real* v) {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(p + o));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    v[0] = real(a.x + ref); v[1] = real(a.y + ref); v[2] = real(b.x + ref); v[3] = real(b.y + ref);
  }
};

// ---------------------------------------------------------------------------
// bounds-check builds (-DLBM_BOUNDS_CHECK): every population access of the
// step kernels must lie inside one of the handle's two population buffers;
// one outside is skipped (a load gives 0) and counted.  Other builds compile
// the check away.
// ---------------------------------------------------------------------------
#ifdef LBM_BOUNDS_CHECK
namespace {
__device__ unsigned long long g_oob;                 // accesses outside the buffers (this unit's kernels)
unsigned long long read_oob() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, g_oob, sizeof(v));
  return v;
}
struct OobReaderRegistration {
  OobReaderRegistration() { register_oob_reader(&read_oob); }
} g_oob_registration;
}  // namespace
#endif

// access to the n elements ptr[off .. off + n) is inside a population buffer of p
template <typename T>
__device__ __forceinline__ bool pop_ok(const Params& p, const T* ptr, long long off, int n = 1) {
#ifdef LBM_BOUNDS_CHECK
  const T* a = ptr + off;
  const long long len = 2LL * p.Q * p.plane;
  for (int k = 0; k < 2; ++k) {
    const T* lo = static_cast<const T*>(p.pop[k]);
    if (lo && a >= lo && a + n <= lo + len) return true;
  }
  atomicAdd(&g_oob, 1ULL);
  return false;
#else
  return true;
#endif
}

// ---------------------------------------------------------------------------
// geometry helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ long long node_off(const Params& p, int xp, int y, int z) {
  return ((long long)z * p.Ny + y) * p.pitch + xp;
}

// padded x of interior coordinate x (+ shift), wrapped when x is periodic
__device__ __forceinline__ int xpad(const Params& p, int xp_shifted) {
  return p.periodic_x ? wrap(xp_shifted, p.Nx) : xp_shifted;
}

// x of the node whose density the Laplacian of the Korteweg force (Eq. FK)
// reads at interior coordinate gx: gx itself, or its mirror image across a
// wall face when gx is a ghost column of that face (the wall is a symmetry
// plane of the capillary terms)
__host__ __device__ __forceinline__ int wall_mirror(const Params& p, int gx) {
  if (gx < 0 && p.bc_lo == LBM_BC_WALL) return -1 - gx;
  if (gx >= p.Nx && p.bc_hi == LBM_BC_WALL) return 2 * p.Nx - 1 - gx;
  return gx;
}

// decode a linear index over [xlo, xhi) x Ny x Nz (padded x)
__device__ __forceinline__ bool decode(const Params& p, long long gid, int xlo, int xhi, int& xp, int& y, int& z) {
  const int nx = xhi - xlo;
  const long long n = (long long)nx * p.Ny * p.Nz;
  if (gid >= n) return false;
  xp = xlo + int(gid % nx);
  long long r = gid / nx;
  y = int(r % p.Ny);
  z = int(r / p.Ny);
  return true;
}

// Primitive state at interior coordinate (x, y, z) extended by the x-face
// rules: inflow faces give their prescribed state, outflow faces the nearest
// interior node, wall faces the nearest interior node's density with the
// wall's velocity and temperature, periodic wraps.  rho, u (D planes), T:
// interior FP64 fields.
template <int D>
__device__ inline void prim_ext(const Params& p, const double* rho, const double* u, const double* T,
                                int x, int y, int z, double& r, double* uu, double& t) {
  const long long N = (long long)p.Nx * p.Ny * p.Nz;
  const double* st = nullptr;
  const double* wall = nullptr;
  if (p.periodic_x) {
    x = wrap(x, p.Nx);
  } else if (x < 0) {
    if (p.bc_lo == LBM_BC_INFLOW) st = p.st_lo; else x = 0;
    if (p.bc_lo == LBM_BC_WALL) wall = p.st_lo;
  } else if (x >= p.Nx) {
    if (p.bc_hi == LBM_BC_INFLOW) st = p.st_hi; else x = p.Nx - 1;
    if (p.bc_hi == LBM_BC_WALL) wall = p.st_hi;
  }
  if (st) {
    r = st[0];
    for (int a = 0; a < D; ++a) uu[a] = st[1 + a];
    t = st[4];
    return;
  }
  const long long n = x + (long long)p.Nx * (y + (long long)p.Ny * z);
  r = rho[n];
  for (int a = 0; a < D; ++a) uu[a] = wall ? wall[1 + a] : u[a * N + n];
  t = wall ? wall[4] : T[n];
}

// ---------------------------------------------------------------------------
// initialisation: pulled value at every node used by a step = equilibrium of
// the (extended) initial primitive state there (Fig. FlowChart, Initialize).
// Thread per source node x in [-G-1, Nx+G] (bounded) or [0, Nx) (periodic);
// writes A_i(x - c_i) = eq_i(x), which is what node x - c_i + c_i = x pulls.
// ---------------------------------------------------------------------------
// (Params as a grid constant: prim_ext takes the address of its inflow state,
// which would otherwise copy the whole parameter block to local memory)
template <int D, typename S>
__global__ void k_init(const __grid_constant__ Params p, typename Store<S>::T* A, const double* rho, const double* u,
                       const double* T) {
  using L = Lattice<D>;
  const int xlo = p.periodic_x ? 0 : -p.G - 1;
  const int xhi = p.periodic_x ? p.Nx : p.Nx + p.G + 1;
  int x, y, z;
  if (!decode(p, blockIdx.x * (long long)blockDim.x + threadIdx.x, xlo, xhi, x, y, z)) return;
  double r, uu[D], t;
  prim_ext<D>(p, rho, u, T, x, y, z, r, uu, t);
  Model<double> m = model_of<double>(p);
  double feq[L::Q], geq[L::Q];
  equilibria<D, double>(m, r, uu, t, feq, geq);
  const int NxP = p.Nx + 2 * p.G;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    int xs = x - L::c(i, 0) + p.G;
    if (p.periodic_x) xs = wrap(xs, p.Nx);
    else if (xs < 0 || xs >= NxP) continue;
    const int ys = wrap(y - L::c(i, 1), p.Ny);
    const int zs = D == 3 ? wrap(z - L::c(i, 2), p.Nz) : z;
    const long long o = node_off(p, xs, ys, zs);
    if (pop_ok(p, A, i * p.plane + o)) Store<S>::template st<double>(A, i * p.plane + o, feq[i], p.ref[i]);
    if (pop_ok(p, A, (L::Q + i) * p.plane + o))
      Store<S>::template st<double>(A, (L::Q + i) * p.plane + o, geq[i], p.ref[L::Q + i]);
  }
}

// pulled populations of node (xp, y, z): 2Q values, f then g
template <int D, typename S, typename real>
__device__ __forceinline__ void pull(const Params& p, const typename Store<S>::T* A, int xp, int y, int z, real* fg) {
  using L = Lattice<D>;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int xs = xpad(p, xp - L::c(i, 0));
    const int ys = wrap(y - L::c(i, 1), p.Ny);
    const int zs = D == 3 ? wrap(z - L::c(i, 2), p.Nz) : z;
    const long long o = node_off(p, xs, ys, zs);
    fg[i] = pop_ok(p, A, i * p.plane + o) ? Store<S>::template ld<real>(A, i * p.plane + o, p.ref[i]) : real(0);
    fg[L::Q + i] = pop_ok(p, A, (L::Q + i) * p.plane + o)
                       ? Store<S>::template ld<real>(A, (L::Q + i) * p.plane + o, p.ref[L::Q + i])
                       : real(0);
  }
}

// x range (padded) of the moment region: radius 3 beyond the interior
__host__ __device__ inline void moment_range(const Params& p, int r, int& lo, int& hi) {
  if (p.periodic_x) { lo = 0; hi = p.Nx; }
  else { lo = p.G - r; hi = p.G + p.Nx + r; }
}

// ---------------------------------------------------------------------------
// pass 1: moments rho, j = sum c f, S = sum g (Eqs. def_h, def_u, def_E) of
// the pulled populations, on the interior plus 3 ghost layers.
// M planes: rho, j_0..j_{D-1}, S   (each p.plane elements, padded layout)
// ---------------------------------------------------------------------------
template <int D, typename S, typename real>
__global__ void k_moments(Params p, const typename Store<S>::T* A, real* M) {
  using L = Lattice<D>;
  int lo, hi;
  moment_range(p, 3, lo, hi);
  int xp, y, z;
  if (!decode(p, blockIdx.x * (long long)blockDim.x + threadIdx.x, lo, hi, xp, y, z)) return;
  real fg[2 * L::Q];
  pull<D, S, real>(p, A, xp, y, z, fg);
  real rho = 0, j[D], Se = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    rho += fg[i];
    Se += fg[L::Q + i];
  }
  first_moment<D, real>(fg, j);
  const long long o = node_off(p, xp, y, z);
  M[o] = rho;
  for (int a = 0; a < D; ++a) M[(1 + a) * p.plane + o] = j[a];
  M[(1 + D) * p.plane + o] = Se;
}

// neighbour offset along axis a by s (wrapping periodic axes)
__device__ __forceinline__ long long nb_off(const Params& p, int xp, int y, int z, int a, int s) {
  if (a == 0) return node_off(p, xpad(p, xp + s), y, z);
  if (a == 1) return node_off(p, xp, wrap(y + s, p.Ny), z);
  return node_off(p, xp, y, wrap(z + s, p.Nz));
}

// compact Laplacian of rho at (xp, y, z); ghost columns of a wall face read
// their mirror image (wall_mirror)
template <int D, typename real>
__device__ __forceinline__ real lap_rho(const Params& p, const real* rho, int xp, int y, int z) {
  const int xc = wall_mirror(p, xp - p.G) + p.G;
  const real c = rho[node_off(p, xc, y, z)];
  const int xr = wall_mirror(p, xpad(p, xp + 1) - p.G) + p.G, xl = wall_mirror(p, xpad(p, xp - 1) - p.G) + p.G;
  real l = rho[node_off(p, xr, y, z)] - real(2) * c + rho[node_off(p, xl, y, z)];
#pragma unroll
  for (int a = 1; a < D; ++a) l += rho[nb_off(p, xc, y, z, a, 1)] - real(2) * c + rho[nb_off(p, xc, y, z, a, -1)];
  return l;
}

__device__ __forceinline__ void shift(const Params& p, int& xp, int& y, int& z, int a, int s) {
  if (a == 0) xp = xpad(p, xp + s);
  else if (a == 1) y = wrap(y + s, p.Ny);
  else z = wrap(z + s, p.Nz);
}

// ---------------------------------------------------------------------------
// pass 2: Korteweg force and primitive fields on interior + 1 ghost layer.
// W planes: u_0..u_{D-1}, T, h, Lam_0..Lam_{D-1}, F_0..F_{D-1}
// ---------------------------------------------------------------------------
template <int D, typename real>
__global__ void k_prims(Params p, const real* M, real* W) {
  int lo, hi;
  moment_range(p, 1, lo, hi);
  int xp, y, z;
  if (!decode(p, blockIdx.x * (long long)blockDim.x + threadIdx.x, lo, hi, xp, y, z)) return;
  Model<real> m = model_of<real>(p);
  const long long o = node_off(p, xp, y, z);
  const real rho = M[o];
  real F[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    int x1 = xp, y1 = y, z1 = z, x2 = xp, y2 = y, z2 = z;
    shift(p, x1, y1, z1, a, 1);
    shift(p, x2, y2, z2, a, -1);
    F[a] = m.kappa * rho * real(0.5) * (lap_rho<D, real>(p, M, x1, y1, z1) - lap_rho<D, real>(p, M, x2, y2, z2));  // Eq. FK
  }
  real u[D], uF = 0, u2 = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    u[a] = div_rn(M[(1 + a) * p.plane + o] + real(0.5) * F[a], rho);                // Eq. def_u
    uF += u[a] * F[a];
    u2 += u[a] * u[a];
  }
  const real E = div_rn(M[(1 + D) * p.plane + o] + real(0.5) * uF, rho);           // Eq. def_E
  real T, P, h;
  // p.t64: the temperature inversion in FP64 from the FP32 moments (as the
  // fused step's T64 closures)
  const bool t64 = sizeof(real) == 4 && p.t64;
  if (m.kind == LBM_EOS_PR) {   // the caloric relation inverted for T; h = e + P/rho
    real e;
    if (t64) {
      const double ed = double(E) - 0.5 * double(u2);
      e = real(ed);
      T = pr_temperature_q(m, rho, ed);
    } else {
      e = E - real(0.5) * u2;
      T = eos_temperature(m, rho, e);
    }
    P = pr_pressure(m, rho, T);
    h = e + P / rho;
  } else {
    if constexpr (sizeof(real) == 4) {
      if (t64) {
        real e;
        T = vdw_temperature_fp64(p.a, 1.0 / p.cv, rho, E, u2, e);
      } else {
        T = (E - real(0.5) * u2 + m.a * rho) / m.cv;                                // Eq. lbm_temp
      }
    } else {
      T = (E - real(0.5) * u2 + m.a * rho) / m.cv;                                  // Eq. lbm_temp
    }
    P = vdw_pressure(m, rho, T);
    h = vdw_energy(m, rho, T) + P / rho;                                             // Eq. enthalpy
  }
  const real theta = P / rho;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    W[a * p.plane + o] = u[a];
    W[(D + 2 + a) * p.plane + o] = rho * u[a] * u[a] * u[a] + real(3) * rho * u[a] * (theta - real(1.0 / 3.0));
    W[(2 * D + 2 + a) * p.plane + o] = F[a];
  }
  W[D * p.plane + o] = T;
  W[(D + 1) * p.plane + o] = h;
}

// ---------------------------------------------------------------------------
// pass 3: derivatives and collision of every interior node (Eqs. fLBGK,
// gLBGK), written to dst at the node (pull scheme).
// ---------------------------------------------------------------------------
template <int D, typename S, typename real>
__global__ void k_collide(Params p, const typename Store<S>::T* A, typename Store<S>::T* B, const real* M,
                          const real* W, unsigned* err) {
  using L = Lattice<D>;
  int xp, y, z;
  if (!decode(p, blockIdx.x * (long long)blockDim.x + threadIdx.x, p.G, p.G + p.Nx, xp, y, z)) return;
  Model<real> m = model_of<real>(p);
  real fg[2 * L::Q];
  pull<D, S, real>(p, A, xp, y, z, fg);
  const long long o = node_off(p, xp, y, z);
  NodeState<D, real> s;
  s.rho = M[o];
  s.T = W[D * p.plane + o];
  s.P = eos_pressure(m, s.rho, s.T);
  s.cs2 = eos_cs2(m, s.rho, s.T);
  s.e = eos_energy(m, s.rho, s.T);
  s.sc = p.sc_on != 0;
  s.mu_num = s.eta_num = s.k_num = real(0);
  if (s.sc) {
    const real* V = static_cast<const real*>(p.sc_visc);
    s.mu_num = V[o];
    s.eta_num = V[p.plane + o];
    s.k_num = V[2 * p.plane + o];
  }
  s.div_u = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    s.u[a] = W[a * p.plane + o];
    s.F[a] = W[(2 * D + 2 + a) * p.plane + o];
    const long long op = nb_off(p, xp, y, z, a, 1), om = nb_off(p, xp, y, z, a, -1);
    s.div_u += real(0.5) * (W[a * p.plane + op] - W[a * p.plane + om]);
    s.gradT[a] = real(0.5) * (W[D * p.plane + op] - W[D * p.plane + om]);
    s.gradh[a] = real(0.5) * (W[(D + 1) * p.plane + op] - W[(D + 1) * p.plane + om]);
    const real lc = W[(D + 2 + a) * p.plane + o];
    const real back = lc - W[(D + 2 + a) * p.plane + om];
    const real fwd = W[(D + 2 + a) * p.plane + op] - lc;
    // upwind-biased difference (Sec. 3.2): sgn(u) picks the side, sgn(0) = 0 averages
    s.dLam[a] = s.u[a] > real(0) ? back : (s.u[a] < real(0) ? fwd : real(0.5) * (back + fwd));
  }
  const unsigned fl = collide_node<D, real>(m, s, fg, fg + L::Q);
  if (fl) atomicOr(err, fl);
#pragma unroll
  for (int i = 0; i < 2 * L::Q; ++i)
    if (pop_ok(p, B, i * p.plane + o)) Store<S>::template st<real>(B, i * p.plane + o, fg[i], p.ref[i]);
}

// ---------------------------------------------------------------------------
// ghost fill of the post-collision buffer (non-periodic x only), one ghost
// node (layer g of the 2G, row y, z): inflow faces get the stored equilibria
// of their state, outflow faces copy the nearest interior node, wall faces
// re-emit the mass that the nearest interior node sends into the wall with
// the equilibrium of the wall (diffuse reflection): s f^eq, s g^eq at
// (rho_e, u_wall, T_wall), rho_e that node's density, s = (its f with c_x
// towards the wall) / (the f^eq with c_x away from it).  Reads only the
// interior nodes next to the faces, so ghost nodes may be filled in any order.
// ---------------------------------------------------------------------------
template <int D, typename S>
__device__ inline void ghost_node(const Params& p, typename Store<S>::T* B, int g, int y, int z) {
  using L = Lattice<D>;
  const bool low = g < p.G;
  const int xp = low ? g : p.Nx + g;
  const int bc = low ? p.bc_lo : p.bc_hi;
  const long long o = node_off(p, xp, y, z);
  const long long os = node_off(p, low ? p.G : p.G + p.Nx - 1, y, z);
  if (bc == LBM_BC_WALL) {
    const int towards = low ? -1 : 1;
    double rho_e = 0.0, into = 0.0;
    for (int i = 0; i < L::Q; ++i) {
      const double v = pop_ok(p, B, i * p.plane + os) ? Store<S>::template ld<double>(B, i * p.plane + os, p.ref[i])
                                                       : 0.0;
      rho_e += v;
      if (L::c(i, 0) == towards) into += v;
    }
    const double* st = low ? p.st_lo : p.st_hi;
    double uw[D], feq[L::Q], geq[L::Q];
    for (int a = 0; a < D; ++a) uw[a] = st[1 + a];
    equilibria<D, double>(model_of<double>(p), rho_e, uw, st[4], feq, geq);
    double out = 0.0;
    for (int i = 0; i < L::Q; ++i)
      if (L::c(i, 0) == -towards) out += feq[i];
    const double s = into / out;
    for (int i = 0; i < L::Q; ++i) {
      if (pop_ok(p, B, i * p.plane + o)) Store<S>::template st<double>(B, i * p.plane + o, s * feq[i], p.ref[i]);
      if (pop_ok(p, B, (L::Q + i) * p.plane + o))
        Store<S>::template st<double>(B, (L::Q + i) * p.plane + o, s * geq[i], p.ref[L::Q + i]);
    }
    return;
  }
  const double* eq = low ? p.eq_lo : p.eq_hi;
  for (int i = 0; i < 2 * L::Q; ++i) {
    if (!pop_ok(p, B, i * p.plane + o) || !pop_ok(p, B, i * p.plane + os)) continue;
    if (bc == LBM_BC_INFLOW) Store<S>::template st<double>(B, i * p.plane + o, eq[i], p.ref[i]);
    else B[i * p.plane + o] = B[i * p.plane + os];
  }
}

// thread per (ghost layer, y, z)
template <int D, typename S>
__global__ void k_ghosts(Params p, typename Store<S>::T* B) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = 2LL * p.G * p.Ny * p.Nz;
  if (gid >= n) return;
  const int g = int(gid % (2 * p.G));
  const long long r = gid / (2 * p.G);
  ghost_node<D, S>(p, B, g, int(r % p.Ny), int(r / p.Ny));
}

// ---------------------------------------------------------------------------
// outputs: interior rho, u, T as FP64 (interior layout) and FP64 totals
// ---------------------------------------------------------------------------
template <int D, typename real>
__global__ void k_pack(Params p, const real* M, const real* W, double* rho, double* u, double* T) {
  int xp, y, z;
  if (!decode(p, blockIdx.x * (long long)blockDim.x + threadIdx.x, p.G, p.G + p.Nx, xp, y, z)) return;
  const long long o = node_off(p, xp, y, z);
  const long long N = (long long)p.Nx * p.Ny * p.Nz;
  const long long n = (xp - p.G) + (long long)p.Nx * (y + (long long)p.Ny * z);
  if (rho) rho[n] = double(M[o]);
  if (u)
    for (int a = 0; a < D; ++a) u[a * N + n] = double(W[a * p.plane + o]);
  if (T) T[n] = double(W[D * p.plane + o]);
}

// block partials of (sum rho, sum (j + F/2), sum (S + u.F/2)) in FP64:
// warp-shuffle reduction, then one value per warp through shared memory.
template <int D, typename real>
__global__ void k_totals(Params p, const real* M, const real* W, double* partials) {
  constexpr int K = D + 2;
  double acc[K];
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  const long long n = (long long)p.Nx * p.Ny * p.Nz;
  for (long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x; gid < n;
       gid += (long long)gridDim.x * blockDim.x) {
    int xp, y, z;
    decode(p, gid, p.G, p.G + p.Nx, xp, y, z);
    const long long o = node_off(p, xp, y, z);
    acc[0] += double(M[o]);
    double uF = 0.0;
    for (int a = 0; a < D; ++a) {
      const double F = double(W[(2 * D + 2 + a) * p.plane + o]);
      acc[1 + a] += double(M[(1 + a) * p.plane + o]) + 0.5 * F;
      uF += double(W[a * p.plane + o]) * F;
    }
    acc[1 + D] += double(M[(1 + D) * p.plane + o]) + 0.5 * uF;
  }
  __shared__ double sh[32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < K; ++k) {
    double v = acc[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double v = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) v += sh[w][threadIdx.x];
    partials[blockIdx.x * K + threadIdx.x] = v;
  }
}

// fixed-order sum of the block partials (one thread per component)
template <int D>
__global__ void k_totals_final(const double* partials, int nblocks, double* totals) {
  constexpr int K = D + 2;
  const int k = threadIdx.x;
  if (k >= K) return;
  double v = 0.0;
  for (int b = 0; b < nblocks; ++b) v += partials[b * K + k];
  totals[k] = v;
}

}  // namespace lbm
