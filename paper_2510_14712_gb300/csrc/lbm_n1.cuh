// lbm_n1.cuh - shock-capturing numerical transport coefficients (Sec. 4.4,
// Eqs. shock_cap and shock_cap_k), computed after each step from that step's
// primitive fields and used by the next step's collision:
//
//   {mu, eta}^num = rho C_{mu,eta} F(|grad^4 S|),  k^num = rho c_s C_k F(|grad^4 |grad s||)
//
// with S = |grad u + grad u^T| / 2, grad s = (c_v/T) grad T - R/(rho (1 - b rho)) grad rho
// (van der Waals; the general identity for Peng-Robinson), |grad^4 f| =
// sqrt(sum_a (d_a^4 f)^2) over the per-axis five-point fourth differences
// (r = 5, delta x^(r+1) = 1), F the separable binomial filter (1, 4, 6, 4, 1)/16
// along every axis, c_s the fluid's sound speed at (rho, T).  Neighbours wrap
// on periodic axes and are clamped to the nearest interior node on
// non-periodic x faces.  Fields live on the padded plane layout of the handle
// (offset (z Ny + y) pitch + x + G, one plane per component).  Three forms
// share the per-node arithmetic: 2-D tiles in shared memory (two launches),
// row-mapped launches in 3-D (D + 2), and one block per row for batches.
#pragma once

#include "lbm_fused.cuh"

namespace lbm {

// v mod n for a shift of at most a few nodes: one comparison in range
__device__ __forceinline__ int n1_wrap(int v, int n) { return unsigned(v) < unsigned(n) ? v : modp(v, n); }

// Values a stage computes at one node, stored to K planes of its output.
template <typename real, int K> struct N1Vals {
  real v[K];
};

template <typename real, int K>
__device__ __forceinline__ void n1_store(const Params& p, real* out, unsigned o, const N1Vals<real, K>& r) {
#pragma unroll
  for (int k = 0; k < K; ++k) out[k * p.plane + o] = r.v[k];
}

// Thread layout of the stencil kernels: threads along x, blocks along x and over
// groups of kN1Rows consecutive rows (y, z), each block walking groups gridDim.y
// apart.  f(x, y, z, o) computes the values of every interior node of the
// thread, o its element offset in a plane (a plane holds fewer than 2^31
// elements: the buffers of a handle stay below 2^32 elements, checked at
// create).  The values of a whole group are computed before any is stored, so
// that the loads of its rows can all be in flight together (the compiler
// cannot move a load across a store to a pointer it cannot tell apart).
constexpr int kN1Rows = 4;
template <int K, typename real, class F>
__device__ __forceinline__ void n1_rows(const Params& p, real* out, F&& f) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.Nx) return;
  const int rows = p.Ny * p.Nz;
  auto off = [&](const int row) { return unsigned(row) * unsigned(p.pitch) + unsigned(x + p.G); };
  for (int r0 = blockIdx.y * kN1Rows; r0 < rows; r0 += gridDim.y * kN1Rows) {
    if (r0 + kN1Rows <= rows) {
      N1Vals<real, K> res[kN1Rows];
#pragma unroll
      for (int r = 0; r < kN1Rows; ++r) res[r] = f(x, (r0 + r) % p.Ny, (r0 + r) / p.Ny, off(r0 + r));
#pragma unroll
      for (int r = 0; r < kN1Rows; ++r) n1_store(p, out, off(r0 + r), res[r]);
    } else {
      for (int row = r0; row < rows; ++row) n1_store(p, out, off(row), f(x, row % p.Ny, row / p.Ny, off(row)));
    }
  }
}

// offset of the interior neighbour (x, y, z) + s e_a of the node at offset o:
// wrapped on periodic axes, clamped to the nearest interior node on a
// non-periodic x
__device__ __forceinline__ unsigned n1_nb(const Params& p, int x, int y, int z, unsigned o, int a, int s) {
  if (a == 0) {
    int xs = x + s;
    xs = p.periodic_x ? n1_wrap(xs, p.Nx) : (xs < 0 ? 0 : (xs >= p.Nx ? p.Nx - 1 : xs));
    return o + unsigned(xs - x);
  }
  if (a == 1) return o + unsigned((n1_wrap(y + s, p.Ny) - y) * p.pitch);
  return o + unsigned((n1_wrap(z + s, p.Nz) - z) * p.Ny * p.pitch);
}

// ---- per-node stages (shared by the single-instance and batched kernels) ----
// No stage reads a buffer it writes, so every input goes through the read-only
// path (__ldg).  Each returns its values; the caller stores them.

template <typename real> __device__ __forceinline__ real n1_ld(const real* q) { return __ldg(q); }

// five-point fourth difference and binomial (1, 4, 6, 4, 1)/16 of the values at
// offsets -2 .. +2 along one axis, and the coefficients from the filtered norms
// (one definition for the row-mapped and the tiled forms)
template <typename real>
__device__ __forceinline__ real n1_fourth(real vm2, real vm1, real v0, real vp1, real vp2) {
  return vp2 - real(4) * vp1 + real(6) * v0 - real(4) * vm1 + vm2;
}
template <typename real>
__device__ __forceinline__ real n1_binom5(real vm2, real vm1, real v0, real vp1, real vp2) {
  return (vm2 + real(4) * vm1 + real(6) * v0 + real(4) * vp1 + vp2) / real(16);
}
template <typename real>
__device__ __forceinline__ N1Vals<real, 3> n1_coefs(const Params& p, const Model<real>& m, real r, real t, real s4,
                                                    real g4) {
  const real cs2 = eos_cs2(m, r, t);
  const real cs = sqrt(cs2 > real(0) ? cs2 : real(0));
  return {{r * real(p.sc_c[0]) * s4, r * real(p.sc_c[1]) * s4, r * cs * real(p.sc_c[2]) * g4}};
}

// S and |grad s| at the node
template <int D, typename real>
__device__ __forceinline__ N1Vals<real, 2> n1_strain_at(const Params& p, const real* __restrict__ rho,
                                                        const real* __restrict__ u, const real* __restrict__ T,
                                                        int x, int y, int z, unsigned o) {
  unsigned op[D], om[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    op[a] = n1_nb(p, x, y, z, o, a, 1);
    om[a] = n1_nb(p, x, y, z, o, a, -1);
  }
  real g[D][D];                                    // g[a][b] = d_a u_b (central)
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b)
      g[a][b] = real(0.5) * (n1_ld(u + b * p.plane + op[a]) - n1_ld(u + b * p.plane + om[a]));
  real acc = real(0);
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) acc += (g[a][b] + g[b][a]) * (g[a][b] + g[b][a]);
  const real S = real(0.5) * sqrt(acc);
  const real r = n1_ld(rho + o), t = n1_ld(T + o);
  real cT, cR;
  if (p.eos_kind == LBM_EOS_PR) {
    eos_entropy_coefs(model_of<real>(p), r, t, cT, cR);
  } else {
    cR = real(p.R) / (r * (real(1) - real(p.b) * r));
    cT = real(p.cv) / t;
  }
  real gs2 = real(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const real gT = real(0.5) * (n1_ld(T + op[a]) - n1_ld(T + om[a]));
    const real gr = real(0.5) * (n1_ld(rho + op[a]) - n1_ld(rho + om[a]));
    const real gs = cT * gT - cR * gr;
    gs2 += gs * gs;
  }
  return {{S, sqrt(gs2)}};
}

// norm of the per-axis fourth differences of the two fields of `in` at the node
template <int D, typename real>
__device__ __forceinline__ N1Vals<real, 2> n1_d4_at(const Params& p, const real* __restrict__ in, int x, int y, int z,
                                                    unsigned o) {
  unsigned nb[D][4];                               // offsets of the -2, -1, +1, +2 neighbours along a
#pragma unroll
  for (int a = 0; a < D; ++a) {
    nb[a][0] = n1_nb(p, x, y, z, o, a, -2);
    nb[a][1] = n1_nb(p, x, y, z, o, a, -1);
    nb[a][2] = n1_nb(p, x, y, z, o, a, 1);
    nb[a][3] = n1_nb(p, x, y, z, o, a, 2);
  }
  N1Vals<real, 2> res;
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    const real* v = in + f * p.plane;
    real acc = real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const real d4 = n1_fourth(n1_ld(v + nb[a][0]), n1_ld(v + nb[a][1]), n1_ld(v + o), n1_ld(v + nb[a][2]),
                                n1_ld(v + nb[a][3]));
      acc += d4 * d4;
    }
    res.v[f] = sqrt(acc);
  }
  return res;
}

// binomial (1, 4, 6, 4, 1)/16 along axis a of field f of `in` at the node
template <typename real>
__device__ __forceinline__ real n1_binomial(const Params& p, const real* __restrict__ in, int f, int a, int x, int y,
                                            int z, unsigned o) {
  const unsigned m2 = n1_nb(p, x, y, z, o, a, -2), m1 = n1_nb(p, x, y, z, o, a, -1);
  const unsigned p1 = n1_nb(p, x, y, z, o, a, 1), p2 = n1_nb(p, x, y, z, o, a, 2);
  const real* v = in + f * p.plane;
  return n1_binom5(n1_ld(v + m2), n1_ld(v + m1), n1_ld(v + o), n1_ld(v + p1), n1_ld(v + p2));
}

template <typename real>
__device__ __forceinline__ N1Vals<real, 2> n1_filter_at(const Params& p, int a, const real* __restrict__ in, int x,
                                                        int y, int z, unsigned o) {
  return {{n1_binomial(p, in, 0, a, x, y, z, o), n1_binomial(p, in, 1, a, x, y, z, o)}};
}

// the last filter pass (along axis D-1) and the coefficients from the filtered
// norms: mu, eta, k numerical (the three planes of visc)
template <int D, typename real>
__device__ __forceinline__ N1Vals<real, 3> n1_filter_coef_at(const Params& p, const Model<real>& m,
                                                             const real* __restrict__ in, const real* __restrict__ rho,
                                                             const real* __restrict__ T, int x, int y, int z,
                                                             unsigned o) {
  const real s4 = n1_binomial(p, in, 0, D - 1, x, y, z, o), g4 = n1_binomial(p, in, 1, D - 1, x, y, z, o);
  return n1_coefs(p, m, n1_ld(rho + o), n1_ld(T + o), s4, g4);
}

// Buffers of one handle's shock capturing: the step's rho, u (D planes), T (by
// default the fused step's copy in sc_prims), the coefficients (3 planes)
// followed by the work planes w0, w1 (2 each).  The stages run strain -> w0,
// fourth differences w0 -> w1, filter passes alternating w1 -> w0 -> w1 ...,
// the last pass with the coefficients.
template <int D, typename real> struct N1Buffers {
  const real *rho, *u, *T;
  real *visc, *w0, *w1;
  __host__ __device__ N1Buffers(const Params& p, const real* rho_, const real* u_, const real* T_)
      : rho(rho_), u(u_), T(T_) {
    visc = static_cast<real*>(const_cast<void*>(p.sc_visc));
    w0 = visc + 3 * p.plane;
    w1 = w0 + 2 * p.plane;
  }
  __host__ __device__ explicit N1Buffers(const Params& p)
      : N1Buffers(p, static_cast<const real*>(p.sc_prims), static_cast<const real*>(p.sc_prims) + p.plane,
                  static_cast<const real*>(p.sc_prims) + (1 + D) * p.plane) {}
  // input of filter pass a (a = D - 1: the pass fused with the coefficients)
  __host__ __device__ const real* filter_in(int a) const { return a % 2 == 0 ? w1 : w0; }
  __host__ __device__ real* filter_out(int a) const { return a % 2 == 0 ? w0 : w1; }
};

// ---- single-instance kernels ----

template <int D, typename real>
__global__ void k_n1_strain(Params p, const real* __restrict__ rho, const real* __restrict__ u,
                            const real* __restrict__ T) {
  const N1Buffers<D, real> b(p, rho, u, T);
  n1_rows<2>(p, b.w0,
             [&](int x, int y, int z, unsigned o) { return n1_strain_at<D, real>(p, b.rho, b.u, b.T, x, y, z, o); });
}

template <int D, typename real> __global__ void k_n1_d4(Params p) {
  const N1Buffers<D, real> b(p);
  n1_rows<2>(p, b.w1, [&](int x, int y, int z, unsigned o) { return n1_d4_at<D, real>(p, b.w0, x, y, z, o); });
}

template <int D, typename real> __global__ void k_n1_filter(Params p, int a) {
  const N1Buffers<D, real> b(p);
  n1_rows<2>(p, b.filter_out(a),
             [&](int x, int y, int z, unsigned o) { return n1_filter_at<real>(p, a, b.filter_in(a), x, y, z, o); });
}

template <int D, typename real>
__global__ void k_n1_filter_coef(Params p, const real* __restrict__ rho, const real* __restrict__ T) {
  const N1Buffers<D, real> b(p, rho, nullptr, T);
  const Model<real> m = model_of<real>(p);
  n1_rows<3>(p, b.visc, [&](int x, int y, int z, unsigned o) {
    return n1_filter_coef_at<D, real>(p, m, b.filter_in(D - 1), b.rho, b.T, x, y, z, o);
  });
}

// ---- 2-D single-instance form: two launches over tiles of the plane ----
// A block owns kN1TileX x kN1TileY nodes (threads along x) and walks tiles
// gridDim.y apart along y.  The strain launch evaluates S and |grad s| on the
// tile and a two-node halo into shared memory and takes the fourth
// differences there; the filter launch runs the x pass on the tile's columns
// and a two-row halo, then the y pass with the coefficients.  Halo positions
// take the values of the node the row-mapped stencils read there: x wrapped
// on a periodic x, clamped to the nearest interior node otherwise; y wrapped.
// The arithmetic of every value is that of the per-node stages above.
constexpr int kN1TileX = 128, kN1TileY = 16;
constexpr int kN1HX = kN1TileX + 4, kN1HY = kN1TileY + 4;

// x of the node whose values a stencil reads at x (any integer)
__device__ __forceinline__ int n1_xsrc(const Params& p, int x) {
  return p.periodic_x ? modp(x, p.Nx) : (x < 0 ? 0 : (x >= p.Nx ? p.Nx - 1 : x));
}

template <typename real>
__global__ void __launch_bounds__(kN1TileX)
k_n1_strain_d4_2d(Params p, const real* __restrict__ rho, const real* __restrict__ u, const real* __restrict__ T) {
  __shared__ real sv[2][kN1HY][kN1HX];             // S, |grad s| on the tile and its halo
  const N1Buffers<2, real> b(p, rho, u, T);
  const unsigned pitch = unsigned(p.pitch);
  const int x0 = blockIdx.x * kN1TileX, tx = threadIdx.x;
  const int ntile = (p.Ny + kN1TileY - 1) / kN1TileY;
  for (int ty = blockIdx.y; ty < ntile; ty += gridDim.y) {
    const int y0 = ty * kN1TileY;
#pragma unroll 4
    for (int k = tx; k < kN1HX * kN1HY; k += kN1TileX) {
      const int hx = k % kN1HX, hy = k / kN1HX;
      const int xs = n1_xsrc(p, x0 + hx - 2), ys = modp(y0 + hy - 2, p.Ny);
      const N1Vals<real, 2> v =
          n1_strain_at<2, real>(p, b.rho, b.u, b.T, xs, ys, 0, unsigned(ys) * pitch + unsigned(xs + p.G));
      sv[0][hy][hx] = v.v[0];
      sv[1][hy][hx] = v.v[1];
    }
    __syncthreads();
    const int x = x0 + tx, hx = tx + 2;
    if (x < p.Nx) {
      for (int r = 0; r < kN1TileY && y0 + r < p.Ny; ++r) {
        const int hy = r + 2;
        N1Vals<real, 2> res;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          const real(*v)[kN1HX] = sv[f];
          real acc = real(0);                        // axis x, then y (n1_d4_at)
          const real dx = n1_fourth(v[hy][hx - 2], v[hy][hx - 1], v[hy][hx], v[hy][hx + 1], v[hy][hx + 2]);
          acc += dx * dx;
          const real dy = n1_fourth(v[hy - 2][hx], v[hy - 1][hx], v[hy][hx], v[hy + 1][hx], v[hy + 2][hx]);
          acc += dy * dy;
          res.v[f] = sqrt(acc);
        }
        n1_store(p, b.w1, unsigned(y0 + r) * pitch + unsigned(x + p.G), res);
      }
    }
    __syncthreads();                                 // the next tile overwrites sv
  }
}

template <typename real>
__global__ void __launch_bounds__(kN1TileX)
k_n1_filter_coef_2d(Params p, const real* __restrict__ rho, const real* __restrict__ T) {
  __shared__ real sf[2][kN1HY][kN1TileX];          // x-filtered norms; each thread reads only its own column
  const N1Buffers<2, real> b(p, rho, nullptr, T);
  const Model<real> m = model_of<real>(p);
  const unsigned pitch = unsigned(p.pitch);
  const int tx = threadIdx.x, x = blockIdx.x * kN1TileX + tx;
  if (x >= p.Nx) return;
  const int ntile = (p.Ny + kN1TileY - 1) / kN1TileY;
  for (int ty = blockIdx.y; ty < ntile; ty += gridDim.y) {
    const int y0 = ty * kN1TileY;
#pragma unroll 4
    for (int hy = 0; hy < kN1HY; ++hy) {
      const int ys = modp(y0 + hy - 2, p.Ny);
      const N1Vals<real, 2> v = n1_filter_at<real>(p, 0, b.w1, x, ys, 0, unsigned(ys) * pitch + unsigned(x + p.G));
      sf[0][hy][tx] = v.v[0];
      sf[1][hy][tx] = v.v[1];
    }
    for (int r = 0; r < kN1TileY && y0 + r < p.Ny; ++r) {
      const int hy = r + 2;
      // y pass, then the coefficients (as n1_filter_coef_at)
      const real s4 =
          n1_binom5(sf[0][hy - 2][tx], sf[0][hy - 1][tx], sf[0][hy][tx], sf[0][hy + 1][tx], sf[0][hy + 2][tx]);
      const real g4 =
          n1_binom5(sf[1][hy - 2][tx], sf[1][hy - 1][tx], sf[1][hy][tx], sf[1][hy + 1][tx], sf[1][hy + 2][tx]);
      const unsigned o = unsigned(y0 + r) * pitch + unsigned(x + p.G);
      n1_store(p, b.visc, o, n1_coefs(p, m, n1_ld(b.rho + o), n1_ld(b.T + o), s4, g4));
    }
  }
}

// The whole update of a handle's coefficients from the step's rho, u (D planes),
// T (padded plane layout): 2 launches in 2-D, D + 2 in 3-D.
template <int D, typename real>
inline int n1_update(const Params& p, cudaStream_t st, const real* rho, const real* u, const real* T) {
  if constexpr (D == 2) {
    const int ntile = (p.Ny + kN1TileY - 1) / kN1TileY;
    const dim3 grid(unsigned((p.Nx + kN1TileX - 1) / kN1TileX), unsigned(ntile < 65535 ? ntile : 65535));
    k_n1_strain_d4_2d<real><<<grid, kN1TileX, 0, st>>>(p, rho, u, T);
    k_n1_filter_coef_2d<real><<<grid, kN1TileX, 0, st>>>(p, rho, T);
    return 2;
  } else {
    const int groups = (p.Ny * p.Nz + kN1Rows - 1) / kN1Rows;
    const dim3 block(128), grid(unsigned((p.Nx + 127) / 128), unsigned(groups < 65535 ? groups : 65535));
    k_n1_strain<D, real><<<grid, block, 0, st>>>(p, rho, u, T);
    k_n1_d4<D, real><<<grid, block, 0, st>>>(p);
    for (int a = 0; a + 1 < D; ++a) k_n1_filter<D, real><<<grid, block, 0, st>>>(p, a);
    k_n1_filter_coef<D, real><<<grid, block, 0, st>>>(p, rho, T);
    return D + 2;
  }
}

// ---- batched kernels: one block per row of every instance with shock capturing ----

// rowstart[k] = first global row of instance k (prefix sum of Ny Nz over the
// instances with shock capturing on, 0 rows for the others); rowstart[n] = total
__device__ __forceinline__ int n1_instance(const int* __restrict__ rowstart, int n, int row) {
  int lo = 0, hi = n;                              // largest k < n with rowstart[k] <= row
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (rowstart[mid] <= row) lo = mid;
    else hi = mid;
  }
  return lo;
}

// stage 0: strain, 1: fourth differences, 2: filter pass a, 3: last pass + coefficients
template <int D, typename real, int STAGE>
__global__ void k_n1_batch(const BatchInstance* __restrict__ insts, const int* __restrict__ rowstart, int n, int a) {
  const int k = n1_instance(rowstart, n, blockIdx.x);
  const Params& p = insts[k].p;
  const N1Buffers<D, real> b(p);
  const int row = blockIdx.x - rowstart[k];
  const int y = row % p.Ny, z = row / p.Ny;
  const Model<real> m = model_of<real>(p);
  for (int x = threadIdx.x; x < p.Nx; x += blockDim.x) {
    const unsigned o = unsigned(row) * unsigned(p.pitch) + unsigned(x + p.G);
    if constexpr (STAGE == 0) n1_store(p, b.w0, o, n1_strain_at<D, real>(p, b.rho, b.u, b.T, x, y, z, o));
    else if constexpr (STAGE == 1) n1_store(p, b.w1, o, n1_d4_at<D, real>(p, b.w0, x, y, z, o));
    else if constexpr (STAGE == 2)
      n1_store(p, b.filter_out(a), o, n1_filter_at<real>(p, a, b.filter_in(a), x, y, z, o));
    else n1_store(p, b.visc, o, n1_filter_coef_at<D, real>(p, m, b.filter_in(D - 1), b.rho, b.T, x, y, z, o));
  }
}

// the update of every instance with shock capturing on: D + 2 launches over
// `rows` global rows
template <int D, typename real>
inline int n1_update_batch(const BatchInstance* insts, const int* rowstart, int n, int rows, cudaStream_t st) {
  k_n1_batch<D, real, 0><<<rows, 128, 0, st>>>(insts, rowstart, n, 0);
  k_n1_batch<D, real, 1><<<rows, 128, 0, st>>>(insts, rowstart, n, 0);
  for (int a = 0; a + 1 < D; ++a) k_n1_batch<D, real, 2><<<rows, 128, 0, st>>>(insts, rowstart, n, a);
  k_n1_batch<D, real, 3><<<rows, 128, 0, st>>>(insts, rowstart, n, D - 1);
  return D + 2;
}

}  // namespace lbm
