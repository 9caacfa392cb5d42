// lbm_n1.cuh - shock-capturing numerical transport coefficients (Sec. 4.4,
// Eqs. shock_cap and shock_cap_k), computed after each step from that step's
// primitive fields and used by the next step's collision:
//
//   {mu, eta}^num = rho C_{mu,eta} F(|grad^4 S|),  k^num = rho c_s C_k F(|grad^4 |grad s||)
//
// with S = |grad u + grad u^T| / 2, grad s = (c_v/T) grad T - R/(rho (1 - b rho)) grad rho,
// |grad^4 f| = sqrt(sum_a (d_a^4 f)^2) over the per-axis five-point fourth
// differences (r = 5, delta x^(r+1) = 1), F the separable binomial filter
// (1, 4, 6, 4, 1)/16 along every axis, c_s the van der Waals sound speed
// at (rho, T).  Neighbours wrap on periodic axes and are clamped to the
// nearest interior node on non-periodic x faces.  Fields live on the padded
// plane layout of the handle (offset (z Ny + y) pitch + x + G, one plane per
// component); threads along x, blocks over x and the rows.
#pragma once

#include "lbm_fused.cuh"

namespace lbm {

// v mod n for a shift of at most a few nodes: one comparison in range
__device__ __forceinline__ int n1_wrap(int v, int n) { return unsigned(v) < unsigned(n) ? v : modp(v, n); }

// Thread layout of the stencil kernels: threads along x, blocks along x and over
// the rows (y, z), each block walking rows gridDim.y apart; f(x, y, z, o) for
// every interior node of the thread, o its element offset in a plane (a plane
// holds fewer than 2^31 elements: the buffers of a handle stay below 2^32
// elements, checked at create).
template <class F> __device__ __forceinline__ void n1_rows(const Params& p, F&& f) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.Nx) return;
  const int rows = p.Ny * p.Nz;
  for (int row = blockIdx.y; row < rows; row += gridDim.y)
    f(x, row % p.Ny, row / p.Ny, unsigned(row) * unsigned(p.pitch) + unsigned(x + p.G));
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

// S and |grad s| of every interior node: out[0 .. plane) = S, out[plane ..) = |grad s|
template <int D, typename real>
__global__ void k_n1_strain(Params p, const real* __restrict__ rho, const real* __restrict__ u,
                            const real* __restrict__ T, real* __restrict__ out) {
  n1_rows(p, [&](const int x, const int y, const int z, const unsigned o) {
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
      for (int b = 0; b < D; ++b) g[a][b] = real(0.5) * (u[b * p.plane + op[a]] - u[b * p.plane + om[a]]);
    real acc = real(0);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) acc += (g[a][b] + g[b][a]) * (g[a][b] + g[b][a]);
    out[o] = real(0.5) * sqrt(acc);
    const real r = rho[o], t = T[o];
    const real cR = real(p.R) / (r * (real(1) - real(p.b) * r)), cT = real(p.cv) / t;
    real gs2 = real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const real gT = real(0.5) * (T[op[a]] - T[om[a]]), gr = real(0.5) * (rho[op[a]] - rho[om[a]]);
      const real gs = cT * gT - cR * gr;
      gs2 += gs * gs;
    }
    out[p.plane + o] = sqrt(gs2);
  });
}

// norm of the per-axis fourth differences of the two fields of `in`
template <int D, typename real>
__global__ void k_n1_d4(Params p, const real* __restrict__ in, real* __restrict__ out) {
  n1_rows(p, [&](const int x, const int y, const int z, const unsigned o) {
    unsigned nb[D][4];                               // offsets of the -2, -1, +1, +2 neighbours along a
#pragma unroll
    for (int a = 0; a < D; ++a) {
      nb[a][0] = n1_nb(p, x, y, z, o, a, -2);
      nb[a][1] = n1_nb(p, x, y, z, o, a, -1);
      nb[a][2] = n1_nb(p, x, y, z, o, a, 1);
      nb[a][3] = n1_nb(p, x, y, z, o, a, 2);
    }
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const real* v = in + f * p.plane;
      real acc = real(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const real d4 = v[nb[a][3]] - real(4) * v[nb[a][2]] + real(6) * v[o] - real(4) * v[nb[a][1]] + v[nb[a][0]];
        acc += d4 * d4;
      }
      out[f * p.plane + o] = sqrt(acc);
    }
  });
}

// binomial (1, 4, 6, 4, 1)/16 along axis a of the two fields of `in`
template <int D, typename real>
__global__ void k_n1_filter(Params p, int a, const real* __restrict__ in, real* __restrict__ out) {
  n1_rows(p, [&](const int x, const int y, const int z, const unsigned o) {
    const unsigned m2 = n1_nb(p, x, y, z, o, a, -2), m1 = n1_nb(p, x, y, z, o, a, -1);
    const unsigned p1 = n1_nb(p, x, y, z, o, a, 1), p2 = n1_nb(p, x, y, z, o, a, 2);
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const real* v = in + f * p.plane;
      out[f * p.plane + o] = (v[m2] + real(4) * v[m1] + real(6) * v[o] + real(4) * v[p1] + v[p2]) / real(16);
    }
  });
}

// the last filter pass (along axis D-1) and the coefficients from the filtered
// norms in one pass: visc[0..2] planes = mu, eta, k numerical
template <int D, typename real>
__global__ void k_n1_filter_coef(Params p, const real* __restrict__ in, const real* __restrict__ rho,
                                 const real* __restrict__ T, real* __restrict__ visc) {
  const Model<real> m = model_of<real>(p);
  n1_rows(p, [&](const int x, const int y, const int z, const unsigned o) {
    constexpr int a = D - 1;
    const unsigned m2 = n1_nb(p, x, y, z, o, a, -2), m1 = n1_nb(p, x, y, z, o, a, -1);
    const unsigned p1 = n1_nb(p, x, y, z, o, a, 1), p2 = n1_nb(p, x, y, z, o, a, 2);
    real fv[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const real* v = in + f * p.plane;
      fv[f] = (v[m2] + real(4) * v[m1] + real(6) * v[o] + real(4) * v[p1] + v[p2]) / real(16);
    }
    const real r = rho[o];
    const real cs2 = vdw_cs2(m, r, T[o]);
    const real cs = sqrt(cs2 > real(0) ? cs2 : real(0));
    visc[o] = r * real(p.sc_c[0]) * fv[0];
    visc[p.plane + o] = r * real(p.sc_c[1]) * fv[0];
    visc[2 * p.plane + o] = r * cs * real(p.sc_c[2]) * fv[1];
  });
}

// the whole update of the coefficients: rho, u (D planes), T -> visc (3 planes),
// using work (4 planes); D + 2 launches
template <int D, typename real>
inline int n1_update(const Params& p, cudaStream_t st, const real* rho, const real* u, const real* T, real* visc,
                     real* work) {
  const dim3 block(128), grid(unsigned((p.Nx + 127) / 128), unsigned(p.Ny * p.Nz < 65535 ? p.Ny * p.Nz : 65535));
  real* w0 = work;
  real* w1 = work + 2 * p.plane;
  k_n1_strain<D, real><<<grid, block, 0, st>>>(p, rho, u, T, w0);
  k_n1_d4<D, real><<<grid, block, 0, st>>>(p, w0, w1);
  real* src = w1;
  real* dst = w0;
  for (int a = 0; a + 1 < D; ++a) {
    k_n1_filter<D, real><<<grid, block, 0, st>>>(p, a, src, dst);
    real* t = src;
    src = dst;
    dst = t;
  }
  k_n1_filter_coef<D, real><<<grid, block, 0, st>>>(p, src, rho, T, visc);
  return D + 2;
}

}  // namespace lbm
