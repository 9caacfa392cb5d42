// lbm_ops.cuh - launch wrappers of one (D, storage, arithmetic) kernel set.
// Each k_*.cu translation unit instantiates one of them.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

constexpr int kBlock = 256;

inline unsigned grid_for(long long n) { return unsigned((n + kBlock - 1) / kBlock); }

template <int D, typename S, typename real> struct OpsImpl {
  using ST = typename Store<S>::T;

  static real* M(Handle& h) { return reinterpret_cast<real*>(h.scratch); }
  static real* W(Handle& h) { return reinterpret_cast<real*>(h.scratch) + (D + 2) * h.p.plane; }

  static void init(Handle& h, const double* rho, const double* u, const double* T) {
    const Params& p = h.p;
    const long long n = (long long)(p.periodic_x ? p.Nx : p.Nx + 2 * p.G + 2) * p.Ny * p.Nz;
    k_init<D, S><<<grid_for(n), kBlock, 0, h.stream>>>(p, reinterpret_cast<ST*>(h.pop[h.cur]), rho, u, T);
    h.launches += 1;
  }

  // moments + primitive fields of `src` into scratch
  static void fields(Handle& h, const void* src) {
    const Params& p = h.p;
    int lo, hi;
    moment_range(p, 3, lo, hi);
    k_moments<D, S, real><<<grid_for((long long)(hi - lo) * p.Ny * p.Nz), kBlock, 0, h.stream>>>(
        p, reinterpret_cast<const ST*>(src), M(h));
    moment_range(p, 1, lo, hi);
    k_prims<D, real><<<grid_for((long long)(hi - lo) * p.Ny * p.Nz), kBlock, 0, h.stream>>>(p, M(h), W(h));
    h.launches += 2;
  }

  static void step(Handle& h, const void* src, void* dst) {
    const Params& p = h.p;
    fields(h, src);
    k_collide<D, S, real><<<grid_for((long long)p.Nx * p.Ny * p.Nz), kBlock, 0, h.stream>>>(
        p, reinterpret_cast<const ST*>(src), reinterpret_cast<ST*>(dst), M(h), W(h), h.err_dev);
    h.launches += 1;
    if (!p.periodic_x) {
      k_ghosts<D, S><<<grid_for(2LL * p.G * p.Ny * p.Nz), kBlock, 0, h.stream>>>(p, reinterpret_cast<ST*>(dst));
      h.launches += 1;
    }
  }

  static void macro(Handle& h, const void* src, double* rho, double* u, double* T, double* totals) {
    const Params& p = h.p;
    fields(h, src);
    const long long n = (long long)p.Nx * p.Ny * p.Nz;
    if (rho || u || T) {
      k_pack<D, real><<<grid_for(n), kBlock, 0, h.stream>>>(p, M(h), W(h), rho, u, T);
      h.launches += 1;
    }
    if (totals) {
      int nb = int((n + kBlock - 1) / kBlock);
      if (nb > kMaxPartials) nb = kMaxPartials;
      k_totals<D, real><<<nb, kBlock, 0, h.stream>>>(p, M(h), W(h), h.partials);
      k_totals_final<D><<<1, 32, 0, h.stream>>>(h.partials, nb, totals);
      h.launches += 2;
    }
  }

  static size_t scratch_bytes(const Params& p) { return size_t(4 * D + 4) * size_t(p.plane) * sizeof(real); }

  static const Ops* ops() {
    static const Ops o = {&init, &step, &macro};
    return &o;
  }
};

}  // namespace lbm
