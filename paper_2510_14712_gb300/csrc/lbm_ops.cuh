// lbm_ops.cuh - launch wrappers of one (D, storage, arithmetic) kernel set.
// Each k_*.cu translation unit instantiates one of them.
#pragma once

#include <type_traits>

#include <algorithm>
#include <vector>

#include "lbm_n1.cuh"

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

  // One tile shape of the fused kernel (TX x TY in-plane nodes, MINB CTAs
  // per SM for the register budget) with thermodynamic closure CL.
  template <int TX, int TY, int MINB, class CL, int OPT = 0> struct Fused {
    using FG = FusedGeom<D, TX, TY, CL::kExtra, planes_per_interval<OPT>()>;
    static size_t smem() { return FG::template smem_bytes<real>() + CL::kSmem; }
    struct Launch {
      int grid = 0, ncolx = 0, ncoly = 0, nseg = 1;
      bool small = false, rows = false;
    };
    // One CTA per (column, z-segment), never more items than resident CTA
    // slots so that all run together.  In 3-D the plane is cut into ncolx
    // columns along x and ncoly bands along y (at least ceil(Ny / TY) bands,
    // at most TY rows each); the number of bands and of z-segments (each at
    // least 16 planes long: a segment repeats 6 warm-up planes) is the one that
    // minimises the modelled time rounds x (rows per band + 1.5) x (planes per
    // segment + 6): with 256 x 256 planes and 304 slots, 38 bands of 6-7 rows
    // give every slot one column, where 32 bands of 8 rows would leave 48 slots
    // without work.
    static Launch plan(const Params& p) {
      static int blocks_per_sm = -1, sms = 0;
      if (blocks_per_sm < 0) {
        auto kern = k_step_fused<D, S, real, TX, TY, MINB, false, CL, OPT>;
        auto kern_pos = k_step_fused<D, S, real, TX, TY, MINB, false, CL, OPT & ~kOptRows>;
        auto kern_small = k_step_fused<D, S, real, TX, TY, MINB, true, CL, OPT & ~kOptRows>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
        cudaFuncSetAttribute(kern_pos, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
        cudaFuncSetAttribute(kern_small, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, FG::NT, smem());
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (blocks_per_sm < 1) blocks_per_sm = 1;
      }
      Launch l;
      l.ncolx = (p.Nx + TX - 1) / TX;
      const int Nm = D == 3 ? p.Nz : p.Ny;
      const long long slots = (long long)blocks_per_sm * sms;
      const int nb0 = D == 3 ? (p.Ny + TY - 1) / TY : 1;
      const int nb1 = D == 3 ? std::min(p.Ny, 2 * nb0) : 1;
      double best = 1e300;
      for (int nb = nb0; nb <= nb1; ++nb) {
        const long long ncol = (long long)l.ncolx * nb;
        long long nseg = slots / ncol;
        if (nseg > Nm / 16) nseg = Nm / 16;
        if (nseg < 1) nseg = 1;
        const long long items = ncol * nseg;
        const double rounds = double((items + slots - 1) / slots);
        const double rows = D == 3 ? double((p.Ny + nb - 1) / nb) : 1.0;
        const double cost = rounds * (rows + 1.5) * (double((Nm + nseg - 1) / nseg) + 6.0);
        if (cost < best * (1.0 - 1e-9)) {
          best = cost;
          l.ncoly = nb;
          l.nseg = int(nseg);
        }
      }
      long long g = (long long)l.ncolx * l.ncoly * l.nseg;
      if (g > slots) g = slots;
      l.grid = int(g);
      l.small = (p.periodic_x && p.Nx < TX + 6) || (D == 3 && p.Ny < TY + 6);
      // row form of stage A: aligned 4-node chunks (Nx and the ghost width are
      // multiples of 4), no wall face (mirror densities in stage A)
      l.rows = (OPT & kOptRows) && D == 3 && sizeof(real) == 4 && !l.small && p.Nx % 4 == 0 && p.G % 4 == 0 &&
               p.bc_lo != LBM_BC_WALL && p.bc_hi != LBM_BC_WALL;
      return l;
    }
    static void launch(Handle& h, const void* src, void* dst) {
      const Params& p = h.p;
      const Launch l = plan(p);
      auto kern = l.small ? k_step_fused<D, S, real, TX, TY, MINB, true, CL, OPT & ~kOptRows>
                          : (l.rows ? k_step_fused<D, S, real, TX, TY, MINB, false, CL, OPT>
                                    : k_step_fused<D, S, real, TX, TY, MINB, false, CL, OPT & ~kOptRows>);
      kern<<<l.grid, FG::NT, smem(), h.stream>>>(p, reinterpret_cast<const ST*>(src), reinterpret_cast<ST*>(dst),
                                                 h.err_dev, l.ncolx, l.ncoly, l.nseg);
      h.launches += 1;
    }
  };

  // Candidate tile shapes, first = default.  FP64 keeps one shape (its
  // arithmetic, not the tile, bounds it).
  using LaunchFn = void (*)(Handle&, const void*, void*);
  // The learned closure adds a register-hungry network evaluation to stage C,
  // so its list also offers the unrestricted (MINB 1) allocation.
  template <class CL> static int candidates(const LaunchFn** fns) {
    if constexpr (CL::kPr) {                                   // one shape: the Peng-Robinson sets compile fast
      static const LaunchFn c[] = {D == 3 ? &Fused<32, 8, sizeof(real) == 8 ? 1 : 2, CL, kOptRows>::launch
                                          : &Fused<256, 1, 2, CL>::launch};
      *fns = c;
      return 1;
    } else if constexpr (D == 3) {
      if constexpr (sizeof(real) == 8) {
        static const LaunchFn c[] = {&Fused<32, 8, 1, CL>::launch};
        *fns = c;
        return 1;
      } else if constexpr (CL::kWarp) {
        static const LaunchFn c[] = {&Fused<32, 8, 2, CL>::launch, &Fused<32, 8, 1, CL>::launch,
                                     &Fused<32, 16, 1, CL>::launch, &Fused<32, 8, 1, CL, kOptRows>::launch};
        *fns = c;
        return 4;
      } else {
        static const LaunchFn c[] = {&Fused<32, 8, 2, CL, kOptRows>::launch, &Fused<32, 16, 1, CL, kOptRows>::launch,
                                     &Fused<16, 16, 2, CL, kOptRows>::launch,
                                     &Fused<32, 8, 2, CL, kOptRows | kOptPair>::launch,
                                     &Fused<32, 16, 1, CL, kOptRows | kOptPair>::launch};
        *fns = c;
        return 5;
      }
    } else if constexpr (sizeof(real) == 4 && !CL::kWarp) {
      // narrow tiles spread small domains (few columns) over more SMs; the
      // 2-D FP32 body also fits 80 registers without spills, so 768 threads
      // per SM (3 x 256, 6 x 128) can hide more of the latency of its short
      // per-row stages
      static const LaunchFn c[] = {&Fused<256, 1, 2, CL>::launch, &Fused<128, 1, 4, CL>::launch,
                                   &Fused<512, 1, 1, CL>::launch, &Fused<64, 1, 8, CL>::launch,
                                   &Fused<32, 1, 16, CL>::launch, &Fused<256, 1, 3, CL>::launch,
                                   &Fused<128, 1, 6, CL>::launch, &Fused<128, 1, 6, CL, kOptPair>::launch,
                                   &Fused<256, 1, 3, CL, kOptPair>::launch};
      *fns = c;
      return 9;
    } else {
      static const LaunchFn c[] = {&Fused<256, 1, 2, CL>::launch, &Fused<128, 1, 4, CL>::launch,
                                   &Fused<512, 1, 1, CL>::launch, &Fused<64, 1, 8, CL>::launch,
                                   &Fused<32, 1, 16, CL>::launch};
      *fns = c;
      return 5;
    }
  }

  static void ghosts(Handle& h, void* dst) {
    const Params& p = h.p;
    if (!p.periodic_x) {
      k_ghosts<D, S><<<grid_for(2LL * p.G * p.Ny * p.Nz), kBlock, 0, h.stream>>>(p, reinterpret_cast<ST*>(dst));
      h.launches += 1;
    }
  }

  // shock capturing: numerical mu, eta, k for the next step from this step's
  // rho, u (D planes), T
  static void shock_capturing(Handle& h, const real* rho, const real* u, const real* T) {
    h.launches += n1_update<D, real>(h.p, h.stream, rho, u, T);
  }

  template <class CL> static void step_cl(Handle& h, const void* src, void* dst) {
    const LaunchFn* fns;
    const int n = candidates<CL>(&fns);
    fns[h.tile_cfg < n ? h.tile_cfg : 0](h, src, dst);
    ghosts(h, dst);
    if (h.p.sc_on) {
      const real* W = static_cast<const real*>(h.p.sc_prims);
      shock_capturing(h, W, W + h.p.plane, W + (1 + D) * h.p.plane);
    }
  }
  static void step(Handle& h, const void* src, void* dst) { step_cl<ExactClosure<real>>(h, src, dst); }

  // Time every candidate shape for `reps` steps from the current state into
  // the spare buffer (the state is not advanced) and keep the fastest.
  template <class CL> static int autotune_cl(Handle& h, int reps, float* best_ms) {
    const LaunchFn* fns;
    const int n = candidates<CL>(&fns);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0;
    float bt = 1e30f;
    const void* src = h.pop[h.cur];
    void* dst = h.pop[h.cur ^ 1];
    for (int c = 0; c < n; ++c) {
      fns[c](h, src, dst);                                   // warm-up / occupancy query
      cudaEventRecord(e0, h.stream);
      for (int r = 0; r < reps; ++r) fns[c](h, src, dst);
      cudaEventRecord(e1, h.stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (c < kMaxTiles) h.tune_ms[c] = ms / (reps > 0 ? reps : 1);
      if (ms < bt) {
        bt = ms;
        best = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h.tile_cfg = best;
    h.tune_n = n < kMaxTiles ? n : kMaxTiles;
    if (best_ms) *best_ms = bt / (reps > 0 ? reps : 1);
    return best;
  }
  static int autotune(Handle& h, int reps, float* best_ms) { return autotune_cl<ExactClosure<real>>(h, reps, best_ms); }
  template <class CL> static int ntiles_cl() {
    const LaunchFn* fns;
    return candidates<CL>(&fns);
  }
  static int ntiles() { return ntiles_cl<ExactClosure<real>>(); }

  static void step_multipass(Handle& h, const void* src, void* dst) {
    const Params& p = h.p;
    fields(h, src);
    k_collide<D, S, real><<<grid_for((long long)p.Nx * p.Ny * p.Nz), kBlock, 0, h.stream>>>(
        p, reinterpret_cast<const ST*>(src), reinterpret_cast<ST*>(dst), M(h), W(h), h.err_dev);
    h.launches += 1;
    if (!p.periodic_x) {
      k_ghosts<D, S><<<grid_for(2LL * p.G * p.Ny * p.Nz), kBlock, 0, h.stream>>>(p, reinterpret_cast<ST*>(dst));
      h.launches += 1;
    }
    if (p.sc_on) shock_capturing(h, M(h), W(h), W(h) + D * p.plane);
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

  // ---- batches -------------------------------------------------------------
  template <int TX, int TY, int MINB> struct BatchFused {
    using FG = FusedGeom<D, TX, TY>;
    static int prepare(Batch& b) {
      std::vector<BatchInstance> ti(b.n);
      std::vector<BatchItem> items;
      const int seg_len = 128;                                // planes per work item (long columns split)
      for (int k = 0; k < b.n; ++k) {
        const Handle& h = *b.inst[k];
        BatchInstance& bi = ti[k];
        bi.p = h.p;
        bi.pop[0] = h.pop[0];
        bi.pop[1] = h.pop[1];
        bi.ncolx = (h.p.Nx + TX - 1) / TX;
        bi.ncoly = D == 3 ? (h.p.Ny + TY - 1) / TY : 1;
        const int Nm = D == 3 ? h.p.Nz : h.p.Ny;
        const int nseg = Nm > seg_len ? (Nm + seg_len - 1) / seg_len : 1;
        for (int c = 0; c < bi.ncolx * bi.ncoly; ++c)
          for (int sg = 0; sg < nseg; ++sg)
            items.push_back({k, c, int((long long)Nm * sg / nseg), int((long long)Nm * (sg + 1) / nseg)});
      }
      std::stable_sort(items.begin(), items.end(),
                       [](const BatchItem& a, const BatchItem& c) { return a.me - a.mb > c.me - c.mb; });
      // rows of the batched shock-capturing kernels: instances with it on
      std::vector<int> rowstart(b.n + 1, 0);
      for (int k = 0; k < b.n; ++k)
        rowstart[k + 1] = rowstart[k] + (ti[k].p.sc_on ? ti[k].p.Ny * ti[k].p.Nz : 0);
      if (b.d_insts) cudaFree(b.d_insts);
      if (b.d_items) cudaFree(b.d_items);
      if (b.d_n1rows) cudaFree(b.d_n1rows);
      b.d_insts = b.d_items = nullptr;
      b.d_n1rows = nullptr;
      if (dev_malloc(&b.d_insts, sizeof(BatchInstance) * b.n) != cudaSuccess) return LBM_ENOMEM;
      if (dev_malloc(&b.d_items, sizeof(BatchItem) * items.size()) != cudaSuccess) return LBM_ENOMEM;
      if (dev_malloc(&b.d_n1rows, sizeof(int) * (b.n + 1)) != cudaSuccess) return LBM_ENOMEM;
      cudaMemcpy(b.d_insts, ti.data(), sizeof(BatchInstance) * b.n, cudaMemcpyHostToDevice);
      cudaMemcpy(b.d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
      cudaMemcpy(b.d_n1rows, rowstart.data(), sizeof(int) * (b.n + 1), cudaMemcpyHostToDevice);
      b.n1rows = rowstart[b.n];
      b.nitems = int(items.size());
      const size_t smem = FG::template smem_bytes<real>();
      auto kern = k_step_fused_batch<D, S, real, TX, TY, MINB>;
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      int bps = 1, sms = 1, dev = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, FG::NT, smem);
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      b.grid = (bps < 1 ? 1 : bps) * sms;
      if (b.grid > b.nitems) b.grid = b.nitems;
      return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
    }
    static void enqueue(Batch& b, int parity) {
      cudaMemsetAsync(b.d_counter, 0, sizeof(int), b.stream);
      k_step_fused_batch<D, S, real, TX, TY, MINB><<<b.grid, FG::NT, FG::template smem_bytes<real>(), b.stream>>>(
          reinterpret_cast<const BatchInstance*>(b.d_insts), reinterpret_cast<const BatchItem*>(b.d_items), b.nitems,
          parity, b.d_counter, b.d_errs);
      k_ghosts_batch<D, S><<<b.n, 256, 0, b.stream>>>(reinterpret_cast<const BatchInstance*>(b.d_insts), parity);
      b.launches += 2;
      if (b.n1rows > 0 && !b.tuning)
        b.launches += n1_update_batch<D, real>(reinterpret_cast<const BatchInstance*>(b.d_insts), b.d_n1rows, b.n,
                                               b.n1rows, b.stream);
    }
  };

  using PrepFn = int (*)(Batch&);
  using EnqFn = void (*)(Batch&, int);
  static int batch_cands(const PrepFn** pf, const EnqFn** ef) {
    if constexpr (D == 3) {
      if constexpr (sizeof(real) == 8) {
        static const PrepFn p[] = {&BatchFused<32, 8, 1>::prepare};
        static const EnqFn e[] = {&BatchFused<32, 8, 1>::enqueue};
        *pf = p; *ef = e;
        return 1;
      } else {
        static const PrepFn p[] = {&BatchFused<32, 8, 2>::prepare, &BatchFused<16, 16, 2>::prepare};
        static const EnqFn e[] = {&BatchFused<32, 8, 2>::enqueue, &BatchFused<16, 16, 2>::enqueue};
        *pf = p; *ef = e;
        return 2;
      }
    } else if constexpr (sizeof(real) == 4) {
      static const PrepFn p[] = {&BatchFused<256, 1, 2>::prepare, &BatchFused<128, 1, 4>::prepare,
                                 &BatchFused<64, 1, 8>::prepare, &BatchFused<256, 1, 3>::prepare,
                                 &BatchFused<128, 1, 6>::prepare};
      static const EnqFn e[] = {&BatchFused<256, 1, 2>::enqueue, &BatchFused<128, 1, 4>::enqueue,
                                &BatchFused<64, 1, 8>::enqueue, &BatchFused<256, 1, 3>::enqueue,
                                &BatchFused<128, 1, 6>::enqueue};
      *pf = p; *ef = e;
      return 5;
    } else {
      static const PrepFn p[] = {&BatchFused<256, 1, 2>::prepare, &BatchFused<128, 1, 4>::prepare,
                                 &BatchFused<64, 1, 8>::prepare};
      static const EnqFn e[] = {&BatchFused<256, 1, 2>::enqueue, &BatchFused<128, 1, 4>::enqueue,
                                &BatchFused<64, 1, 8>::enqueue};
      *pf = p; *ef = e;
      return 3;
    }
  }
  static int batch_ncfg() {
    const PrepFn* pf;
    const EnqFn* ef;
    return batch_cands(&pf, &ef);
  }
  static int batch_prepare(Batch& b, int cfg) {
    const PrepFn* pf;
    const EnqFn* ef;
    const int n = batch_cands(&pf, &ef);
    return pf[cfg < n ? cfg : 0](b);
  }
  static void batch_enqueue(Batch& b, int parity) {
    const PrepFn* pf;
    const EnqFn* ef;
    const int n = batch_cands(&pf, &ef);
    ef[b.tile_cfg < n ? b.tile_cfg : 0](b, parity);
  }

  static const Ops* ops() {
    static const Ops o = {&init,       &step,          &step_multipass, &macro, &autotune,
                          &batch_ncfg, &batch_prepare, &batch_enqueue,  &ntiles};
    return &o;
  }
};

}  // namespace lbm
