// lbm_capi.cu - the extern "C" interface declared in include/lbm.h.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.cuh"

namespace lbm {
size_t scratch_bytes_d2_fp64(const Params&);
size_t scratch_bytes_d2_fp32(const Params&);
size_t scratch_bytes_d3_fp64(const Params&);
size_t scratch_bytes_d3_fp32(const Params&);
size_t scratch_bytes_d2_fp16(const Params&);
size_t scratch_bytes_d3_fp16(const Params&);
}  // namespace lbm

using namespace lbm;


namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                     \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Exact-closure table with the fused step and the autotuner swapped for the
// learned-closure ones (multi-pass and batched steps are exact-only).
Ops with_mlp(const Ops* base, void (*step)(Handle&, const void*, void*), int (*tune)(Handle&, int, float*),
              int (*ntiles)()) {
  Ops o = *base;
  o.step = step;
  o.autotune = tune;
  o.ntiles = ntiles;
  o.step_multipass = nullptr;
  o.batch_ncfg = nullptr;
  o.batch_prepare = nullptr;
  o.batch_enqueue = nullptr;
  return o;
}

// Exact-closure table with the fused step and the autotuner of the Peng-Robinson
// closure (the multi-pass step is EOS-generic; batches are van der Waals only).
Ops with_pr(const Ops* base, void (*step)(Handle&, const void*, void*), int (*tune)(Handle&, int, float*),
             int (*ntiles)()) {
  Ops o = *base;
  o.step = step;
  o.autotune = tune;
  o.ntiles = ntiles;
  o.batch_ncfg = nullptr;
  o.batch_prepare = nullptr;
  o.batch_enqueue = nullptr;
  return o;
}

// Exact-closure table with the fused step and the autotuner of the FP64
// temperature inversion (the multi-pass step reads Params::t64; batches keep
// the FP32 inversion).
Ops with_t64(const Ops* base, void (*step)(Handle&, const void*, void*), int (*tune)(Handle&, int, float*),
             int (*ntiles)()) {
  Ops o = *base;
  o.step = step;
  o.autotune = tune;
  o.ntiles = ntiles;
  return o;
}

const Ops* ops_for(const Handle& h) {
  if (h.p.eos_kind == LBM_EOS_PR) {
    static const Ops p2f = with_pr(ops_d2_fp32(), step_d2_fp32_pr, autotune_d2_fp32_pr, ntiles_d2_fp32_pr);
    static const Ops p3f = with_pr(ops_d3_fp32(), step_d3_fp32_pr, autotune_d3_fp32_pr, ntiles_d3_fp32_pr);
    static const Ops p2d = with_pr(ops_d2_fp64(), step_d2_fp64_pr, autotune_d2_fp64_pr, ntiles_d2_fp64_pr);
    static const Ops p3d = with_pr(ops_d3_fp64(), step_d3_fp64_pr, autotune_d3_fp64_pr, ntiles_d3_fp64_pr);
    static const Ops p2t = with_pr(ops_d2_fp32(), step_d2_fp32_pr_t64, autotune_d2_fp32_pr_t64, ntiles_d2_fp32_pr_t64);
    static const Ops p3t = with_pr(ops_d3_fp32(), step_d3_fp32_pr_t64, autotune_d3_fp32_pr_t64, ntiles_d3_fp32_pr_t64);
    if (h.precision == LBM_FP64) return h.D == 2 ? &p2d : &p3d;
    if (h.t64) return h.D == 2 ? &p2t : &p3t;
    return h.D == 2 ? &p2f : &p3f;
  }
  if (h.closure == LBM_CLOSURE_MLP) {
    static const Ops m2 = with_mlp(ops_d2_fp32(), step_d2_fp32_mlp, autotune_d2_fp32_mlp, ntiles_d2_fp32_mlp);
    static const Ops m3 = with_mlp(ops_d3_fp32(), step_d3_fp32_mlp, autotune_d3_fp32_mlp, ntiles_d3_fp32_mlp);
    return h.D == 2 ? &m2 : &m3;
  }
  if (h.t64 && h.precision != LBM_FP64) {
    static const Ops t2f = with_t64(ops_d2_fp32(), step_d2_fp32_t64, autotune_d2_fp32_t64, ntiles_d2_fp32_t64);
    static const Ops t3f = with_t64(ops_d3_fp32(), step_d3_fp32_t64, autotune_d3_fp32_t64, ntiles_d3_fp32_t64);
    static const Ops t2h = with_t64(ops_d2_fp16(), step_d2_fp16_t64, autotune_d2_fp16_t64, ntiles_d2_fp16_t64);
    static const Ops t3h = with_t64(ops_d3_fp16(), step_d3_fp16_t64, autotune_d3_fp16_t64, ntiles_d3_fp16_t64);
    if (h.precision == LBM_FP32) return h.D == 2 ? &t2f : &t3f;
    return h.D == 2 ? &t2h : &t3h;
  }
  if (h.D == 2) {
    if (h.precision == LBM_FP64) return ops_d2_fp64();
    if (h.precision == LBM_FP32) return ops_d2_fp32();
    return ops_d2_fp16();
  }
  if (h.precision == LBM_FP64) return ops_d3_fp64();
  if (h.precision == LBM_FP32) return ops_d3_fp32();
  return ops_d3_fp16();
}

size_t scratch_for(const Handle& h) {
  if (h.D == 2) {
    if (h.precision == LBM_FP64) return scratch_bytes_d2_fp64(h.p);
    if (h.precision == LBM_FP32) return scratch_bytes_d2_fp32(h.p);
    return scratch_bytes_d2_fp16(h.p);
  }
  if (h.precision == LBM_FP64) return scratch_bytes_d3_fp64(h.p);
  if (h.precision == LBM_FP32) return scratch_bytes_d3_fp32(h.p);
  return scratch_bytes_d3_fp16(h.p);
}

Model<double> host_model(const Handle& h) { return model_of<double>(h.p); }

// Two-step CUDA graphs of a handle, one per starting buffer parity, with the
// configuration they were captured for (kernel arguments are baked in).
struct StepGraphs {
  cudaGraphExec_t exec[2];
  cudaStream_t stream;        // capture / replay stream (owned when the handle uses the legacy stream)
  bool own_stream;
  Params p;
  void* pop[2];
  int tile_cfg, closure, step_kernel;
  long long launches;         // kernel launches per replay
  bool ready;
};

void drop_graphs(Handle& h) {
  StepGraphs* g = static_cast<StepGraphs*>(h.graphs);
  if (!g) return;
  for (int k = 0; k < 2; ++k)
    if (g->exec[k]) cudaGraphExecDestroy(g->exec[k]);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
  h.graphs = nullptr;
}

bool graphs_match(const Handle& h, const StepGraphs& g) {
  return g.ready && std::memcmp(&g.p, &h.p, sizeof(Params)) == 0 && g.pop[0] == h.pop[0] && g.pop[1] == h.pop[1] &&
         g.tile_cfg == h.tile_cfg && g.closure == h.closure && g.step_kernel == h.step_kernel &&
         (g.own_stream ? h.stream == nullptr : g.stream == h.stream);
}

void free_state(Handle& h) {
  for (int k = 0; k < 2; ++k) {
    if (h.pop[k]) cudaFree(h.pop[k]);
    h.pop[k] = nullptr;
    h.p.pop[k] = nullptr;
  }
  if (h.scratch) cudaFree(h.scratch);
  h.scratch = nullptr;
  if (h.io_dev) cudaFree(h.io_dev);
  h.io_dev = nullptr;
}

// shock-capturing fields: rho, u, T of the last step (D+2 planes), the
// numerical mu, eta, k (3 planes), work (4 planes), in compute precision
size_t sc_bytes(const Handle& h) {
  return size_t(h.D + 9) * size_t(h.p.plane) * (h.precision == LBM_FP64 ? 8 : 4);
}

int sc_alloc(Handle& h) {
  if (h.sc_buf) cudaFree(h.sc_buf);
  h.sc_buf = nullptr;
  h.p.sc_prims = nullptr;
  h.p.sc_visc = nullptr;
  if (!h.p.sc_on) return LBM_OK;
  CK(dev_malloc(&h.sc_buf, sc_bytes(h)));
  CK(cudaMemsetAsync(h.sc_buf, 0, sc_bytes(h), h.stream));
  const size_t es = h.precision == LBM_FP64 ? 8 : 4;
  h.p.sc_prims = h.sc_buf;
  h.p.sc_visc = static_cast<char*>(h.sc_buf) + size_t(h.D + 2) * size_t(h.p.plane) * es;
  return LBM_OK;
}

// geometry of the padded layout and the device allocations that depend on it
int layout(Handle& h) {
  free_state(h);
  Params& p = h.p;
  p.G = p.periodic_x ? 0 : kGhost;
  const int nxp = p.Nx + 2 * p.G;
  p.pitch = ((nxp + 31) / 32) * 32;      // rows start on 128-element (>= 256 B) boundaries
  p.plane = (long long)p.Nz * p.Ny * p.pitch;
  if ((long long)(2 * h.Q) * p.plane >= (1LL << 32))
    return fail(LBM_EINVAL, "domain too large: 2 Q Nz Ny pitch must stay below 2^32 elements");
  const size_t pop_bytes = size_t(2 * h.Q) * size_t(p.plane) * h.elem_bytes;
  for (int k = 0; k < 2; ++k) {
    CK(dev_malloc(&h.pop[k], pop_bytes));
    CK(cudaMemsetAsync(h.pop[k], 0, pop_bytes, h.stream));
    p.pop[k] = h.pop[k];
  }
  h.scratch_bytes = scratch_for(h);
  CK(dev_malloc(&h.scratch, h.scratch_bytes));
  h.io_bytes = size_t(h.D + 2) * size_t(h.Nx) * h.Ny * h.Nz * sizeof(double);
  CK(dev_malloc(&h.io_dev, h.io_bytes));
  h.cur = 0;
  h.initialized = 0;
  return sc_alloc(h);
}

void set_face_eq(Handle& h, int face) {
  Params& p = h.p;
  const double* st = face == 0 ? p.st_lo : p.st_hi;
  double* eq = face == 0 ? p.eq_lo : p.eq_hi;
  Model<double> m = host_model(h);
  double feq[27], geq[27], u[3] = {st[1], st[2], st[3]};
  if (h.D == 2) equilibria<2, double>(m, st[0], u, st[4], feq, geq);
  else equilibria<3, double>(m, st[0], u, st[4], feq, geq);
  for (int i = 0; i < h.Q; ++i) {
    eq[i] = feq[i];
    eq[h.Q + i] = geq[i];
  }
}

// Autotune results of this process, keyed by lattice, precision and padded
// geometry and closure: a new handle of the same shape starts with the tuned
// tile.
struct TuneEntry {
  int Q, precision, Nx, Ny, Nz, periodic_x, closure, cfg;
};
TuneEntry g_tuned[32];
int g_ntuned = 0;
std::mutex g_tune_mu;

int tuned_cfg(const Handle& h) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (int k = 0; k < g_ntuned; ++k) {
    const TuneEntry& e = g_tuned[k];
    if (e.Q == h.Q && e.precision == h.precision && e.Nx == h.Nx && e.Ny == h.Ny && e.Nz == h.Nz &&
        e.periodic_x == h.p.periodic_x && e.closure == h.closure)
      return e.cfg;
  }
  return 0;
}

void remember_cfg(const Handle& h) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (int k = 0; k < g_ntuned; ++k) {
    TuneEntry& e = g_tuned[k];
    if (e.Q == h.Q && e.precision == h.precision && e.Nx == h.Nx && e.Ny == h.Ny && e.Nz == h.Nz &&
        e.periodic_x == h.p.periodic_x && e.closure == h.closure) {
      e.cfg = h.tile_cfg;
      return;
    }
  }
  if (g_ntuned < 32) g_tuned[g_ntuned++] = {h.Q, h.precision, h.Nx, h.Ny, h.Nz, h.p.periodic_x, h.closure, h.tile_cfg};
}

int read_err(Handle& h) {
  CK(cudaMemcpyAsync(h.err_host, h.err_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, h.stream));
  CK(cudaStreamSynchronize(h.stream));
  if (*h.err_host & (LBM_FLAG_NONFINITE | LBM_FLAG_NEGATIVE)) {
    h.unstable = 1;
    return fail(LBM_EUNSTABLE, "non-finite or non-positive density/temperature produced");
  }
  return LBM_OK;
}

}  // namespace

namespace lbm {
std::vector<unsigned long long (*)()>& oob_readers() {
  static std::vector<unsigned long long (*)()> r;   // constructed on first use (static initialisers of other units)
  return r;
}
void register_oob_reader(unsigned long long (*reader)()) { oob_readers().push_back(reader); }

// allocations left until the injected failure (0: none armed)
std::atomic<int> g_fail_alloc{0};

cudaError_t dev_malloc(void** p, size_t bytes) {
  int k = g_fail_alloc.load();
  while (k > 0 && !g_fail_alloc.compare_exchange_weak(k, k - 1)) {
  }
  if (k == 1) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}
}  // namespace lbm

extern "C" {

const char* lbm_last_error(void) { return g_err.c_str(); }
const char* lbm_version(void) { return "gb300-nonideal-lbm 0.1"; }


long long lbm_debug_bounds_violations(void) {
#ifdef LBM_BOUNDS_CHECK
  unsigned long long n = 0;
  for (auto r : oob_readers()) n += r();
  return (long long)n;
#else
  return -1;
#endif
}

int lbm_debug_fail_alloc(int k) {
  if (k < 0) return fail(LBM_EINVAL, "k must be >= 0");
  g_fail_alloc.store(k);
  return LBM_OK;
}

int lbm_create(lbm_t* out, int lattice, int Nx, int Ny, int Nz, const lbm_eos* eos, double tau, double Pr,
               double cv) {
  if (!out || !eos) return fail(LBM_EINVAL, "out and eos must be non-NULL");
  *out = nullptr;
  if (lattice != LBM_D2Q9 && lattice != LBM_D3Q27) return fail(LBM_EINVAL, "lattice must be 9 or 27");
  const int D = lattice == LBM_D2Q9 ? 2 : 3;
  if (Nx < 1 || Ny < 1 || Nz < 1) return fail(LBM_EINVAL, "sizes must be >= 1");
  if (D == 2 && Nz != 1) return fail(LBM_EINVAL, "D2Q9 needs Nz == 1");
  if (!(tau > 0) || !(Pr > 0) || !(cv > 0)) return fail(LBM_EINVAL, "tau, Pr, cv must be > 0");
  if (eos->kind != LBM_EOS_VDW && eos->kind != LBM_EOS_PR) return fail(LBM_EINVAL, "unknown equation of state");
  if (eos->kind == LBM_EOS_PR) {
    if (!(eos->Tc > 0) || !(eos->m >= 0) || !std::isfinite(eos->m))
      return fail(LBM_EINVAL, "Peng-Robinson needs Tc > 0 and a finite m >= 0");
    if (eos->precision == LBM_FP16DEV) return fail(LBM_EINVAL, "Peng-Robinson handles use FP32 or FP64 storage");
  }
  if (!(eos->rho_ref > 0) || !(eos->T_ref > 0) || !(eos->b * eos->rho_ref < 1) || !(eos->R > 0))
    return fail(LBM_EINVAL, "need rho_ref > 0, T_ref > 0, R > 0, b rho_ref < 1");
  if (eos->precision < LBM_FP64 || eos->precision > LBM_FP16DEV) return fail(LBM_EINVAL, "bad precision");
  if (eos->closure != LBM_CLOSURE_EXACT)
    return fail(LBM_EINVAL, "create with LBM_CLOSURE_EXACT; a learned closure is attached by lbm_mlp_attach");
  if ((long long)Nx * Ny * Nz > (1LL << 31)) return fail(LBM_EINVAL, "too many nodes");

  lbm_s* h = new (std::nothrow) lbm_s();
  if (!h) return fail(LBM_ENOMEM, "host allocation failed");
  std::memset(static_cast<Handle*>(h), 0, sizeof(Handle));
  h->D = D;
  h->Q = lattice;
  h->Nx = Nx; h->Ny = Ny; h->Nz = Nz;
  h->eos = *eos;
  h->tau = tau; h->Pr = Pr; h->cv = cv;
  h->precision = eos->precision;
  h->elem_bytes = eos->precision == LBM_FP64 ? 8 : (eos->precision == LBM_FP32 ? 4 : 2);
  h->stream = nullptr;
  Params& p = h->p;
  p.D = D; p.Q = lattice; p.Nx = Nx; p.Ny = Ny; p.Nz = Nz;
  p.periodic_x = 1;
  p.bc_lo = p.bc_hi = LBM_BC_PERIODIC;
  p.a = eos->a; p.b = eos->b; p.R = eos->R; p.cv = cv;
  p.kappa = eos->kappa; p.eta_over_mu = eos->eta_over_mu;
  p.eos_kind = eos->kind;
  p.Tc = eos->kind == LBM_EOS_PR ? eos->Tc : 0.0;
  p.mpr = eos->kind == LBM_EOS_PR ? eos->m : 0.0;
  // the FP64 temperature inversion of the FP32 kernels is off until switched on
  h->t64 = p.t64 = 0;
  Model<double> m = host_model(*h);
  const double P_ref = eos_pressure(m, eos->rho_ref, eos->T_ref);
  if (!(P_ref > 0)) {
    delete h;
    return fail(LBM_EINVAL, "P(rho_ref, T_ref) must be > 0");
  }
  p.mu = tau * P_ref;                                      // tau = mu / P at the reference state
  const double RT = eos->R * eos->T_ref, x = 1.0 - eos->b * eos->rho_ref;
  double cp = cv + eos->R * eos->R * eos->T_ref / (RT - 2.0 * eos->a * eos->rho_ref * x * x);  // Eq. cpvdW
  if (eos->kind == LBM_EOS_PR) {   // c_p = c_v(rho, T) + T (dP/dT)^2 / (rho^2 dP/drho)
    const double r = eos->rho_ref, T = eos->T_ref, dPdT = pr_dPdT(m, r, T);
    const double cs2 = pr_cs2(m, r, T), cvr = pr_cv(m, r, T);
    const double dPdr = cs2 - T * dPdT * dPdT / (r * r * cvr);
    cp = cvr + T * dPdT * dPdT / (r * r * dPdr);
  }
  p.k_over_mu = cp / Pr;                                   // Pr = mu c_p / k
  set_model_fp32(p);
  m = host_model(*h);
  if (h->precision == LBM_FP16DEV) {
    double feq[27], geq[27], u0[3] = {0, 0, 0};
    if (D == 2) equilibria<2, double>(m, eos->rho_ref, u0, eos->T_ref, feq, geq);
    else equilibria<3, double>(m, eos->rho_ref, u0, eos->T_ref, feq, geq);
    for (int i = 0; i < h->Q; ++i) {
      p.ref[i] = float(feq[i]);
      p.ref[h->Q + i] = float(geq[i]);
    }
  }
  int rc;
  cudaError_t ae = dev_malloc(&h->partials, kMaxPartials * 5 * sizeof(double));
  if (ae == cudaSuccess) ae = dev_malloc(&h->totals_dev, 8 * sizeof(double));
  if (ae == cudaSuccess) ae = dev_malloc(&h->err_dev, sizeof(unsigned));
  if (ae == cudaSuccess) ae = cudaMallocHost(&h->err_host, sizeof(unsigned));
  if (ae != cudaSuccess) {
    rc = cuda_fail(ae, "allocation");
    const std::string msg = g_err;
    lbm_destroy(h);
    return fail(rc, msg);
  }
  cudaMemset(h->err_dev, 0, sizeof(unsigned));
  rc = layout(*h);
  if (rc != LBM_OK) {
    std::string msg = g_err;
    lbm_destroy(h);
    return fail(rc, msg);
  }
  *out = h;
  return LBM_OK;
}

int lbm_set_boundary(lbm_t h, int face, int type, const double* state) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (face != LBM_FACE_XLO && face != LBM_FACE_XHI) return fail(LBM_EINVAL, "face must be XLO or XHI");
  if (type != LBM_BC_PERIODIC && type != LBM_BC_OUTFLOW && type != LBM_BC_INFLOW && type != LBM_BC_WALL)
    return fail(LBM_EINVAL, "bad boundary type");
  Params& p = h->p;
  const int was_periodic = p.periodic_x;
  if (type == LBM_BC_PERIODIC) {
    p.bc_lo = p.bc_hi = LBM_BC_PERIODIC;
    p.periodic_x = 1;
  } else {
    if (type == LBM_BC_INFLOW) {
      if (!state) return fail(LBM_EINVAL, "inflow needs a state");
      if (!(state[0] > 0) || !(state[h->D + 1] > 0)) return fail(LBM_EINVAL, "inflow rho and T must be > 0");
      double* st = face == 0 ? p.st_lo : p.st_hi;
      st[0] = state[0];
      st[1] = st[2] = st[3] = 0.0;
      for (int a = 0; a < h->D; ++a) st[1 + a] = state[1 + a];
      st[4] = state[h->D + 1];
      set_face_eq(*h, face);
    }
    if (type == LBM_BC_WALL) {
      if (!state) return fail(LBM_EINVAL, "wall needs a state");
      if (!(state[h->D] > 0)) return fail(LBM_EINVAL, "wall T must be > 0");
      if (h->Nx < 4) return fail(LBM_EINVAL, "a wall face needs Nx >= 4 (mirror of the ghost layers)");
      double* st = face == 0 ? p.st_lo : p.st_hi;
      st[0] = st[1] = st[2] = st[3] = 0.0;      // st[0] unused: the wall density follows the fluid
      for (int a = 0; a < h->D; ++a) st[1 + a] = state[a];
      st[4] = state[h->D];
    }
    if (was_periodic) {  // the other face becomes outflow until set
      p.bc_lo = p.bc_hi = LBM_BC_OUTFLOW;
    }
    (face == 0 ? p.bc_lo : p.bc_hi) = type;
    p.periodic_x = 0;
  }
  if (was_periodic != p.periodic_x) return layout(*h);
  return LBM_OK;
}

int lbm_set_stream(lbm_t h, void* stream) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  return LBM_OK;
}

static int init_common(lbm_t h, const double* d_rho, const double* d_u, const double* d_T) {
  CK(cudaMemsetAsync(h->err_dev, 0, sizeof(unsigned), h->stream));
  if (h->sc_buf) CK(cudaMemsetAsync(h->sc_buf, 0, sc_bytes(*h), h->stream));   // no numerical transport at step 0
  h->cur = 0;
  h->tile_cfg = tuned_cfg(*h);
  ops_for(*h)->init(*h, d_rho, d_u, d_T);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  h->initialized = 1;
  h->unstable = 0;
  return LBM_OK;
}

int lbm_init(lbm_t h, const double* rho, const double* u, const double* T) {
  if (!h || !rho || !u || !T) return fail(LBM_EINVAL, "NULL argument");
  const size_t N = size_t(h->Nx) * h->Ny * h->Nz;
  double* d = h->io_dev;
  CK(cudaMemcpyAsync(d, rho, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(d + N, u, h->D * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(d + (h->D + 1) * N, T, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  return init_common(h, d, d + N, d + (h->D + 1) * N);
}

int lbm_init_device(lbm_t h, const double* d_rho, const double* d_u, const double* d_T) {
  if (!h || !d_rho || !d_u || !d_T) return fail(LBM_EINVAL, "NULL argument");
  return init_common(h, d_rho, d_u, d_T);
}

int lbm_step_async(lbm_t h, int n) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (!h->initialized) return fail(LBM_ESTATE, "lbm_init has not been called");
  if (h->unstable) return fail(LBM_ESTATE, "state is unstable; call lbm_init");
  if (n < 0) return fail(LBM_EINVAL, "n must be >= 0");
  const Ops* o = ops_for(*h);
  auto fn = h->step_kernel == LBM_STEP_MULTIPASS ? o->step_multipass : o->step;
  if (!fn) return fail(LBM_EINVAL, "the learned closure runs in the fused step only");
  if (h->use_graphs && n >= 2) {
    StepGraphs* g = static_cast<StepGraphs*>(h->graphs);
    if (!g || !graphs_match(*h, *g)) {
      drop_graphs(*h);
      g = new (std::nothrow) StepGraphs();
      if (!g) return fail(LBM_ENOMEM, "host allocation failed");
      std::memset(g, 0, sizeof(*g));
      h->graphs = g;
      if (h->stream) {
        g->stream = h->stream;
      } else {
        CK(cudaStreamCreate(&g->stream));
        g->own_stream = true;
      }
      const cudaStream_t saved = h->stream;
      const long long l0 = h->launches;
      for (int par = 0; par < 2; ++par) {
        cudaGraph_t graph = nullptr;
        h->stream = g->stream;
        cudaError_t e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          fn(*h, h->pop[par], h->pop[par ^ 1]);
          fn(*h, h->pop[par ^ 1], h->pop[par]);
          e = cudaStreamEndCapture(g->stream, &graph);
        }
        h->stream = saved;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec[par], graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
          drop_graphs(*h);
          h->launches = l0;
          return cuda_fail(e, "step graph capture");
        }
      }
      g->launches = (h->launches - l0) / 2;
      h->launches = l0;
      g->p = h->p;
      g->pop[0] = h->pop[0];
      g->pop[1] = h->pop[1];
      g->tile_cfg = h->tile_cfg;
      g->closure = h->closure;
      g->step_kernel = h->step_kernel;
      g->ready = true;
    }
    for (; n >= 2; n -= 2) {                 // two steps return to the same parity
      CK(cudaGraphLaunch(g->exec[h->cur], g->stream));
      h->launches += g->launches;
    }
  }
  for (int k = 0; k < n; ++k) {
    fn(*h, h->pop[h->cur], h->pop[h->cur ^ 1]);
    h->cur ^= 1;
  }
  CK(cudaGetLastError());
  return LBM_OK;
}

int lbm_sync(lbm_t h) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  return read_err(*h);
}

int lbm_step(lbm_t h, int n) {
  int rc = lbm_step_async(h, n);
  if (rc != LBM_OK) return rc;
  return read_err(*h);
}

int lbm_moments_device(lbm_t h, double* d_rho, double* d_u, double* d_T, double* totals) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (!h->initialized) return fail(LBM_ESTATE, "lbm_init has not been called");
  ops_for(*h)->macro(*h, h->pop[h->cur], d_rho, d_u, d_T, totals ? h->totals_dev : nullptr);
  CK(cudaGetLastError());
  if (totals)
    CK(cudaMemcpyAsync(totals, h->totals_dev, (h->D + 2) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_moments(lbm_t h, double* rho, double* u, double* T, double* totals) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (!h->initialized) return fail(LBM_ESTATE, "lbm_init has not been called");
  const size_t N = size_t(h->Nx) * h->Ny * h->Nz;
  double* d = h->io_dev;
  int rc = lbm_moments_device(h, rho ? d : nullptr, u ? d + N : nullptr, T ? d + (h->D + 1) * N : nullptr, totals);
  if (rc != LBM_OK) return rc;
  if (rho) CK(cudaMemcpyAsync(rho, d, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (u) CK(cudaMemcpyAsync(u, d + N, h->D * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (T) CK(cudaMemcpyAsync(T, d + (h->D + 1) * N, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_get_flags(lbm_t h, unsigned* flags) {
  if (!h || !flags) return fail(LBM_EINVAL, "NULL argument");
  CK(cudaMemcpyAsync(h->err_host, h->err_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *flags = *h->err_host;
  return LBM_OK;
}

size_t lbm_population_bytes(lbm_t h) {
  if (!h) return 0;
  return size_t(2 * h->Q) * size_t(h->p.plane) * h->elem_bytes;
}

int lbm_get_populations(lbm_t h, void* host, size_t bytes) {
  if (!h || !host) return fail(LBM_EINVAL, "NULL argument");
  if (bytes != lbm_population_bytes(h)) return fail(LBM_EINVAL, "size mismatch");
  if (!h->initialized) return fail(LBM_ESTATE, "lbm_init has not been called");
  CK(cudaMemcpyAsync(host, h->pop[h->cur], bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_set_populations(lbm_t h, const void* host, size_t bytes) {
  if (!h || !host) return fail(LBM_EINVAL, "NULL argument");
  if (bytes != lbm_population_bytes(h)) return fail(LBM_EINVAL, "size mismatch");
  CK(cudaMemcpyAsync(h->pop[h->cur], host, bytes, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemsetAsync(h->err_dev, 0, sizeof(unsigned), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->initialized = 1;
  h->unstable = 0;
  return LBM_OK;
}

int lbm_set_step_kernel(lbm_t h, int kind) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (kind != LBM_STEP_FUSED && kind != LBM_STEP_MULTIPASS) return fail(LBM_EINVAL, "unknown step kernel");
  h->step_kernel = kind;
  return LBM_OK;
}

int lbm_autotune(lbm_t h, int reps, int* chosen, float* ms_per_step) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (!h->initialized) return fail(LBM_ESTATE, "lbm_init has not been called");
  if (reps < 1) return fail(LBM_EINVAL, "reps must be >= 1");
  const int c = ops_for(*h)->autotune(*h, reps, ms_per_step);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  remember_cfg(*h);
  if (chosen) *chosen = c;
  return LBM_OK;
}

int lbm_set_shock_capturing(lbm_t h, double C_mu, double C_eta, double C_k) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (!(C_mu >= 0) || !(C_eta >= 0) || !(C_k >= 0) || !std::isfinite(C_mu) || !std::isfinite(C_eta) ||
      !std::isfinite(C_k))
    return fail(LBM_EINVAL, "shock-capturing coefficients must be finite and >= 0");
  const int on = (C_mu > 0 || C_eta > 0 || C_k > 0) ? 1 : 0;
  h->p.sc_c[0] = C_mu;
  h->p.sc_c[1] = C_eta;
  h->p.sc_c[2] = C_k;
  if (on != h->p.sc_on) {
    CK(cudaStreamSynchronize(h->stream));
    h->p.sc_on = on;
    int rc = sc_alloc(*h);
    if (rc != LBM_OK) {
      h->p.sc_on = 0;
      return rc;
    }
  }
  return LBM_OK;
}

int lbm_set_temperature_fp64(lbm_t h, int on) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  h->t64 = (on && h->precision != LBM_FP64) ? 1 : 0;   // FP64 arithmetic inverts in FP64 anyway
  h->p.t64 = h->t64;                                    // step graphs are re-captured (they record Params)
  return LBM_OK;
}

int lbm_get_temperature_fp64(lbm_t h) { return h ? h->t64 : 0; }

int lbm_set_graphs(lbm_t h, int on) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  h->use_graphs = on ? 1 : 0;
  if (!on) {
    if (h->graphs) CK(cudaDeviceSynchronize());
    drop_graphs(*h);
  }
  return LBM_OK;
}

int lbm_autotune_times(lbm_t h, float* ms_per_step, int n) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  for (int k = 0; k < h->tune_n && k < n; ++k)
    if (ms_per_step) ms_per_step[k] = h->tune_ms[k];
  return h->tune_n;
}

int lbm_tile_count(lbm_t h) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  return ops_for(*h)->ntiles();
}

int lbm_set_tile(lbm_t h, int index) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  const int n = ops_for(*h)->ntiles();
  if (index < 0 || index >= n)
    return fail(LBM_EINVAL, "tile index " + std::to_string(index) + " out of range [0, " + std::to_string(n) + ")");
  h->tile_cfg = index;                 // step graphs are re-captured (they record the tile)
  return LBM_OK;
}

long long lbm_launch_count(lbm_t h) { return h ? h->launches : 0; }

int lbm_destroy(lbm_t h) {
  if (!h) return LBM_OK;
  if (h->graphs) cudaDeviceSynchronize();
  drop_graphs(*h);
  free_state(*h);
  if (h->sc_buf) cudaFree(h->sc_buf);
  if (h->mlp_img) cudaFree(h->mlp_img);
  if (h->partials) cudaFree(h->partials);
  if (h->totals_dev) cudaFree(h->totals_dev);
  if (h->err_dev) cudaFree(h->err_dev);
  if (h->err_host) cudaFreeHost(h->err_host);
  delete h;
  return LBM_OK;
}

}  // extern "C"
