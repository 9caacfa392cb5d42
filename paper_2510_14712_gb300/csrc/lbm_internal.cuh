// lbm_internal.cuh - handle, kernel parameters and the dispatch table that
// the C interface (lbm_capi.cu) uses to reach the per-lattice /
// per-precision kernel instantiations (k_*.cu).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbm {

constexpr int kGhost = 4;         // ghost layers per non-periodic x face
constexpr int kMaxPartials = 1024;
constexpr int kMaxTiles = 16;     // tile candidates whose autotune times are kept

// Everything a kernel needs, passed by value.
struct Params {
  // geometry: padded x index xp = x + G; node offset = (z*Ny + y)*pitch + xp
  int D, Q, Nx, Ny, Nz, G, pitch;
  long long plane;            // elements per population plane = Nz*Ny*pitch
  int periodic_x;
  int bc_lo, bc_hi;           // LBM_BC_* of the x faces
  // model (FP64 master copy)
  double a, b, R, cv, kappa, eta_over_mu, mu, k_over_mu;
  int eos_kind;               // LBM_EOS_VDW | LBM_EOS_PR
  double Tc, mpr;             // Peng-Robinson T_c and alpha slope
  // inflow states (rho, u[3], T) and their equilibria (post-collision ghosts);
  // wall faces: (unused, u[3], T) of the wall
  double st_lo[5], st_hi[5];
  double eq_lo[54], eq_hi[54];   // f then g
  // FP16-deviation reference populations (f then g)
  float ref[54];
  // learned closure: device inference image (mlp::Image), NULL for the exact closure
  const void* mlp;
  // shock capturing (Sec. 4.4): on/off, coefficients C_mu, C_eta, C_k; the step
  // writes rho, u[D], T of every interior node to sc_prims (D+2 planes) and
  // reads the numerical mu, eta, k of the node from sc_visc (3 planes), both in
  // compute precision on the padded plane layout
  int sc_on;
  double sc_c[3];
  void* sc_prims;
  const void* sc_visc;
  // FP64 temperature inversion in FP32 arithmetic (lbm_set_temperature_fp64);
  // read by the multi-pass step (the fused step selects its closure instead)
  int t64;
  // the handle's two population buffers (2 Q plane elements each): the
  // bounds of every population access in bounds-check builds
  const void* pop[2];
  // the model constants above rounded to FP32 once on the host (set_model_fp32),
  // so that FP32 kernels read them as they are instead of converting the FP64
  // copies (a conversion the compiler may repeat inside loops, on the FP64 pipe)
  Model<float> mf;
};

template <typename real> __host__ __device__ inline Model<real> model_convert(const Params& p) {
  Model<real> m;
  m.a = real(p.a); m.b = real(p.b); m.R = real(p.R); m.cv = real(p.cv);
  m.kappa = real(p.kappa); m.eta_over_mu = real(p.eta_over_mu);
  m.mu = real(p.mu); m.k_over_mu = real(p.k_over_mu);
  m.kind = p.eos_kind; m.Tc = real(p.Tc); m.mpr = real(p.mpr);
  return m;
}

// model constants in the arithmetic type
template <typename real> __host__ __device__ inline Model<real> model_of(const Params& p) {
  if constexpr (sizeof(real) == 4) return p.mf;
  else return model_convert<real>(p);
}

// fill Params::mf from the FP64 constants (after every change of them)
inline void set_model_fp32(Params& p) { p.mf = model_convert<float>(p); }

// One solver instance.
struct Handle {
  int D, Q, Nx, Ny, Nz;
  lbm_eos eos;
  double tau, Pr, cv;
  Params p;
  int precision;
  size_t elem_bytes;          // bytes per stored population value
  void* pop[2];               // ping-pong population buffers
  int cur;                    // index of the buffer holding the current state
  void* scratch;              // moment / primitive fields of the multi-pass path
  size_t scratch_bytes;
  double* partials;           // kMaxPartials*(D+2) reduction partials
  double* totals_dev;         // D+2
  unsigned* err_dev;          // sticky status word
  unsigned* err_host;         // pinned
  double* io_dev;             // staging for host <-> device field copies
  size_t io_bytes;
  cudaStream_t stream;
  int initialized, unstable;
  int step_kernel;            // LBM_STEP_FUSED | LBM_STEP_MULTIPASS
  int tile_cfg;               // index of the fused kernel's tile shape (lbm_autotune)
  long long launches;
  int closure;                // LBM_CLOSURE_EXACT | LBM_CLOSURE_MLP
  void* mlp_img;              // device copy of the attached network's inference image
  float tune_ms[kMaxTiles];    // ms per step of every candidate at the last lbm_autotune
  int tune_n;
  int use_graphs;             // lbm_set_graphs: replay captured two-step graphs
  void* graphs;               // StepGraphs (lbm_capi.cu), created on first use
  void* sc_buf;               // shock capturing: prims (D+2), visc (3), work (4) planes
  int t64;                    // FP64 temperature inversion in the FP32 / FP16-deviation kernels
};

struct Batch;

// Per (D, precision) kernel set.
struct Ops {
  // state[i] at every padded node from FP64 device fields (interior layout)
  void (*init)(Handle& h, const double* rho, const double* u, const double* T);
  // one step: pop[cur] -> pop[cur^1] (including the ghost fill)
  void (*step)(Handle& h, const void* src, void* dst);
  void (*step_multipass)(Handle& h, const void* src, void* dst);
  // macroscopic FP64 fields of pop[cur] into device outputs (any may be NULL);
  // totals (device, D+2 doubles) when non-NULL
  void (*macro)(Handle& h, const void* src, double* rho, double* u, double* T, double* totals);
  // time the fused kernel's tile shapes, keep the fastest; returns its index
  int (*autotune)(Handle& h, int reps, float* best_ms);
  // batches: number of tile shapes; build the device instance table and the
  // sorted work list of shape cfg; enqueue one batched step from `parity`
  int (*batch_ncfg)();
  int (*batch_prepare)(Batch& b, int cfg);
  void (*batch_enqueue)(Batch& b, int parity);
  // number of tile shapes of the fused step (indices of lbm_set_tile / lbm_autotune)
  int (*ntiles)();
};

// A batch of instances stepped together (lbm_batch_* in include/lbm.h).
struct Batch {
  int n, D, Q, precision;
  Handle** inst;              // one handle per instance (own buffers and scratch)
  void* d_insts;              // device table of BatchInstance
  void* d_items;              // device work list of BatchItem, longest first
  int nitems;
  int* d_n1rows;              // first global row of each instance's shock capturing (n + 1 entries)
  int n1rows;                 // rows with shock capturing over all instances (0: none)
  int graph_launches;         // kernel launches of one step's graph
  int tuning;                 // graphs for timing tile shapes: no shock-capturing stencils (they would
                              // overwrite the coefficients the next real step reads)
  int* d_counter;             // work-list counter of the persistent kernel
  unsigned* d_errs;           // status word per instance
  unsigned* h_errs;           // pinned copy
  cudaStream_t stream;
  int own_stream;
  int cur;                    // parity of the current state (same for all instances)
  int tile_cfg;
  int grid;                   // persistent CTAs
  cudaGraphExec_t graph[2];   // one step from parity 0 / 1
  int graph_ready;
  int unstable;
  long long launches;
};

// Bounds-check builds (-DLBM_BOUNDS_CHECK) count the population accesses that
// fall outside the handle's buffers in one device counter per translation
// unit; each unit registers a reader of its counter here (a static
// initialiser), and lbm_debug_bounds_violations sums them.
void register_oob_reader(unsigned long long (*reader)());

// Device allocation of the library: cudaMalloc, except that the allocation
// chosen by lbm_debug_fail_alloc fails with cudaErrorMemoryAllocation (and
// allocates nothing), so that tests can take every out-of-memory path.
cudaError_t dev_malloc(void** p, size_t bytes);
template <class T> inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}

// the opaque handle type of the C interface
}  // namespace lbm
struct lbm_s : public lbm::Handle {};
struct lbm_batch_s : public lbm::Batch {};
namespace lbm {

const Ops* ops_d2_fp64();
const Ops* ops_d2_fp32();
const Ops* ops_d3_fp64();
const Ops* ops_d3_fp32();
const Ops* ops_d2_fp16();
const Ops* ops_d3_fp16();
// fused step and tile autotuner with the learned closure (FP32 storage)
void step_d2_fp32_mlp(Handle& h, const void* src, void* dst);
void step_d3_fp32_mlp(Handle& h, const void* src, void* dst);
// exact Peng-Robinson closure (lbm_eos.kind LBM_EOS_PR): fused step and its autotuner
void step_d2_fp32_pr(Handle& h, const void* src, void* dst);
void step_d3_fp32_pr(Handle& h, const void* src, void* dst);
void step_d2_fp64_pr(Handle& h, const void* src, void* dst);
void step_d3_fp64_pr(Handle& h, const void* src, void* dst);
int autotune_d2_fp32_pr(Handle& h, int reps, float* best_ms);
int autotune_d3_fp32_pr(Handle& h, int reps, float* best_ms);
int autotune_d2_fp64_pr(Handle& h, int reps, float* best_ms);
int autotune_d3_fp64_pr(Handle& h, int reps, float* best_ms);
int autotune_d2_fp32_mlp(Handle& h, int reps, float* best_ms);
int autotune_d3_fp32_mlp(Handle& h, int reps, float* best_ms);
int ntiles_d2_fp32_pr();
int ntiles_d3_fp32_pr();
int ntiles_d2_fp64_pr();
int ntiles_d3_fp64_pr();
int ntiles_d2_fp32_mlp();
int ntiles_d3_fp32_mlp();
// FP32 arithmetic with the FP64 temperature inversion (exact closures):
// fused step, autotuner and tile count of FP32 and FP16-deviation storage,
// van der Waals and Peng-Robinson
void step_d2_fp32_t64(Handle& h, const void* src, void* dst);
void step_d3_fp32_t64(Handle& h, const void* src, void* dst);
void step_d2_fp16_t64(Handle& h, const void* src, void* dst);
void step_d3_fp16_t64(Handle& h, const void* src, void* dst);
void step_d2_fp32_pr_t64(Handle& h, const void* src, void* dst);
void step_d3_fp32_pr_t64(Handle& h, const void* src, void* dst);
int autotune_d2_fp32_t64(Handle& h, int reps, float* best_ms);
int autotune_d3_fp32_t64(Handle& h, int reps, float* best_ms);
int autotune_d2_fp16_t64(Handle& h, int reps, float* best_ms);
int autotune_d3_fp16_t64(Handle& h, int reps, float* best_ms);
int autotune_d2_fp32_pr_t64(Handle& h, int reps, float* best_ms);
int autotune_d3_fp32_pr_t64(Handle& h, int reps, float* best_ms);
int ntiles_d2_fp32_t64();
int ntiles_d3_fp32_t64();
int ntiles_d2_fp16_t64();
int ntiles_d3_fp16_t64();
int ntiles_d2_fp32_pr_t64();
int ntiles_d3_fp32_pr_t64();

}  // namespace lbm
