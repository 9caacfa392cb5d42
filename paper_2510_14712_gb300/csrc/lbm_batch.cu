// lbm_batch.cu - batches of instances stepped by one persistent launch per
// step (include/lbm.h, lbm_batch_*).  Each instance is an ordinary handle
// (own buffers, boundaries, moments); the batch adds a device table of the
// instances, a work list of (instance, column, plane range) items sorted
// longest first, and one CUDA graph per buffer parity holding a step:
// counter reset, the persistent fused kernel, the batched ghost fill and, when
// any instance has shock capturing on, the batched shock-capturing stencils.
#include <cstring>
#include <new>
#include <string>

#include "lbm_internal.cuh"

using namespace lbm;

namespace {

thread_local std::string g_berr;

int bfail(int code, const std::string& msg) {
  g_berr = msg;
  return code;
}

#define BCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return bfail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,                   \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

const Ops* bops(const Batch& b) {
  if (b.D == 2) return b.precision == LBM_FP64 ? ops_d2_fp64() : (b.precision == LBM_FP32 ? ops_d2_fp32() : ops_d2_fp16());
  return b.precision == LBM_FP64 ? ops_d3_fp64() : (b.precision == LBM_FP32 ? ops_d3_fp32() : ops_d3_fp16());
}

void drop_graphs(Batch& b) {
  for (int k = 0; k < 2; ++k)
    if (b.graph[k]) {
      cudaGraphExecDestroy(b.graph[k]);
      b.graph[k] = nullptr;
    }
  b.graph_ready = 0;
}

// (re)build the device tables for the current tile shape and capture the two
// one-step graphs
int ready(Batch& b) {
  if (b.graph_ready) return LBM_OK;
  drop_graphs(b);
  int rc = bops(b)->batch_prepare(b, b.tile_cfg);
  if (rc != LBM_OK) return bfail(rc, "batch work list preparation failed");
  for (int par = 0; par < 2; ++par) {
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeThreadLocal));
    const long long l0 = b.launches;
    bops(b)->batch_enqueue(b, par);
    b.graph_launches = int(b.launches - l0);   // kernel launches of one replay
    b.launches = l0;
    BCK(cudaStreamEndCapture(b.stream, &g));
    cudaError_t e = cudaGraphInstantiate(&b.graph[par], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(LBM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  b.graph_ready = 1;
  return LBM_OK;
}

int check_errs(Batch& b) {
  BCK(cudaMemcpyAsync(b.h_errs, b.d_errs, sizeof(unsigned) * b.n, cudaMemcpyDeviceToHost, b.stream));
  BCK(cudaStreamSynchronize(b.stream));
  for (int k = 0; k < b.n; ++k)
    if (b.h_errs[k] & (LBM_FLAG_NONFINITE | LBM_FLAG_NEGATIVE)) {
      b.unstable = 1;
      return bfail(LBM_EUNSTABLE, "instance " + std::to_string(k) + ": non-finite or non-positive density/temperature");
    }
  return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_batch_last_error(void) { return g_berr.c_str(); }

int lbm_batch_create(lbm_batch_t* out, int lattice, int n, const int* Nx, const int* Ny, const int* Nz,
                     const lbm_eos* eos, double tau, double Pr, double cv) {
  if (!out || !Nx || !Ny || !eos) return bfail(LBM_EINVAL, "NULL argument");
  *out = nullptr;
  if (n < 1) return bfail(LBM_EINVAL, "n must be >= 1");
  if (lattice != LBM_D2Q9 && lattice != LBM_D3Q27) return bfail(LBM_EINVAL, "lattice must be 9 or 27");
  if (lattice == LBM_D3Q27 && !Nz) return bfail(LBM_EINVAL, "D3Q27 batches need Nz");
  if (eos->kind != LBM_EOS_VDW) return bfail(LBM_EINVAL, "batches use the van der Waals fluid");
  lbm_batch_s* b = new (std::nothrow) lbm_batch_s();
  if (!b) return bfail(LBM_ENOMEM, "host allocation failed");
  std::memset(static_cast<Batch*>(b), 0, sizeof(Batch));
  b->n = n;
  b->D = lattice == LBM_D2Q9 ? 2 : 3;
  b->Q = lattice;
  b->precision = eos->precision;
  b->inst = new (std::nothrow) Handle*[n]();
  if (!b->inst) {
    delete b;
    return bfail(LBM_ENOMEM, "host allocation failed");
  }
  int rc = LBM_OK;
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) rc = LBM_ECUDA;
  b->own_stream = 1;
  for (int k = 0; k < n && rc == LBM_OK; ++k) {
    lbm_t h = nullptr;
    rc = lbm_create(&h, lattice, Nx[k], Ny[k], lattice == LBM_D2Q9 ? 1 : Nz[k], eos, tau, Pr, cv);
    if (rc != LBM_OK) {
      g_berr = std::string("instance ") + std::to_string(k) + ": " + lbm_last_error();
      break;
    }
    b->inst[k] = h;
    lbm_set_stream(h, b->stream);
  }
  if (rc == LBM_OK && (dev_malloc(&b->d_counter, sizeof(int)) != cudaSuccess ||
                       dev_malloc(&b->d_errs, sizeof(unsigned) * n) != cudaSuccess ||
                       cudaMallocHost(&b->h_errs, sizeof(unsigned) * n) != cudaSuccess))
    rc = LBM_ENOMEM;
  if (rc == LBM_OK && cudaMemset(b->d_errs, 0, sizeof(unsigned) * n) != cudaSuccess) rc = LBM_ECUDA;
  if (rc != LBM_OK) {
    std::string msg = g_berr.empty() ? "batch creation failed" : g_berr;
    lbm_batch_destroy(b);
    return bfail(rc, msg);
  }
  *out = b;
  return LBM_OK;
}

int lbm_batch_set_boundary(lbm_batch_t b, int k, int face, int type, const double* state) {
  if (!b || k < 0 || k >= b->n) return bfail(LBM_EINVAL, "bad batch or instance index");
  const int rc = lbm_set_boundary(static_cast<lbm_t>(b->inst[k]), face, type, state);
  if (rc != LBM_OK) return bfail(rc, lbm_last_error());
  b->graph_ready = 0;   // the instance table holds the boundary states and buffer pointers
  return LBM_OK;
}

int lbm_batch_set_shock_capturing(lbm_batch_t b, int k, double C_mu, double C_eta, double C_k) {
  if (!b || k < -1 || k >= b->n) return bfail(LBM_EINVAL, "bad batch or instance index");
  for (int j = (k < 0 ? 0 : k); j < (k < 0 ? b->n : k + 1); ++j) {
    const int rc = lbm_set_shock_capturing(static_cast<lbm_t>(b->inst[j]), C_mu, C_eta, C_k);
    if (rc != LBM_OK) return bfail(rc, lbm_last_error());
  }
  b->graph_ready = 0;   // the instance table holds the coefficients and buffer pointers
  return LBM_OK;
}

int lbm_batch_set_stream(lbm_batch_t b, void* stream) {
  if (!b || !stream) return bfail(LBM_EINVAL, "a batch needs a non-default stream");
  if (b->own_stream) cudaStreamDestroy(b->stream);
  b->own_stream = 0;
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  for (int k = 0; k < b->n; ++k) lbm_set_stream(static_cast<lbm_t>(b->inst[k]), stream);
  b->graph_ready = 0;
  return LBM_OK;
}

int lbm_batch_init(lbm_batch_t b, int k, const double* rho, const double* u, const double* T) {
  if (!b || k < 0 || k >= b->n) return bfail(LBM_EINVAL, "bad batch or instance index");
  Handle& h = *b->inst[k];
  int rc = lbm_init(static_cast<lbm_t>(b->inst[k]), rho, u, T);   // writes buffer 0
  if (rc != LBM_OK) return bfail(rc, lbm_last_error());
  if (b->cur == 1) {   // the batch's state lives in buffer 1: move the new state there
    BCK(cudaMemcpyAsync(h.pop[1], h.pop[0], lbm_population_bytes(static_cast<lbm_t>(b->inst[k])),
                        cudaMemcpyDeviceToDevice, b->stream));
  }
  h.cur = b->cur;
  BCK(cudaMemsetAsync(b->d_errs + k, 0, sizeof(unsigned), b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  b->unstable = 0;
  for (int j = 0; j < b->n; ++j)
    if (!b->inst[j]->initialized) return LBM_OK;
  return LBM_OK;
}

int lbm_batch_step_async(lbm_batch_t b, int n) {
  if (!b) return bfail(LBM_EINVAL, "NULL batch");
  if (n < 0) return bfail(LBM_EINVAL, "n must be >= 0");
  for (int k = 0; k < b->n; ++k)
    if (!b->inst[k]->initialized) return bfail(LBM_ESTATE, "instance " + std::to_string(k) + " not initialised");
  if (b->unstable) return bfail(LBM_ESTATE, "an instance is unstable; re-initialise it");
  int rc = ready(*b);
  if (rc != LBM_OK) return rc;
  for (int s = 0; s < n; ++s) {
    BCK(cudaGraphLaunch(b->graph[b->cur], b->stream));
    b->launches += b->graph_launches;
    b->cur ^= 1;
  }
  for (int k = 0; k < b->n; ++k) b->inst[k]->cur = b->cur;
  return LBM_OK;
}

int lbm_batch_sync(lbm_batch_t b) {
  if (!b) return bfail(LBM_EINVAL, "NULL batch");
  return check_errs(*b);
}

int lbm_batch_step(lbm_batch_t b, int n) {
  int rc = lbm_batch_step_async(b, n);
  if (rc != LBM_OK) return rc;
  return check_errs(*b);
}

int lbm_batch_moments(lbm_batch_t b, int k, double* rho, double* u, double* T, double* totals) {
  if (!b || k < 0 || k >= b->n) return bfail(LBM_EINVAL, "bad batch or instance index");
  b->inst[k]->cur = b->cur;
  const int rc = lbm_moments(static_cast<lbm_t>(b->inst[k]), rho, u, T, totals);
  return rc == LBM_OK ? rc : bfail(rc, lbm_last_error());
}

int lbm_batch_flags(lbm_batch_t b, int k, unsigned* flags) {
  if (!b || k < 0 || k >= b->n || !flags) return bfail(LBM_EINVAL, "bad argument");
  BCK(cudaMemcpyAsync(b->h_errs, b->d_errs, sizeof(unsigned) * b->n, cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  *flags = b->h_errs[k];
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch_t b, int reps, int* chosen, float* ms_per_step) {
  if (!b || reps < 1) return bfail(LBM_EINVAL, "bad argument");
  for (int k = 0; k < b->n; ++k)
    if (!b->inst[k]->initialized) return bfail(LBM_ESTATE, "instance " + std::to_string(k) + " not initialised");
  const int ncfg = bops(*b)->batch_ncfg();
  // the timing events and the tuning mode are released on every return path
  struct Guard {
    lbm::Batch* b;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Guard() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      b->tuning = 0;
    }
  } g{b};
  BCK(cudaEventCreate(&g.e0));
  BCK(cudaEventCreate(&g.e1));
  int best = 0;
  float bt = 1e30f;
  b->tuning = 1;                                             // tile shapes only change the fused step
  for (int c = 0; c < ncfg; ++c) {
    b->tile_cfg = c;
    b->graph_ready = 0;
    int rc = ready(*b);
    if (rc != LBM_OK) return rc;
    BCK(cudaGraphLaunch(b->graph[b->cur], b->stream));      // warm-up; writes the spare buffers only
    BCK(cudaEventRecord(g.e0, b->stream));
    for (int r = 0; r < reps; ++r) BCK(cudaGraphLaunch(b->graph[b->cur], b->stream));
    BCK(cudaEventRecord(g.e1, b->stream));
    BCK(cudaEventSynchronize(g.e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g.e0, g.e1);
    if (ms < bt) {
      bt = ms;
      best = c;
    }
  }
  b->tuning = 0;
  b->tile_cfg = best;
  b->graph_ready = 0;
  int rc = ready(*b);
  if (rc != LBM_OK) return rc;
  BCK(cudaMemsetAsync(b->d_errs, 0, sizeof(unsigned) * b->n, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (chosen) *chosen = best;
  if (ms_per_step) *ms_per_step = bt / reps;
  return LBM_OK;
}

long long lbm_batch_nodes(lbm_batch_t b) {
  if (!b) return 0;
  long long s = 0;
  for (int k = 0; k < b->n; ++k) s += (long long)b->inst[k]->Nx * b->inst[k]->Ny * b->inst[k]->Nz;
  return s;
}

long long lbm_batch_launch_count(lbm_batch_t b) { return b ? b->launches : 0; }

int lbm_batch_destroy(lbm_batch_t b) {
  if (!b) return LBM_OK;
  drop_graphs(*b);
  if (b->inst)
    for (int k = 0; k < b->n; ++k)
      if (b->inst[k]) lbm_destroy(static_cast<lbm_t>(b->inst[k]));
  delete[] b->inst;
  if (b->d_insts) cudaFree(b->d_insts);
  if (b->d_n1rows) cudaFree(b->d_n1rows);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->d_errs) cudaFree(b->d_errs);
  if (b->h_errs) cudaFreeHost(b->h_errs);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return LBM_OK;
}

}  // extern "C"
