// lbm_noalloc.cu - conservation totals of caller-provided device fields,
// computed without allocating any memory.
//
// Who needs this: code that may not call cudaMalloc, e.g. a caller that is
// in the middle of capturing a stream into a CUDA graph (allocation calls are
// not allowed there), a real-time loop with a fixed device-memory budget, or
// a host framework whose device memory all comes from its own pool.  Such a
// caller owns the input fields and the output buffer; the block partials of
// the reduction live in one file-scope device array of fixed size instead of
// memory allocated per call.
//
// The array is shared by every call on a device and keeps the contents of the
// last call.  Each call writes every partial it reads, so nothing has to be
// cleared first; but two calls that overlap on the GPU (different streams,
// no ordering between them) race on it.  Its device address is looked up once
// per device and kept for the life of the process: after cudaDeviceReset (or
// any teardown of the device's primary context) the kept address is stale, so
// a process that resets a device must not call this entry point again.
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/lbm.h"

namespace {

constexpr int kThreads = 256;                     // threads per block
constexpr int kPerThread = 32;                    // nodes per thread
constexpr int kMaxBlocks = 8192;                  // partial-sum slots
constexpr int kMaxComp = 5;                       // D + 2 <= 5 sums per block
constexpr long long kNodesPerBlock = (long long)kThreads * kPerThread;
constexpr long long kMaxNodes = kNodesPerBlock * kMaxBlocks;   // 67,108,864 nodes

// 8192 x 5 doubles = 320 KiB, resident on every GPU that loads the library
static __device__ __align__(256) double g_partials[kMaxBlocks * kMaxComp];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_partials_ptr[kMaxDevices] = {};        // device address of g_partials, per device

thread_local std::string g_msg;

int fail(int code, const std::string& msg) {
  g_msg = msg;
  return code;
}

// one contiguous chunk of kNodesPerBlock nodes per block, fixed order
template <int D>
__global__ void k_field_totals(const double* __restrict__ rho, const double* __restrict__ u,
                               const double* __restrict__ T, long long n, double a, double cv,
                               double* __restrict__ partials) {
  constexpr int K = D + 2;
  double acc[K];
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  const long long begin = blockIdx.x * kNodesPerBlock;
  for (int r = 0; r < kPerThread; ++r) {
    const long long i = begin + (long long)r * kThreads + threadIdx.x;
    if (i >= n) break;
    const double rh = rho[i];
    double u2 = 0.0;
    acc[0] += rh;
    for (int d = 0; d < D; ++d) {
      const double ud = u[d * n + i];
      acc[1 + d] += rh * ud;
      u2 += ud * ud;
    }
    acc[1 + D] += rh * (cv * T[i] - a * rh + 0.5 * u2);   // rho E = rho (e + u^2/2), e = c_v T - a rho
  }
  __shared__ double sh[kThreads / 32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < K; ++k) {
    double v = acc[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v += sh[w][threadIdx.x];
    partials[blockIdx.x * K + threadIdx.x] = v;
  }
}

template <int D>
__global__ void k_field_totals_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
  constexpr int K = D + 2;
  const int k = threadIdx.x;
  if (k >= K) return;
  double v = 0.0;
  for (int b = 0; b < nblocks; ++b) v += partials[b * K + k];
  out[k] = v;
}

// device address of the fixed scratch on the current device (set up once)
int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(LBM_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_partials_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_partials);
    if (e != cudaSuccess || !p)
      return fail(LBM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_partials_ptr[dev] = p;
  }
  *out = g_partials_ptr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_totals_noalloc(int lattice, long long n, const double* d_rho, const double* d_u,
                                  const double* d_T, double a, double cv, double* d_totals, void* stream) {
  if (lattice != LBM_D2Q9 && lattice != LBM_D3Q27) return fail(LBM_EINVAL, "lattice must be 9 or 27");
  if (!d_rho || !d_u || !d_T || !d_totals) return fail(LBM_EINVAL, "NULL pointer");
  if (n < 1) return fail(LBM_EINVAL, "n must be >= 1");
  if (n > kMaxNodes)
    return fail(LBM_EINVAL, "n exceeds the fixed scratch of lbm_totals_noalloc (at most 67108864 nodes)");
  double* partials = nullptr;
  int rc = scratch_for_current_device(&partials);
  if (rc != LBM_OK) return rc;
  // an error left pending by earlier, unrelated work is taken off the error
  // state here, so that the check after the launches sees this call's own
  // launches only (a sticky error of a broken context fails them again)
  const cudaError_t earlier = cudaGetLastError();
  const int nblocks = int((n + kNodesPerBlock - 1) / kNodesPerBlock);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (lattice == LBM_D2Q9) {
    k_field_totals<2><<<nblocks, kThreads, 0, s>>>(d_rho, d_u, d_T, n, a, cv, partials);
    k_field_totals_final<2><<<1, 32, 0, s>>>(partials, nblocks, d_totals);
  } else {
    k_field_totals<3><<<nblocks, kThreads, 0, s>>>(d_rho, d_u, d_T, n, a, cv, partials);
    k_field_totals_final<3><<<1, 32, 0, s>>>(partials, nblocks, d_totals);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(LBM_ECUDA, std::string("launch: ") + cudaGetErrorString(e) +
                               (earlier != cudaSuccess ? std::string(" (an earlier error was pending: ") +
                                                             cudaGetErrorString(earlier) + ")"
                                                       : std::string()));
  return LBM_OK;
}

extern "C" const char* lbm_totals_noalloc_error(void) { return g_msg.c_str(); }
