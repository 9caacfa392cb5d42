// lbm_mlp.cu - training and standalone evaluation of the learned closure and
// the lbm_mlp_* interface of include/lbm_mlp.h.
//
// One training step is six launches on the network's stream:
//   k_mlp_batch    draw the minibatch (SplitMix64 indices), exact FP64 labels
//   k_mlp_fwd_bwd  per-sample forward and backward pass, one warp per 32
//                  samples: layer 2 and the input gradient of layer 2 on the
//                  tensor cores (mma.sync BF16 -> FP32), the rest on FP32
//                  pipes; writes the per-sample factors of the weight gradient
//   k_mlp_reduce   per 128-sample chunk: dW2 = dZ2^T H1 on the tensor cores,
//                  the small gradients on FP32 pipes -> one partial per chunk
//   k_mlp_sum      fixed-order sum of the chunk partials (deterministic)
//   k_mlp_adamw    AdamW update of the FP32 master weights
//   k_mlp_image    bfloat16 weights and mma fragments for the next forward
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm_mlp.h"
#include "lbm_internal.cuh"
#include "lbm_mlp.cuh"

using namespace lbm;
using namespace lbm::mlp;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CKM(call)                                                                                      \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess)                                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,                            \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                                 \
  } while (0)

constexpr int kChunk = 128;          // samples per block of k_mlp_reduce
constexpr int kMaxBatch = 1 << 20;
constexpr int kPart = NPARAM + 1;    // partial record: gradient, then loss sum

struct Scale {
  double v[NSCALE];                  // c_rho, s_rho, c_e, s_e, m_T, r_T, m_P, r_P, m_c, r_c
};
struct Eos {
  double a, b, R, cv;
};

// value k (from 0) of SplitMix64 stream `seed` (the input generators' definition)
__device__ __forceinline__ uint64_t splitmix(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// exact van der Waals closure in FP64: Eqs. lbm_temp, Pvdw, vdW_speed_of_sound
__device__ __forceinline__ void exact_fp64(const Eos& q, double rho, double e, double& T, double& P, double& c2) {
  T = (e + q.a * rho) / q.cv;
  const double x = 1.0 - q.b * rho;
  P = rho * q.R * T / x - q.a * rho * rho;
  c2 = q.R * T * (1.0 + q.R / q.cv) / (x * x) - 2.0 * q.a * rho;
}

__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return uint32_t(__bfloat16_as_ushort(lo)) | (uint32_t(__bfloat16_as_ushort(hi)) << 16);
}

// ---------------------------------------------------------------------------
__global__ void k_mlp_image(const float* __restrict__ th, Scale sc, TrainImage* __restrict__ img) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  Image& f = img->fwd;
  const float* W2 = th + OW2;
  if (i < 2048) {
    const int r = i & 1, lane = (i >> 1) & 31, nt = (i >> 6) & 7, ks = i >> 9;
    const int g = lane >> 2, t = lane & 3;
    const int k0 = 16 * ks + 2 * t + 8 * r, n = 8 * nt + g;
    f.w2f[ks][nt][lane][r] = pack_bf16(W2[n * H + k0], W2[n * H + k0 + 1]);      // B[k][n] = W2[n][k]
    img->w2b[ks][nt][lane][r] = pack_bf16(W2[k0 * H + n], W2[(k0 + 1) * H + n]);  // B[k][n] = W2[k][n]
  } else if (i < 2048 + H) {
    const int j = i - 2048;
    auto bf = [](float v) { return __bfloat162float(__float2bfloat16_rn(v)); };
    f.l1[j] = make_float4(bf(th[OW1 + 2 * j]), bf(th[OW1 + 2 * j + 1]), th[OB1 + j], 0.f);
    f.b2[j] = th[OB2 + j];
    for (int o = 0; o < 3; ++o) f.w3[o][j] = bf(th[OW3 + o * H + j]);
  } else if (i == 2048 + H) {
    f.norm[0] = float(sc.v[0]);
    f.norm[1] = float(1.0 / sc.v[1]);
    f.norm[2] = float(sc.v[2]);
    f.norm[3] = float(1.0 / sc.v[3]);
    for (int k = 4; k < NSCALE; ++k) f.norm[k] = float(sc.v[k]);
    f.norm[10] = f.norm[11] = 0.f;
    for (int o = 0; o < 3; ++o) f.b3[o] = th[OB3 + o];
    f.b3[3] = 0.f;
  }
}

__global__ void k_mlp_batch(const double* __restrict__ rho, const double* __restrict__ e, long long n, uint64_t seed,
                            unsigned long long base, int B, Scale sc, Eos q, float* __restrict__ X,
                            float* __restrict__ Y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const long long idx = (long long)(splitmix(seed, base + i) % (unsigned long long)n);
  const double r = rho[idx], ee = e[idx];
  double T, P, c2;
  exact_fp64(q, r, ee, T, P, c2);
  X[2 * i] = float((r - sc.v[0]) / sc.v[1]);
  X[2 * i + 1] = float((ee - sc.v[2]) / sc.v[3]);
  Y[3 * i] = float((T - sc.v[4]) / sc.v[5]);
  Y[3 * i + 1] = float((P - sc.v[6]) / sc.v[7]);
  Y[3 * i + 2] = float((c2 - sc.v[8]) / sc.v[9]);
}

// Per-sample forward and backward pass (4 warps per block, 32 samples per
// warp and iteration).  Outputs per sample s: dY[s] = (dL/dy0..2, |y - Y|^2),
// H1[s] = h1, dZ1[s] = dL/dz1, dZ2[s] = dL/dz2, H2[s] = h2 (64 each).
__global__ void __launch_bounds__(128) k_mlp_fwd_bwd(const TrainImage* __restrict__ img, const float* __restrict__ X,
                                                     const float* __restrict__ Y, int B, float inv3B,
                                                     float* __restrict__ dY, float* __restrict__ H1o,
                                                     float* __restrict__ dZ1o, float* __restrict__ dZ2o,
                                                     float* __restrict__ H2o) {
  __shared__ TrainImage s_img;
  {
    const uint4* src = reinterpret_cast<const uint4*>(img);
    uint4* dst = reinterpret_cast<uint4*>(&s_img);
    for (int k = threadIdx.x; k < int(sizeof(TrainImage) / 16); k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  const Image& w = s_img.fwd;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int ngrp = (B + 31) / 32;
  for (int grp = blockIdx.x * 4 + (threadIdx.x >> 5); grp < ngrp; grp += gridDim.x * 4) {
    const int s0 = grp * 32, s = s0 + lane;
    const bool valid = s < B;
    const float x0 = valid ? X[2 * s] : 0.f, x1 = valid ? X[2 * s + 1] : 0.f;
    float y[3];
    forward_warp(w, x0, x1, y);
    float dy[3], l2 = 0.f;
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const float r = valid ? y[o] - Y[3 * s + o] : 0.f;
      dy[o] = 2.f * r * inv3B;
      l2 += r * r;
    }
    if (valid) *reinterpret_cast<float4*>(dY + 4 * (size_t)s) = make_float4(dy[0], dy[1], dy[2], l2);
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
      float xr[2][2], dyr[2][3];
      int sh[2];
      bool vh[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = 16 * mt + 8 * h + g;
        sh[h] = s0 + row;
        vh[h] = sh[h] < B;
        xr[h][0] = __shfl_sync(full, x0, row);
        xr[h][1] = __shfl_sync(full, x1, row);
#pragma unroll
        for (int o = 0; o < 3; ++o) dyr[h][o] = __shfl_sync(full, dy[o], row);
      }
      // layer 1 in A-operand layout (kept for layer 2), h1 to memory
      uint32_t ah[4][4], al[4][4];
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int c = 16 * ks + 8 * half + 2 * t;
          const float4 wa = w.l1[c], wb = w.l1[c + 1];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float ha = gelu(fmaf(wa.x, xr[h][0], fmaf(wa.y, xr[h][1], wa.z)));
            const float hb = gelu(fmaf(wb.x, xr[h][0], fmaf(wb.y, xr[h][1], wb.z)));
            split_bf16(ha, hb, ah[ks][h + 2 * half], al[ks][h + 2 * half]);
            if (vh[h]) *reinterpret_cast<float2*>(H1o + (size_t)sh[h] * H + c) = make_float2(ha, hb);
          }
        }
      // layer 2 forward, backward through layers 3 and the gelu of layer 2
      uint32_t dza[4][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int c = 8 * nt + 2 * t;
        float d[4] = {w.b2[c], w.b2[c + 1], w.b2[c], w.b2[c + 1]};
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint2 b = *reinterpret_cast<const uint2*>(&w.w2f[ks][nt][lane][0]);
          mma_bf16(d, ah[ks], b.x, b.y);
          mma_bf16(d, al[ks], b.x, b.y);
        }
        float h2[4], dz2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float dg;
          gelu_d(d[q], h2[q], dg);
          const int hq = q >> 1, col = c + (q & 1);
          const float dh2 = dyr[hq][0] * w.w3[0][col] + dyr[hq][1] * w.w3[1][col] + dyr[hq][2] * w.w3[2][col];
          dz2[q] = dh2 * dg;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
          if (vh[h]) {
            *reinterpret_cast<float2*>(H2o + (size_t)sh[h] * H + c) = make_float2(h2[2 * h], h2[2 * h + 1]);
            *reinterpret_cast<float2*>(dZ2o + (size_t)sh[h] * H + c) = make_float2(dz2[2 * h], dz2[2 * h + 1]);
          }
        dza[nt >> 1][2 * (nt & 1)] = pack_bf16(dz2[0], dz2[1]);
        dza[nt >> 1][2 * (nt & 1) + 1] = pack_bf16(dz2[2], dz2[3]);
      }
      // dh1 = dZ2 W2 on the tensor cores, dz1 = dh1 gelu'(z1)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int c = 8 * nt + 2 * t;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint2 b = *reinterpret_cast<const uint2*>(&s_img.w2b[ks][nt][lane][0]);
          mma_bf16(acc, dza[ks], b.x, b.y);
        }
        const float4 wa = w.l1[c], wb = w.l1[c + 1];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float gv, ga, gb;
          gelu_d(fmaf(wa.x, xr[h][0], fmaf(wa.y, xr[h][1], wa.z)), gv, ga);
          gelu_d(fmaf(wb.x, xr[h][0], fmaf(wb.y, xr[h][1], wb.z)), gv, gb);
          if (vh[h])
            *reinterpret_cast<float2*>(dZ1o + (size_t)sh[h] * H + c) = make_float2(acc[2 * h] * ga, acc[2 * h + 1] * gb);
        }
      }
    }
  }
}

// Gradient partial of one chunk of kChunk samples (256 threads).
__global__ void __launch_bounds__(256) k_mlp_reduce(const float* __restrict__ X, const float* __restrict__ H1,
                                                    const float* __restrict__ dZ1, const float* __restrict__ dZ2,
                                                    const float* __restrict__ H2, const float* __restrict__ dY, int B,
                                                    float* __restrict__ partial) {
  constexpr int LD = H + 8;                                  // padded row (bank spread)
  __shared__ __nv_bfloat16 s_dz[kChunk][LD], s_h1[kChunk][LD];
  const int c0 = blockIdx.x * kChunk;
  const int ns = min(kChunk, B - c0);
  for (int i = threadIdx.x; i < kChunk * H; i += blockDim.x) {
    const int r = i / H, j = i % H;
    const bool in = r < ns;
    s_dz[r][j] = __float2bfloat16_rn(in ? dZ2[(size_t)(c0 + r) * H + j] : 0.f);
    s_h1[r][j] = __float2bfloat16_rn(in ? H1[(size_t)(c0 + r) * H + j] : 0.f);
  }
  __syncthreads();
  float* out = partial + (size_t)blockIdx.x * kPart;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  // dW2[j2][j1] = sum_s dZ2[s][j2] H1[s][j1]: A[m = j2][k = s], B[k = s][n = j1]
  {
    const int mt = warp >> 1, nb = 4 * (warp & 1);
    float acc[4][4];
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[n][q] = 0.f;
#pragma unroll 2
    for (int ks = 0; ks < kChunk / 16; ++ks) {
      uint32_t a[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int j2 = 16 * mt + g + 8 * (r & 1), s = 16 * ks + 2 * t + 8 * (r >> 1);
        a[r] = pack_raw(s_dz[s][j2], s_dz[s + 1][j2]);
      }
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        const int j1 = 8 * (nb + n) + g, s = 16 * ks + 2 * t;
        mma_bf16(acc[n], a, pack_raw(s_h1[s][j1], s_h1[s + 1][j1]), pack_raw(s_h1[s + 8][j1], s_h1[s + 9][j1]));
      }
    }
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j2 = 16 * mt + g + 8 * (q >> 1), j1 = 8 * (nb + n) + 2 * t + (q & 1);
        out[OW2 + j2 * H + j1] = acc[n][q];
      }
  }
  // the small gradients on FP32 pipes, samples in order
  if (tid < H) {
    float w0 = 0.f, w1 = 0.f, bb = 0.f;
    for (int r = 0; r < ns; ++r) {
      const size_t s = size_t(c0 + r);
      const float d = dZ1[s * H + tid];
      w0 = fmaf(d, X[2 * s], w0);
      w1 = fmaf(d, X[2 * s + 1], w1);
      bb += d;
    }
    out[OW1 + 2 * tid] = w0;
    out[OW1 + 2 * tid + 1] = w1;
    out[OB1 + tid] = bb;
  } else if (tid < 2 * H) {
    const int j = tid - H;
    float bb = 0.f;
    for (int r = 0; r < ns; ++r) bb += dZ2[size_t(c0 + r) * H + j];
    out[OB2 + j] = bb;
  } else if (tid < 3 * H) {
    const int j = tid - 2 * H;
    float w0 = 0.f, w1 = 0.f, w2 = 0.f;
    for (int r = 0; r < ns; ++r) {
      const size_t s = size_t(c0 + r);
      const float h = H2[s * H + j];
      w0 = fmaf(dY[4 * s], h, w0);
      w1 = fmaf(dY[4 * s + 1], h, w1);
      w2 = fmaf(dY[4 * s + 2], h, w2);
    }
    out[OW3 + j] = w0;
    out[OW3 + H + j] = w1;
    out[OW3 + 2 * H + j] = w2;
  } else if (tid < 3 * H + 4) {
    const int o = tid - 3 * H;                               // 0..2: db3, 3: loss sum
    float bb = 0.f;
    for (int r = 0; r < ns; ++r) bb += dY[4 * size_t(c0 + r) + o];
    out[o < 3 ? OB3 + o : NPARAM] = bb;
  }
}

__global__ void k_mlp_sum(const float* __restrict__ partial, int nchunk, float loss_scale, float* __restrict__ grad,
                          float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > NPARAM) return;
  double acc = 0.0;
  for (int c = 0; c < nchunk; ++c) acc += partial[(size_t)c * kPart + p];
  if (p < NPARAM) grad[p] = float(acc);
  else *loss = float(acc * loss_scale);
}

// AdamW (Loshchilov and Hutter): bias-corrected moments, decoupled decay
__global__ void k_mlp_adamw(float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float bc1, float bc2, float wd) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const float gi = g[p];
  const float mi = 0.9f * m[p] + 0.1f * gi;
  const float vi = 0.999f * v[p] + 0.001f * gi * gi;
  m[p] = mi;
  v[p] = vi;
  th[p] -= lr * ((mi / bc1) / (sqrtf(vi / bc2) + 1e-8f) + wd * th[p]);
}

__global__ void k_mlp_minmax(const double* __restrict__ rho, const double* __restrict__ e, long long n, Eos q,
                             double* __restrict__ part) {
  __shared__ double s_lo[5][256], s_hi[5][256];
  double lo[5], hi[5];
  for (int k = 0; k < 5; ++k) {
    lo[k] = INFINITY;
    hi[k] = -INFINITY;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v[5];
    v[0] = rho[i];
    v[1] = e[i];
    exact_fp64(q, v[0], v[1], v[2], v[3], v[4]);
    for (int k = 0; k < 5; ++k) {
      lo[k] = fmin(lo[k], v[k]);
      hi[k] = fmax(hi[k], v[k]);
    }
  }
  for (int k = 0; k < 5; ++k) {
    s_lo[k][threadIdx.x] = lo[k];
    s_hi[k][threadIdx.x] = hi[k];
  }
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 5; ++k) {
        s_lo[k][threadIdx.x] = fmin(s_lo[k][threadIdx.x], s_lo[k][threadIdx.x + w]);
        s_hi[k][threadIdx.x] = fmax(s_hi[k][threadIdx.x], s_hi[k][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 5) {
    part[blockIdx.x * 10 + 2 * threadIdx.x] = s_lo[threadIdx.x][0];
    part[blockIdx.x * 10 + 2 * threadIdx.x + 1] = s_hi[threadIdx.x][0];
  }
}

// The closure of the fused step for standalone samples (4 warps per block).
__global__ void __launch_bounds__(128) k_mlp_predict(const Image* __restrict__ img, Model<float> m,
                                                     const double* __restrict__ rho, const double* __restrict__ e,
                                                     long long n, double* __restrict__ out) {
  __shared__ Image s_img;
  load_image(img, &s_img);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long ngrp = (n + 31) / 32;
  for (long long grp = blockIdx.x * 4LL + (threadIdx.x >> 5); grp < ngrp; grp += gridDim.x * 4LL) {
    const long long i = grp * 32 + lane;
    const bool act = i < n;
    const float r = act ? float(rho[i]) : 1.f, ee = act ? float(e[i]) : 0.f;
    float T = 0.f, P = 0.f, c2 = 0.f;
    const bool used = closure_warp(s_img, m, r, ee, act, T, P, c2);
    if (act) {
      out[4 * i] = T;
      out[4 * i + 1] = P;
      out[4 * i + 2] = c2;
      out[4 * i + 3] = used ? 1.0 : 0.0;
    }
  }
}

__global__ void k_mlp_energy(const double* __restrict__ rho, double* __restrict__ e, long long n, double a, double cv,
                             double scale) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) e[i] = scale * (cv * e[i] - a * rho[i]);        // e holds T on entry
}

}  // namespace

struct lbm_mlp_s {
  Eos q;
  double scale[NSCALE];
  int scaled;
  float *theta, *m, *v, *grad;
  long long t;                       // AdamW steps taken
  TrainImage* img;
  cudaStream_t stream;
  int cap;                           // minibatch capacity of the work buffers
  float *X, *Y, *dY, *H1, *dZ1, *dZ2, *H2, *partial;
  float* losses;
  int loss_cap;
};

namespace {

Scale scale_of(const lbm_mlp_s& n) {
  Scale s;
  for (int k = 0; k < NSCALE; ++k) s.v[k] = n.scale[k];
  return s;
}

void free_work(lbm_mlp_s& n) {
  float** bufs[] = {&n.X, &n.Y, &n.dY, &n.H1, &n.dZ1, &n.dZ2, &n.H2, &n.partial};
  for (float** b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  n.cap = 0;
}

int ensure_cap(lbm_mlp_s& n, int B) {
  if (B <= n.cap) return LBM_OK;
  free_work(n);
  const size_t b = size_t(B);
  const size_t nchunk = (b + kChunk - 1) / kChunk;
  CKM(cudaMalloc(&n.X, 2 * b * sizeof(float)));
  CKM(cudaMalloc(&n.Y, 3 * b * sizeof(float)));
  CKM(cudaMalloc(&n.dY, 4 * b * sizeof(float)));
  CKM(cudaMalloc(&n.H1, H * b * sizeof(float)));
  CKM(cudaMalloc(&n.dZ1, H * b * sizeof(float)));
  CKM(cudaMalloc(&n.dZ2, H * b * sizeof(float)));
  CKM(cudaMalloc(&n.H2, H * b * sizeof(float)));
  CKM(cudaMalloc(&n.partial, nchunk * kPart * sizeof(float)));
  n.cap = B;
  return LBM_OK;
}

void launch_image(lbm_mlp_s& n) {
  k_mlp_image<<<(2048 + H + 1 + 255) / 256, 256, 0, n.stream>>>(n.theta, scale_of(n), n.img);
}

// loss (written to loss_dev) and gradient (n.grad) on the B samples in n.X, n.Y
void launch_grad(lbm_mlp_s& n, int B, float* loss_dev) {
  const int ngrp = (B + 31) / 32;
  int blocks = (ngrp + 3) / 4;
  if (blocks > 152 * 8) blocks = 152 * 8;
  const float inv3B = float(1.0 / (3.0 * B));
  k_mlp_fwd_bwd<<<blocks, 128, 0, n.stream>>>(n.img, n.X, n.Y, B, inv3B, n.dY, n.H1, n.dZ1, n.dZ2, n.H2);
  const int nchunk = (B + kChunk - 1) / kChunk;
  k_mlp_reduce<<<nchunk, 256, 0, n.stream>>>(n.X, n.H1, n.dZ1, n.dZ2, n.H2, n.dY, B, n.partial);
  k_mlp_sum<<<(kPart + 255) / 256, 256, 0, n.stream>>>(n.partial, nchunk, inv3B, n.grad, loss_dev);
}

int reset_adam(lbm_mlp_s& n) {
  CKM(cudaMemsetAsync(n.m, 0, NPARAM * sizeof(float), n.stream));
  CKM(cudaMemsetAsync(n.v, 0, NPARAM * sizeof(float), n.stream));
  n.t = 0;
  return LBM_OK;
}

double host_uniform(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return double(z >> 11) * 0x1.0p-52 - 1.0;
}

}  // namespace

extern "C" {

const char* lbm_mlp_last_error(void) { return g_err.c_str(); }

int lbm_mlp_destroy(lbm_mlp_t net) {
  if (!net) return LBM_OK;
  free_work(*net);
  float** bufs[] = {&net->theta, &net->m, &net->v, &net->grad, &net->losses};
  for (float** b : bufs)
    if (*b) cudaFree(*b);
  if (net->img) cudaFree(net->img);
  delete net;
  return LBM_OK;
}

int lbm_mlp_create(lbm_mlp_t* out, double a, double b, double R, double cv, uint64_t seed) {
  if (!out) return fail(LBM_EINVAL, "out must be non-NULL");
  *out = nullptr;
  if (!(R > 0) || !(cv > 0) || !(a >= 0) || !(b >= 0)) return fail(LBM_EINVAL, "need R > 0, cv > 0, a >= 0, b >= 0");
  lbm_mlp_s* n = new (std::nothrow) lbm_mlp_s();
  if (!n) return fail(LBM_ENOMEM, "host allocation failed");
  std::memset(n, 0, sizeof(*n));
  n->q = {a, b, R, cv};
  for (int k = 0; k < NSCALE; ++k) n->scale[k] = (k & 1) ? 1.0 : 0.0;
  // Glorot-uniform weights from the SplitMix64 stream, zero biases
  std::vector<float> th(NPARAM, 0.f);
  const struct { int off, rows, cols; } mats[] = {{OW1, H, 2}, {OW2, H, H}, {OW3, 3, H}};
  for (const auto& mt : mats) {
    const double lim = std::sqrt(6.0 / (mt.rows + mt.cols));
    for (int k = 0; k < mt.rows * mt.cols; ++k) th[mt.off + k] = float(lim * host_uniform(seed, uint64_t(mt.off + k)));
  }
  int rc = LBM_OK;
  if (cudaMalloc(&n->theta, NPARAM * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->m, NPARAM * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->v, NPARAM * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->grad, NPARAM * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->img, sizeof(TrainImage)) != cudaSuccess) {
    rc = fail(LBM_ENOMEM, "device allocation failed");
  } else if (cudaMemcpy(n->theta, th.data(), NPARAM * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = fail(LBM_ECUDA, "copy of the initial weights failed");
  } else if ((rc = reset_adam(*n)) == LBM_OK) {
    launch_image(*n);
    if (cudaStreamSynchronize(n->stream) != cudaSuccess) rc = fail(LBM_ECUDA, "image kernel failed");
  }
  if (rc != LBM_OK) {
    lbm_mlp_destroy(n);
    return rc;
  }
  *out = n;
  return LBM_OK;
}

int lbm_mlp_set_stream(lbm_mlp_t net, void* stream) {
  if (!net) return fail(LBM_EINVAL, "NULL network");
  net->stream = static_cast<cudaStream_t>(stream);
  return LBM_OK;
}

int lbm_mlp_collect(lbm_t h, double* d_rho, double* d_e, double e_scale) {
  if (!h || !d_rho || !d_e) return fail(LBM_EINVAL, "NULL argument");
  if (lbm_moments_device(h, d_rho, nullptr, d_e, nullptr) != LBM_OK)
    return fail(LBM_ESTATE, std::string("moments: ") + lbm_last_error());
  const long long n = (long long)h->Nx * h->Ny * h->Nz;
  k_mlp_energy<<<unsigned((n + 255) / 256), 256, 0, h->stream>>>(d_rho, d_e, n, h->p.a, h->p.cv, e_scale);
  CKM(cudaGetLastError());
  CKM(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_mlp_fit_scaling(lbm_mlp_t net, const double* d_rho, const double* d_e, long long n) {
  if (!net || !d_rho || !d_e) return fail(LBM_EINVAL, "NULL argument");
  if (n < 1) return fail(LBM_EINVAL, "n must be >= 1");
  int nb = int((n + 255) / 256);
  if (nb > 1024) nb = 1024;
  double* part = nullptr;
  CKM(cudaMalloc(&part, size_t(nb) * 10 * sizeof(double)));
  k_mlp_minmax<<<nb, 256, 0, net->stream>>>(d_rho, d_e, n, net->q, part);
  std::vector<double> hp(size_t(nb) * 10);
  cudaError_t e = cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, net->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
  cudaFree(part);
  if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("scaling reduction: ") + cudaGetErrorString(e));
  double s[NSCALE];
  for (int k = 0; k < 5; ++k) {
    double lo = INFINITY, hi = -INFINITY;
    for (int b = 0; b < nb; ++b) {
      lo = std::fmin(lo, hp[b * 10 + 2 * k]);
      hi = std::fmax(hi, hp[b * 10 + 2 * k + 1]);
    }
    if (!std::isfinite(lo) || !std::isfinite(hi)) return fail(LBM_EINVAL, "non-finite samples");
    double half = 0.5 * (hi - lo);
    const double mid = 0.5 * (hi + lo);
    if (!(half > 1e-12 * std::fabs(mid))) half = std::fmax(1e-12 * std::fabs(mid), 1e-300);
    s[2 * k] = mid;
    s[2 * k + 1] = half;
  }
  return lbm_mlp_set_scaling(net, s);
}

int lbm_mlp_get_scaling(lbm_mlp_t net, double* scale) {
  if (!net || !scale) return fail(LBM_EINVAL, "NULL argument");
  for (int k = 0; k < NSCALE; ++k) scale[k] = net->scale[k];
  return LBM_OK;
}

int lbm_mlp_set_scaling(lbm_mlp_t net, const double* scale) {
  if (!net || !scale) return fail(LBM_EINVAL, "NULL argument");
  for (int k = 0; k < NSCALE; ++k) {
    if (!std::isfinite(scale[k])) return fail(LBM_EINVAL, "scaling constants must be finite");
    if ((k & 1) && !(scale[k] > 0)) return fail(LBM_EINVAL, "half-widths s and r must be > 0");
  }
  for (int k = 0; k < NSCALE; ++k) net->scale[k] = scale[k];
  net->scaled = 1;
  launch_image(*net);
  CKM(cudaGetLastError());
  CKM(cudaStreamSynchronize(net->stream));
  return LBM_OK;
}

int lbm_mlp_get_params(lbm_mlp_t net, float* theta) {
  if (!net || !theta) return fail(LBM_EINVAL, "NULL argument");
  CKM(cudaMemcpyAsync(theta, net->theta, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, net->stream));
  CKM(cudaStreamSynchronize(net->stream));
  return LBM_OK;
}

int lbm_mlp_set_params(lbm_mlp_t net, const float* theta) {
  if (!net || !theta) return fail(LBM_EINVAL, "NULL argument");
  for (int k = 0; k < NPARAM; ++k)
    if (!std::isfinite(theta[k])) return fail(LBM_EINVAL, "parameters must be finite");
  CKM(cudaMemcpyAsync(net->theta, theta, NPARAM * sizeof(float), cudaMemcpyHostToDevice, net->stream));
  int rc = reset_adam(*net);
  if (rc != LBM_OK) return rc;
  launch_image(*net);
  CKM(cudaGetLastError());
  CKM(cudaStreamSynchronize(net->stream));
  return LBM_OK;
}

int lbm_mlp_loss_grad(lbm_mlp_t net, const float* x, const float* y, int n, double* loss, float* grad) {
  if (!net || !x || !y) return fail(LBM_EINVAL, "NULL argument");
  if (n < 1 || n > kMaxBatch) return fail(LBM_EINVAL, "n must be in [1, 2^20]");
  int rc = ensure_cap(*net, n);
  if (rc != LBM_OK) return rc;
  if (net->loss_cap < 1) {
    CKM(cudaMalloc(&net->losses, sizeof(float)));
    net->loss_cap = 1;
  }
  CKM(cudaMemcpyAsync(net->X, x, size_t(n) * 2 * sizeof(float), cudaMemcpyHostToDevice, net->stream));
  CKM(cudaMemcpyAsync(net->Y, y, size_t(n) * 3 * sizeof(float), cudaMemcpyHostToDevice, net->stream));
  launch_grad(*net, n, net->losses);
  CKM(cudaGetLastError());
  float l = 0.f;
  CKM(cudaMemcpyAsync(&l, net->losses, sizeof(float), cudaMemcpyDeviceToHost, net->stream));
  if (grad) CKM(cudaMemcpyAsync(grad, net->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, net->stream));
  CKM(cudaStreamSynchronize(net->stream));
  if (loss) *loss = l;
  return LBM_OK;
}

int lbm_mlp_train(lbm_mlp_t net, const double* d_rho, const double* d_e, long long n, int batch, int steps,
                  double lr0, double lr1, double wd, uint64_t seed, float* losses) {
  if (!net || !d_rho || !d_e) return fail(LBM_EINVAL, "NULL argument");
  if (!net->scaled) return fail(LBM_ESTATE, "scaling not set (lbm_mlp_fit_scaling)");
  if (n < 1) return fail(LBM_EINVAL, "n must be >= 1");
  if (batch < 32 || batch > kMaxBatch) return fail(LBM_EINVAL, "batch must be in [32, 2^20]");
  if (steps < 0) return fail(LBM_EINVAL, "steps must be >= 0");
  if (!(lr0 >= 0) || !(lr1 >= 0) || !(wd >= 0)) return fail(LBM_EINVAL, "lr0, lr1, wd must be >= 0");
  int rc = ensure_cap(*net, batch);
  if (rc != LBM_OK) return rc;
  if (net->loss_cap < steps) {
    if (net->losses) cudaFree(net->losses);
    net->losses = nullptr;
    net->loss_cap = 0;
    CKM(cudaMalloc(&net->losses, size_t(steps) * sizeof(float)));
    net->loss_cap = steps;
  }
  const Scale sc = scale_of(*net);
  for (int k = 0; k < steps; ++k) {
    const double lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + std::cos(M_PI * k / steps));
    k_mlp_batch<<<(batch + 255) / 256, 256, 0, net->stream>>>(d_rho, d_e, n, seed, (unsigned long long)k * batch,
                                                                batch, sc, net->q, net->X, net->Y);
    launch_grad(*net, batch, net->losses + k);
    net->t += 1;
    const double bc1 = 1.0 - std::pow(0.9, double(net->t)), bc2 = 1.0 - std::pow(0.999, double(net->t));
    k_mlp_adamw<<<(NPARAM + 255) / 256, 256, 0, net->stream>>>(net->theta, net->m, net->v, net->grad, float(lr),
                                                               float(bc1), float(bc2), float(wd));
    launch_image(*net);
  }
  CKM(cudaGetLastError());
  if (losses && steps > 0)
    CKM(cudaMemcpyAsync(losses, net->losses, size_t(steps) * sizeof(float), cudaMemcpyDeviceToHost, net->stream));
  CKM(cudaStreamSynchronize(net->stream));
  return LBM_OK;
}

int lbm_mlp_predict(lbm_mlp_t net, const double* d_rho, const double* d_e, long long n, double* d_out) {
  if (!net || !d_rho || !d_e || !d_out) return fail(LBM_EINVAL, "NULL argument");
  if (!net->scaled) return fail(LBM_ESTATE, "scaling not set (lbm_mlp_fit_scaling)");
  if (n < 1) return fail(LBM_EINVAL, "n must be >= 1");
  Model<float> m{};
  m.a = float(net->q.a);
  m.b = float(net->q.b);
  m.R = float(net->q.R);
  m.cv = float(net->q.cv);
  long long blocks = ((n + 31) / 32 + 3) / 4;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_mlp_predict<<<unsigned(blocks), 128, 0, net->stream>>>(&net->img->fwd, m, d_rho, d_e, n, d_out);
  CKM(cudaGetLastError());
  CKM(cudaStreamSynchronize(net->stream));
  return LBM_OK;
}

int lbm_mlp_attach(lbm_t h, lbm_mlp_t net) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (!net) {
    h->closure = LBM_CLOSURE_EXACT;
    h->p.mlp = nullptr;
    h->tile_cfg = 0;                 // tile lists differ per closure (lbm_autotune)
    return LBM_OK;
  }
  if (h->precision != LBM_FP32) return fail(LBM_EINVAL, "the learned closure needs FP32 population storage");
  if (h->p.eos_kind != LBM_EOS_VDW) return fail(LBM_EINVAL, "the learned closure is trained on the van der Waals fluid");
  if (!net->scaled) return fail(LBM_ESTATE, "scaling not set (lbm_mlp_fit_scaling)");
  if (!h->mlp_img) CKM(cudaMalloc(&h->mlp_img, sizeof(Image)));
  // the network's stream finished its last update before its call returned
  CKM(cudaMemcpyAsync(h->mlp_img, &net->img->fwd, sizeof(Image), cudaMemcpyDeviceToDevice, h->stream));
  CKM(cudaStreamSynchronize(h->stream));
  h->p.mlp = h->mlp_img;
  h->closure = LBM_CLOSURE_MLP;
  h->tile_cfg = 0;
  return LBM_OK;
}

int lbm_get_closure(lbm_t h) { return h ? h->closure : LBM_CLOSURE_EXACT; }

}  // extern "C"
