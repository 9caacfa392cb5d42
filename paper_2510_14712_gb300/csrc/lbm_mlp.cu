// lbm_mlp.cu - training and standalone evaluation of the learned closure and
// the lbm_mlp_* interface of include/lbm_mlp.h.
//
// One training step is five launches on the network's stream:
//   k_mlp_batch     draw the minibatch (SplitMix64 indices), exact FP64 labels
//   k_mlp_train_tc  forward pass, backward pass and every weight gradient of
//                   the minibatch on the fifth-generation tensor cores
//                   (tcgen05.mma, BF16 hi + lo operands, FP32 accumulators in
//                   tensor memory): one partial gradient per block
//   k_mlp_sum       fixed-order sum of the partials (deterministic)
//   k_mlp_adamw     AdamW update of the FP32 master weights
//   k_mlp_image     bfloat16 weights, mma fragments and operand images for the
//                   next forward
// lbm_mlp_set_mma(LBM_MLP_MMA_WARP) selects the warp-level form instead:
//   k_mlp_fwd_bwd   per-sample forward and backward pass (mma.sync for the
//                   64 x 64 products), per-sample factors to memory
//   k_mlp_reduce    per 128-sample chunk: dW2 = dZ2^T H1 (mma.sync, bfloat16
//                   dz2 and h1), the small gradients on FP32 pipes
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm_mlp.h"
#include "lbm_internal.cuh"
#include "lbm_mlp.cuh"
#include "lbm_mlp_tc.cuh"

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
constexpr int kImageThreads = 2048 + H + 1 + H * H;     // threads of k_mlp_image
constexpr size_t kW2kBytes = 2 * H * H * 2;             // the two bfloat16 W2 operands of k_mlp_train_tc

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
__global__ void k_mlp_image(const float* __restrict__ th, Scale sc, TrainImage* __restrict__ img,
                            uint4* __restrict__ w2k) {
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
  } else if (i < kImageThreads) {
    // K-major operands of the tensor-core training kernel: [n = j2][k = j1]
    // (forward) and [n = j1][k = j2] (backward), element (n, k) at
    // tc::kmajor_offset(n, k, 64)
    const int e = i - (2048 + H + 1), n = e >> 6, k = e & (H - 1);
    unsigned short* w = reinterpret_cast<unsigned short*>(w2k);
    const uint32_t o = tc::kmajor_offset(n, k, H) / 2;
    w[o] = __bfloat16_as_ushort(__float2bfloat16_rn(W2[n * H + k]));
    w[H * H + o] = __bfloat16_as_ushort(__float2bfloat16_rn(W2[k * H + n]));
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

// The whole training pass of one minibatch on the fifth-generation tensor
// cores (tcgen05.mma, BF16 operands, FP32 accumulators in tensor memory; the
// primitives are in lbm_mlp_tc.cuh).  One block of 512 threads per SM loops
// over groups of 128 samples.  Sample i of a group is row i of the
// per-sample products and TMEM lane i of their accumulators; four threads
// share it, one per quarter of the 64 hidden units (warp w: lanes
// 32 (w % 4) .. + 31, the lanes its TMEM loads may address; units
// 16 (w / 4) .. + 15), and add their shares of the network output through
// shared memory (in quarter order).
//
// Per group (FP32 values enter the products split into bfloat16 hi + lo, the
// split of lbm_mlp.cuh, so that every product is exact to about 2^-16):
//   forward   D1 = H1 W2^T                 (z2 - b2; A = h1 hi, lo; B = W2)
//   backward  D2 = dZ2 W2                  (dL/dh1; A = dz2 hi, lo; B = W2^T)
//   gradients G2 += [dZ2hi | dZ2lo]^T [H1hi | H1lo | 1]        (dW2, db2)
//             G3 += [H2hi | H2lo]^T X,  G1 += [dZ1hi | dZ1lo]^T X
//             X = [x0 hi, lo, x1 hi, lo, 1, dy0 hi, lo, dy1 hi, lo, dy2 hi, lo]
//                                          (dW3; dW1, db1)
// The three gradient products contract over the samples: their operands are
// the same per-sample rows, read as MN-major matrices.  G1, G2, G3 accumulate
// over all groups of the block; db3 and the loss sum are block reductions.
// The block then writes one partial gradient (the kPart record of
// k_mlp_reduce) and k_mlp_sum adds the partials in block order.
//
// Shared memory: per-sample rows of C bfloat16 columns, element (s, c) at
// tc::kmajor_offset(s, c, C).  As an operand with rows = samples (forward,
// backward) this is K-major (leading byte offset 128, stride byte offset
// C/8 * 128); with rows = columns and K = samples (gradients) it is MN-major,
// whose leading byte offset is the K-direction step between groups of 8
// samples (C/8 * 128) and whose stride byte offset is the step between groups
// of 8 columns (128).
//   HB  [128][144]  h1 hi (0-63), h1 lo (64-127), 1 (128), 0 (129-143)
//   DZ  [128][128]  dz2 hi, lo          Z1B [128][128]  dz1 hi, lo
//   H2B [128][128]  h2 hi, lo           XB  [128][16]   X above, 0 (11-15)
//   WF, WB [64][64] W2 as [n = j2][k = j1] and [n = j1][k = j2] (k_mlp_image)
//   YP  [4][128]    float4 shares of the output y, one per quarter
//   WS              layers 1 and 3 and the biases (WeightsSm)
// Tensor memory (512 columns): D1 0-63, D2 64-127, G1 128-143, G3 144-159,
// G2 256-399.
//
// Synchronisation: thread 0 issues the MMAs and commits them to one
// mbarrier; the block waits on its phase (bounded: a wait that runs out sets
// bit 1 of *status, and the block stops after a last bounded wait and frees
// its tensor memory).  G1 of a group is issued with the forward product of
// the next group (or after the last group), so a group takes two waits.
namespace tcl {
constexpr int kRows = 128;                    // samples per group
constexpr int kSplit = 4, kFeat = H / kSplit; // threads per sample, features per thread
constexpr int kThreads = kRows * kSplit;
constexpr int kCH = 144, kCZ = 128, kCX = 16;
constexpr int oHB = 0, oDZ = oHB + kRows * kCH * 2, oZ1 = oDZ + kRows * kCZ * 2, oH2 = oZ1 + kRows * kCZ * 2,
              oXB = oH2 + kRows * kCZ * 2, oWF = oXB + kRows * kCX * 2, oWB = oWF + H * H * 2,
              oYP = oWB + H * H * 2, oWS = oYP + kSplit * kRows * 4 * 4, oBar = oWS + 2112;
constexpr size_t kSmem = size_t(oBar) + 64;
constexpr uint32_t cD1 = 0, cD2 = 64, cG1 = 128, cG3 = 144, cG2 = 256, kCols = 512;
constexpr uint32_t kWaitLimit = 1u << 22;
static_assert(kSmem <= 227 * 1024, "shared memory of one block");
static_assert(kSmem > 114 * 1024, "one block per SM: the block takes all 512 TMEM columns");
}  // namespace tcl

// layers 1 and 3 of the image in shared memory
struct WeightsSm {
  float4 l1[H];
  float b2[H];
  float w3[3][H];
  float b3[4];
};
static_assert(sizeof(WeightsSm) <= 2112, "weights region of k_mlp_train_tc");

// eight consecutive columns c0 .. c0 + 7 of row `row`: hi to column c0, lo to column c0 + lo_off
__device__ __forceinline__ void put8_split(unsigned char* buf, int C, int row, int c0, int lo_off, const float* v) {
  uint32_t hi[4], lo[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) split_bf16(v[2 * q], v[2 * q + 1], hi[q], lo[q]);
  *reinterpret_cast<uint4*>(buf + tc::kmajor_offset(row, c0, C)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4*>(buf + tc::kmajor_offset(row, c0 + lo_off, C)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

// accumulate = 0 overwrites D on the first K step of a product
__device__ __forceinline__ void mma_k16_steps(uint32_t d, uint32_t a0, uint32_t a_step, uint32_t a_lbo, uint32_t a_sbo,
                                              uint32_t b0, uint32_t b_step, uint32_t b_lbo, uint32_t b_sbo,
                                              uint32_t idesc, int steps, bool accumulate) {
  for (int ks = 0; ks < steps; ++ks)
    tc::mma_bf16(d, tc::smem_desc(a0 + ks * a_step, a_lbo, a_sbo), tc::smem_desc(b0 + ks * b_step, b_lbo, b_sbo),
                 idesc, (accumulate || ks > 0) ? 1u : 0u);
}

__global__ void __launch_bounds__(tcl::kThreads, 1)
    k_mlp_train_tc(const TrainImage* __restrict__ img, const uint4* __restrict__ w2k, const float* __restrict__ X,
                   const float* __restrict__ Y, int B, float* __restrict__ partial, unsigned* __restrict__ status) {
  using namespace tcl;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* hb = sm + oHB;
  unsigned char* dzb = sm + oDZ;
  unsigned char* z1b = sm + oZ1;
  unsigned char* h2b = sm + oH2;
  unsigned char* xb = sm + oXB;
  float* ypart = reinterpret_cast<float*>(sm + oYP);                    // [kSplit][kRows][4]
  WeightsSm& ws = *reinterpret_cast<WeightsSm*>(sm + oWS);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + oBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + oBar + 8);
  const Image& w = img->fwd;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // warp w: TMEM lanes (= rows) 32 (w % 4) .. + 31, features 16 (w / 4) .. + 15
  const int quad = warp & 3, cp = warp >> 2;
  const int row = 32 * quad + lane, f0 = kFeat * cp;
  const float inv3B = float(1.0 / (3.0 * double(B)));
  // W2 in both operand layouts (16 KB, consecutive in w2k and in shared memory)
  for (int i = tid; i < 2 * H * H * 2 / 16; i += kThreads) reinterpret_cast<uint4*>(sm + oWF)[i] = __ldg(&w2k[i]);
  // layers 1 and 3 and the biases (read by every thread in every group)
  if (tid < H) {
    ws.l1[tid] = w.l1[tid];
    ws.b2[tid] = w.b2[tid];
#pragma unroll
    for (int o = 0; o < 3; ++o) ws.w3[o][tid] = w.w3[o][tid];
  } else if (tid < H + 4) {
    ws.b3[tid - H] = w.b3[tid - H];
  }
  // the constant columns of HB: 1 (bfloat16 0x3F80) at column 128, zeros to 143
  if (cp == 0) {
    *reinterpret_cast<uint4*>(hb + tc::kmajor_offset(row, 128, kCH)) = make_uint4(0x3F80u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(hb + tc::kmajor_offset(row, 136, kCH)) = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) tc::mbar_init(bar, 1);
  if (warp == 0) tc::tmem_alloc(tslot, kCols);
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t lanes = uint32_t(32 * quad) << 16;
  const uint32_t a_hb = tc::smem_addr(hb), a_dz = tc::smem_addr(dzb), a_z1 = tc::smem_addr(z1b);
  const uint32_t a_h2 = tc::smem_addr(h2b), a_xb = tc::smem_addr(xb);
  const uint32_t a_wf = tc::smem_addr(sm + oWF), a_wb = tc::smem_addr(sm + oWB);
  constexpr uint32_t kMN = (1u << 15) | (1u << 16);                    // A and B MN-major
  const uint32_t id64 = tc::idesc_bf16_f32(kRows, H);
  const uint32_t id144 = tc::idesc_bf16_f32(kRows, kCH) | kMN, id16 = tc::idesc_bf16_f32(kRows, kCX) | kMN;
  constexpr uint32_t sHB = kCH / 8 * 128, sZ = kCZ / 8 * 128, sX = kCX / 8 * 128;
  // G1 += [dZ1hi | dZ1lo]^T X over the 128 samples of the group in Z1B and XB
  auto issue_g1 = [&](bool acc) {
    mma_k16_steps(tmem + cG1, a_z1, 2 * sZ, sZ, 128, a_xb, 2 * sX, sX, 128, id16, kRows / 16, acc);
  };
  uint32_t phase = 0;
  bool ok = true, g1_pending = false, g1_acc = false, g23_acc = false;
  float acc_dy[3] = {0.f, 0.f, 0.f}, acc_l2 = 0.f;                     // kept by the cp = 0 threads
  for (int s0 = blockIdx.x * kRows; s0 < B; s0 += gridDim.x * kRows) {
    const int s = s0 + row;
    const bool valid = s < B;
    const float x0 = valid ? X[2 * s] : 0.f, x1 = valid ? X[2 * s + 1] : 0.f;
    // layer 1: features f0 .. f0 + 15 of h1 into HB, gelu'(z1) kept
    float dg1[kFeat];
#pragma unroll
    for (int jb = 0; jb < kFeat; jb += 8) {
      float h[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 wa = ws.l1[f0 + jb + q];
        gelu_d(fmaf(wa.x, x0, fmaf(wa.y, x1, wa.z)), h[q], dg1[jb + q]);
      }
      put8_split(hb, kCH, row, f0 + jb, H, h);
    }
    tc::fence_smem_to_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      if (g1_pending) issue_g1(g1_acc);                                   // the previous group's G1
      g1_acc = g1_acc || g1_pending;
      mma_k16_steps(tmem + cD1, a_hb, 256, 128, sHB, a_wf, 256, 128, 1024, id64, H / 16, false);        // h1 hi
      mma_k16_steps(tmem + cD1, a_hb + 1024, 256, 128, sHB, a_wf, 256, 128, 1024, id64, H / 16, true);  // h1 lo
      tc::commit(bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(bar, phase, kWaitLimit));
    if (!ok) break;
    phase ^= 1;
    tc::fence_after_sync();
    // z2 = b2 + D1 (this thread's 16 columns): h2 into H2B, gelu'(z2) kept,
    // this quarter's share of y = W3 h2 to shared memory
    float dg[kFeat];
    {
      float v[kFeat], h2[kFeat], yp[3] = {0.f, 0.f, 0.f};
      tc::tmem_ld16(tmem + lanes + cD1 + f0, v);
#pragma unroll
      for (int k = 0; k < kFeat; ++k) {
        gelu_d(v[k] + ws.b2[f0 + k], h2[k], dg[k]);
#pragma unroll
        for (int o = 0; o < 3; ++o) yp[o] = fmaf(ws.w3[o][f0 + k], h2[k], yp[o]);
      }
      put8_split(h2b, kCZ, row, f0, H, h2);
      put8_split(h2b, kCZ, row, f0 + 8, H, h2 + 8);
      *reinterpret_cast<float4*>(ypart + 4 * (cp * kRows + row)) = make_float4(yp[0], yp[1], yp[2], 0.f);
    }
    __syncthreads();
    float dy[3];
    {
      float y[3] = {ws.b3[0], ws.b3[1], ws.b3[2]};
#pragma unroll
      for (int c = 0; c < kSplit; ++c) {                                 // quarters in order
        const float4 t = *reinterpret_cast<const float4*>(ypart + 4 * (c * kRows + row));
        y[0] += t.x;
        y[1] += t.y;
        y[2] += t.z;
      }
      float l2 = 0.f;
#pragma unroll
      for (int o = 0; o < 3; ++o) {
        const float r = valid ? y[o] - Y[3 * s + o] : 0.f;
        dy[o] = 2.f * r * inv3B;
        l2 += r * r;
      }
      if (cp == 0) {
#pragma unroll
        for (int o = 0; o < 3; ++o) acc_dy[o] += dy[o];
        acc_l2 += l2;
        const float xv[8] = {x0, x1, 1.f, 0.f, dy[0], dy[1], dy[2], 0.f};
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) split_bf16(xv[2 * q], xv[2 * q + 1], hi[q], lo[q]);
        // columns: x0 hi, x0 lo, x1 hi, x1 lo, 1, dy0 hi, dy0 lo, dy1 hi | dy1 lo, dy2 hi, dy2 lo, 0 ...
        const uint32_t one = hi[1] & 0xffffu;
        const uint4 c0 = make_uint4((hi[0] & 0xffffu) | (lo[0] << 16), (hi[0] >> 16) | (lo[0] & 0xffff0000u),
                                    one | (hi[2] << 16), (lo[2] & 0xffffu) | (hi[2] & 0xffff0000u));
        const uint4 c1 = make_uint4((lo[2] >> 16) | (hi[3] << 16), lo[3] & 0xffffu, 0u, 0u);
        *reinterpret_cast<uint4*>(xb + tc::kmajor_offset(row, 0, kCX)) = c0;
        *reinterpret_cast<uint4*>(xb + tc::kmajor_offset(row, 8, kCX)) = c1;
      }
    }
    // dz2 = (W3^T dy) gelu'(z2) into DZ
    {
      float d[kFeat];
#pragma unroll
      for (int k = 0; k < kFeat; ++k) {
        const int j = f0 + k;
        d[k] = (dy[0] * ws.w3[0][j] + dy[1] * ws.w3[1][j] + dy[2] * ws.w3[2][j]) * dg[k];
      }
      put8_split(dzb, kCZ, row, f0, H, d);
      put8_split(dzb, kCZ, row, f0 + 8, H, d + 8);
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      mma_k16_steps(tmem + cD2, a_dz, 256, 128, sZ, a_wb, 256, 128, 1024, id64, H / 16, false);         // dz2 hi
      mma_k16_steps(tmem + cD2, a_dz + 1024, 256, 128, sZ, a_wb, 256, 128, 1024, id64, H / 16, true);   // dz2 lo
      mma_k16_steps(tmem + cG2, a_dz, 2 * sZ, sZ, 128, a_hb, 2 * sHB, sHB, 128, id144, kRows / 16, g23_acc);
      mma_k16_steps(tmem + cG3, a_h2, 2 * sZ, sZ, 128, a_xb, 2 * sX, sX, 128, id16, kRows / 16, g23_acc);
      g23_acc = true;
      tc::commit(bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(bar, phase, kWaitLimit));
    if (!ok) break;
    phase ^= 1;
    tc::fence_after_sync();
    // dz1 = dh1 gelu'(z1), dh1 = D2 (this thread's 16 columns): into Z1B
    {
      float v[kFeat], d[kFeat];
      tc::tmem_ld16(tmem + lanes + cD2 + f0, v);
#pragma unroll
      for (int k = 0; k < kFeat; ++k) d[k] = v[k] * dg1[k];
      put8_split(z1b, kCZ, row, f0, H, d);
      put8_split(z1b, kCZ, row, f0 + 8, H, d + 8);
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();                                                     // Z1B, XB complete; D reads done
    g1_pending = true;
  }
  if (ok && g1_pending) {
    if (tid == 0) {
      tc::fence_after_sync();
      issue_g1(g1_acc);
      tc::commit(bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(bar, phase, kWaitLimit));
    if (ok) phase ^= 1;
    tc::fence_after_sync();
  }
  if (ok) {
    float* out = partial + size_t(blockIdx.x) * kPart;
    if (!g1_pending) {                                                   // no group: a zero partial
      for (int p = tid; p < kPart; p += kThreads) out[p] = 0.f;
    } else {
      // Row m of G1, G2, G3 is column m of [hi | lo]: rows j and j + 64 add up to
      // the gradient of unit j.  Lane quadrants 2 and 3 (rows 64-127) leave their
      // row sums in shared memory (DZ is free: every product has completed),
      // quadrants 0 and 1 add them to their own and write the partial.
      constexpr int kRed = 73;                                           // odd row stride: no bank conflicts
      float* red = reinterpret_cast<float*>(dzb);
      const bool upper = quad >= 2;
      float* r = red + (row & 63) * kRed;
      float a[16], b[16];
      tc::tmem_ld16(tmem + lanes + cG2 + f0, a);
      tc::tmem_ld16(tmem + lanes + cG2 + H + f0, b);
      float g2b[16], g1[16], g3[16];
      if (cp == 0) {
        tc::tmem_ld16(tmem + lanes + cG2 + 2 * H, g2b);
        tc::tmem_ld16(tmem + lanes + cG1, g1);
        tc::tmem_ld16(tmem + lanes + cG3, g3);
      }
      if (upper) {
#pragma unroll
        for (int k = 0; k < 16; ++k) r[f0 + k] = a[k] + b[k];
        if (cp == 0) {
          r[64] = g2b[0];
          r[65] = g1[0] + g1[1];
          r[66] = g1[2] + g1[3];
          r[67] = g1[4];
#pragma unroll
          for (int o = 0; o < 3; ++o) r[68 + o] = g3[5 + 2 * o] + g3[6 + 2 * o];
        }
      }
      __syncthreads();
      if (!upper) {
        const int j = row;
#pragma unroll
        for (int k = 0; k < 16; ++k) out[OW2 + j * H + f0 + k] = (a[k] + b[k]) + r[f0 + k];
        if (cp == 0) {
          out[OB2 + j] = g2b[0] + r[64];
          out[OW1 + 2 * j] = (g1[0] + g1[1]) + r[65];
          out[OW1 + 2 * j + 1] = (g1[2] + g1[3]) + r[66];
          out[OB1 + j] = g1[4] + r[67];
#pragma unroll
          for (int o = 0; o < 3; ++o) out[OW3 + o * H + j] = (g3[5 + 2 * o] + g3[6 + 2 * o]) + r[68 + o];
        }
      }
      // db3 and the loss sum (held by the cp = 0 threads): butterfly over the
      // warp, then the warps in order
      float t[4] = {acc_dy[0], acc_dy[1], acc_dy[2], acc_l2};
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) t[q] += __shfl_xor_sync(0xffffffffu, t[q], m);
      float* wsum = reinterpret_cast<float*>(xb);
      if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) wsum[4 * warp + q] = t[q];
      __syncthreads();
      if (tid < 4) {
        float v = 0.f;
        for (int k = 0; k < 4; ++k) v += wsum[4 * k + tid];              // warps 0-3: the cp = 0 quarter
        out[tid < 3 ? OB3 + tid : NPARAM] = v;
      }
    }
  } else {
    if (tid == 0) atomicOr(status, 2u);
    tc::mbar_wait(bar, phase, kWaitLimit);                               // the products still in flight, if any
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, kCols);
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

// Deterministic sum of the partial records: a block takes 32 entries of the
// record and eight slices of the partials; each thread adds its slice in
// order, then the slices are added in order.
constexpr int kSumCols = 32, kSumSlices = 8, kSumBlocks = (kPart + kSumCols - 1) / kSumCols;
__global__ void __launch_bounds__(kSumCols * kSumSlices)
    k_mlp_sum(const float* __restrict__ partial, int nchunk, float loss_scale, float* __restrict__ grad,
              float* __restrict__ loss) {
  __shared__ double s[kSumSlices][kSumCols + 1];
  const int col = threadIdx.x % kSumCols, sl = threadIdx.x / kSumCols;
  const int p = blockIdx.x * kSumCols + col;
  double acc = 0.0;
  if (p < kPart) {
    const int per = (nchunk + kSumSlices - 1) / kSumSlices;
    const int c1 = min(nchunk, (sl + 1) * per);
    int c = sl * per;
    for (; c + 4 <= c1; c += 4) {
      float v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = __ldg(&partial[size_t(c + k) * kPart + p]);
#pragma unroll
      for (int k = 0; k < 4; ++k) acc += v[k];
    }
    for (; c < c1; ++c) acc += partial[size_t(c) * kPart + p];
  }
  s[sl][col] = acc;
  __syncthreads();
  if (sl == 0 && p < kPart) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < kSumSlices; ++k) t += s[k][col];
    if (p < NPARAM) grad[p] = float(t);
    else *loss = float(t * loss_scale);
  }
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
  int mma;                           // LBM_MLP_MMA_TCGEN05 (default) or LBM_MLP_MMA_WARP
  unsigned* status;                  // device word: bit 1 = a tensor-core completion wait ran out
  uint4* w2k;                        // W2 as the two K-major bfloat16 operands of k_mlp_train_tc
  bool tc_ready;                     // dynamic shared-memory size of the tensor-core kernel set, sms read
  int sms;                           // multiprocessors of the device
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
  k_mlp_image<<<(kImageThreads + 255) / 256, 256, 0, n.stream>>>(n.theta, scale_of(n), n.img, n.w2k);
}

// loss (written to loss_dev) and gradient (n.grad) on the B samples in n.X, n.Y
int launch_grad(lbm_mlp_s& n, int B, float* loss_dev) {
  const int ngrp = (B + 31) / 32;
  int blocks = (ngrp + 3) / 4;
  if (blocks > 152 * 8) blocks = 152 * 8;
  const float inv3B = float(1.0 / (3.0 * B));
  if (n.mma == LBM_MLP_MMA_TCGEN05) {
    if (!n.tc_ready) {
      int dev = 0;
      CKM(cudaGetDevice(&dev));
      CKM(cudaDeviceGetAttribute(&n.sms, cudaDevAttrMultiProcessorCount, dev));
      CKM(cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tcl::kSmem)));
      n.tc_ready = true;
    }
    // one block per SM (all 512 TMEM columns), every block at least one group
    const int groups = (B + tcl::kRows - 1) / tcl::kRows;
    const int grid = groups < n.sms ? groups : n.sms;
    k_mlp_train_tc<<<grid, tcl::kThreads, tcl::kSmem, n.stream>>>(n.img, n.w2k, n.X, n.Y, B, n.partial, n.status);
    k_mlp_sum<<<kSumBlocks, kSumCols * kSumSlices, 0, n.stream>>>(n.partial, grid, inv3B, n.grad, loss_dev);
    return LBM_OK;
  }
  k_mlp_fwd_bwd<<<blocks, 128, 0, n.stream>>>(n.img, n.X, n.Y, B, inv3B, n.dY, n.H1, n.dZ1, n.dZ2, n.H2);
  const int nchunk = (B + kChunk - 1) / kChunk;
  k_mlp_reduce<<<nchunk, 256, 0, n.stream>>>(n.X, n.H1, n.dZ1, n.dZ2, n.H2, n.dY, B, n.partial);
  k_mlp_sum<<<kSumBlocks, kSumCols * kSumSlices, 0, n.stream>>>(n.partial, nchunk, inv3B, n.grad, loss_dev);
  return LBM_OK;
}

// after a synchronisation: a tensor-core wait that ran out is an error of the call
int check_status(lbm_mlp_s& n) {
  unsigned st = 0;
  CKM(cudaMemcpy(&st, n.status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (st) {
    CKM(cudaMemset(n.status, 0, sizeof(unsigned)));
    return fail(LBM_ECUDA, "a tensor-core completion wait of the training kernel ran out");
  }
  return LBM_OK;
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
  if (net->w2k) cudaFree(net->w2k);
  if (net->status) cudaFree(net->status);
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
  n->mma = LBM_MLP_MMA_TCGEN05;
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
      cudaMalloc(&n->img, sizeof(TrainImage)) != cudaSuccess || cudaMalloc(&n->w2k, kW2kBytes) != cudaSuccess ||
      cudaMalloc(&n->status, sizeof(unsigned)) != cudaSuccess || cudaMemset(n->status, 0, sizeof(unsigned)) != cudaSuccess) {
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
  rc = launch_grad(*net, n, net->losses);
  if (rc != LBM_OK) return rc;
  CKM(cudaGetLastError());
  float l = 0.f;
  CKM(cudaMemcpyAsync(&l, net->losses, sizeof(float), cudaMemcpyDeviceToHost, net->stream));
  if (grad) CKM(cudaMemcpyAsync(grad, net->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, net->stream));
  CKM(cudaStreamSynchronize(net->stream));
  rc = check_status(*net);
  if (rc != LBM_OK) return rc;
  if (loss) *loss = l;
  return LBM_OK;
}

int lbm_mlp_set_mma(lbm_mlp_t net, int kind) {
  if (!net) return fail(LBM_EINVAL, "NULL network");
  if (kind != LBM_MLP_MMA_TCGEN05 && kind != LBM_MLP_MMA_WARP) return fail(LBM_EINVAL, "unknown contraction path");
  net->mma = kind;
  return LBM_OK;
}

int lbm_mlp_get_mma(lbm_mlp_t net) { return net ? net->mma : LBM_MLP_MMA_TCGEN05; }

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
    k_mlp_batch<<<(batch + 63) / 64, 64, 0, net->stream>>>(d_rho, d_e, n, seed, (unsigned long long)k * batch,
                                                                batch, sc, net->q, net->X, net->Y);
    rc = launch_grad(*net, batch, net->losses + k);
    if (rc != LBM_OK) return rc;
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
  return check_status(*net);
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
