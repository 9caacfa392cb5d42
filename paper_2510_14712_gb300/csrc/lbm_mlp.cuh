// lbm_mlp.cuh - the learned thermodynamic closure (device side).
//
// A 2 -> 64 -> 64 -> 3 multilayer perceptron maps the normalised state
// x = ((rho - c_rho)/s_rho, (e - c_e)/s_e) to the normalised closure outputs
// y = ((T - m_T)/r_T, (P - m_P)/r_P, (c_s^2 - m_c)/r_c) of the fluid (the
// exact relations it replaces: Eqs. lbm_temp, Pvdw, vdW_speed_of_sound):
//
//   h1 = gelu(W1 x + b1),  h2 = gelu(W2 h1 + b2),  y = W3 h2 + b3.
//
// Number formats.  The weights W1, W2, W3 are bfloat16 values (the network
// is trained with its forward pass on the rounded weights); biases, inputs
// and activations are FP32.  The 64 x 64 contraction W2 h1 runs on the tensor
// cores as BF16 x BF16 -> FP32 (mma.sync m16n8k16) with each activation split
// into two bfloat16 terms h = hi + lo (hi = bf16(h), lo = bf16(h - hi)), so
// the product is exact to about 2^-16 relative (the split of Henry, Tang and
// Heinecke, "Leveraging the bfloat16 artificial intelligence datatype for
// higher-precision computations", 2019).  Layers 1 and 3 (2 and 3 wide) run on
// the FP32 pipes.
//
// gelu is the tanh form of Hendrycks and Gimpel:
//   gelu(z) = z (1 + tanh(u)) / 2 = z / (1 + exp(-2u)),  u = k0 (z + k1 z^3),
// k0 = sqrt(2 / pi), k1 = 0.044715, evaluated through exp and a division
// (relative error a few ulp).
//
// Warp layout.  A warp evaluates the network for 32 nodes (one per lane).
// The 32 nodes are two m-tiles of 16 rows; for m16n8k16 lane l = 4g + t holds
// rows g and g + 8 of a tile and columns 2t, 2t + 1 (+ 8) of each 16-wide
// k-step (A operand) or 8-wide n-tile (accumulator).  Layer 1 is computed
// directly in the A-operand layout (inputs of rows g, g + 8 fetched by
// shuffles); the accumulator of layer 2 feeds layer 3 in place; the three
// outputs are summed over the four lanes of a row and returned to the lane
// that owns the node.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "lbm_device.cuh"

namespace lbm {
namespace mlp {

constexpr int H = 64;                                   // hidden width
constexpr int OW1 = 0, OB1 = OW1 + 2 * H, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + 3 * H;
constexpr int NPARAM = OB3 + 3;                         // 4547: W1, b1, W2, b2, W3, b3 (W row-major [out][in])
constexpr int NSCALE = 10;                              // c_rho, s_rho, c_e, s_e, m_T, r_T, m_P, r_P, m_c, r_c

// The inference image: what a kernel copies into shared memory.
struct alignas(16) Image {
  float norm[12];             // c_rho, 1/s_rho, c_e, 1/s_e, m_T, r_T, m_P, r_P, m_c, r_c, 0, 0
  float4 l1[H];               // {W1[j][0], W1[j][1], b1[j], 0} (W1 bf16-valued)
  float b2[H];
  float w3[3][H];             // bf16-valued
  float b3[4];
  uint32_t w2f[4][8][32][2];  // layer-2 B fragments: [k-step][n-tile][lane][reg], bf16x2
};
static_assert(sizeof(Image) % 16 == 0, "image is copied in 16-byte words");

// Backward fragments of W2 for training (B[k = j2][n = j1] = W2[j2][j1]).
struct alignas(16) TrainImage {
  Image fwd;
  uint32_t w2b[4][8][32][2];
};

constexpr float kG0 = 0.7978845608028654f;              // sqrt(2 / pi)
constexpr float kG1 = 0.044715f;

__device__ __forceinline__ float gelu(float z) {
  float u = kG0 * fmaf(kG1 * z, z * z, z);
  u = fmaxf(u, -40.f);                                  // exp(80) stays finite
  return __fdividef(z, 1.f + __expf(-2.f * u));
}

// gelu and its derivative: s = sigma(2u), gelu = z s,
// gelu' = s + z s (1 - s) 2 k0 (1 + 3 k1 z^2)
__device__ __forceinline__ void gelu_d(float z, float& g, float& dg) {
  float u = kG0 * fmaf(kG1 * z, z * z, z);
  u = fmaxf(u, -40.f);
  const float s = __fdividef(1.f, 1.f + __expf(-2.f * u));
  g = z * s;
  dg = s + z * s * (1.f - s) * (2.f * kG0) * fmaf(3.f * kG1, z * z, 1.f);
}

// {lo, hi} -> bf16x2 register (lo in the low half), round to nearest even
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// two-term split of a pair: hi = bf16(a), lo = bf16(a - hi)
__device__ __forceinline__ void split_bf16(float a0, float a1, uint32_t& hi, uint32_t& lo) {
  hi = pack_bf16(a0, a1);
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
  lo = pack_bf16(a0 - h0, a1 - h1);
}

// D += A B for one m16n8k16 tile, BF16 inputs, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Layer 1 of m-tile rows (g, g+8) in A-operand layout, split into hi / lo.
// xr[h][i]: input i of row g + 8h.  Register r of k-step ks holds columns
// 16 ks + 8 (r >> 1) + 2t, +1 of row g + 8 (r & 1).
__device__ __forceinline__ void layer1_frag(const Image& w, const float (&xr)[2][2], uint32_t (&ah)[4][4],
                                            uint32_t (&al)[4][4]) {
  const int t = threadIdx.x & 3;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int c = 16 * ks + 8 * half + 2 * t;
      const float4 wa = w.l1[c], wb = w.l1[c + 1];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float za = fmaf(wa.x, xr[h][0], fmaf(wa.y, xr[h][1], wa.z));
        const float zb = fmaf(wb.x, xr[h][0], fmaf(wb.y, xr[h][1], wb.z));
        split_bf16(gelu(za), gelu(zb), ah[ks][h + 2 * half], al[ks][h + 2 * half]);
      }
    }
}

// Network outputs for the 32 nodes of a warp.  Every lane of the warp must
// call this (mma.sync is warp-collective); (x0, x1) are the lane's own
// normalised inputs, y its three normalised outputs.
__device__ __forceinline__ void forward_warp(const Image& w, float x0, float x1, float (&y)[3]) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float yp[2][2][3];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    float xr[2][2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      xr[h][0] = __shfl_sync(full, x0, 16 * mt + 8 * h + g);
      xr[h][1] = __shfl_sync(full, x1, 16 * mt + 8 * h + g);
    }
    uint32_t ah[4][4], al[4][4];
    layer1_frag(w, xr, ah, al);
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int o = 0; o < 3; ++o) yp[mt][h][o] = 0.f;
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
#pragma unroll
      for (int q = 0; q < 4; ++q) d[q] = gelu(d[q]);
#pragma unroll
      for (int o = 0; o < 3; ++o) {
        const float w0 = w.w3[o][c], w1 = w.w3[o][c + 1];
        yp[mt][0][o] = fmaf(w0, d[0], fmaf(w1, d[1], yp[mt][0][o]));
        yp[mt][1][o] = fmaf(w0, d[2], fmaf(w1, d[3], yp[mt][1][o]));
      }
    }
  }
  // sum over the four lanes of each row, then hand row r to lane r
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int o = 0; o < 3; ++o) {
        float v = yp[mt][h][o];
        v += __shfl_xor_sync(full, v, 1);
        v += __shfl_xor_sync(full, v, 2);
        yp[mt][h][o] = v;
      }
  const int src = 4 * (lane & 7), mt_own = lane >> 4, h_own = (lane >> 3) & 1;
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    float v = 0.f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float s = __shfl_sync(full, yp[mt][h][o], src);
        if (mt == mt_own && h == h_own) v = s;
      }
    y[o] = v + w.b3[o];
  }
}

// The closure at one node: network outputs where the normalised input lies in
// the training box [-1, 1]^2, the exact van der Waals relations elsewhere
// (Eqs. lbm_temp, Pvdw, vdW_speed_of_sound) and for non-finite input.
// Warp-collective; `act` marks the lanes with a real node.  Returns whether
// the network was used.
__device__ __forceinline__ bool closure_warp(const Image& w, const Model<float>& m, float rho, float e, bool act,
                                             float& T, float& P, float& cs2) {
  float x0 = (rho - w.norm[0]) * w.norm[1], x1 = (e - w.norm[2]) * w.norm[3];
  const bool inr = act && fabsf(x0) <= 1.f && fabsf(x1) <= 1.f;
  if (!inr) x0 = x1 = 0.f;
  if (__any_sync(0xffffffffu, inr)) {
    float y[3];
    forward_warp(w, x0, x1, y);
    if (inr) {
      T = fmaf(w.norm[5], y[0], w.norm[4]);
      P = fmaf(w.norm[7], y[1], w.norm[6]);
      cs2 = fmaf(w.norm[9], y[2], w.norm[8]);
    }
  }
  if (!inr) {
    T = (e + m.a * rho) / m.cv;
    P = vdw_pressure(m, rho, T);
    cs2 = vdw_cs2(m, rho, T);
  }
  return inr;
}

// Copy an image from global memory into shared memory (all threads of the block).
__device__ __forceinline__ void load_image(const Image* __restrict__ src, Image* dst) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int k = threadIdx.x; k < int(sizeof(Image) / 16); k += blockDim.x) d[k] = s[k];
}

}  // namespace mlp
}  // namespace lbm
