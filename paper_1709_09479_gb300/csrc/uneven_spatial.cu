// Direct spatial coding of an uneven batch (CSC_FLAG_SPATIAL on csc_init_uneven, grey images).
//
// The coding iteration of Eq. Inference_solution with the two filter products taken on the pixel
// grid of each H x W image (circular boundaries, as the DFT has them):
//   r   = sum_k d_k * u_k               (u_k = 2 clamp(v_k) - v_k; the product d_hat_k u_hat_k)
//   lam = F^-1(P F(r - x / rho))        (one channel per image: the engine's transforms)
//   w_k = d_k (correlated with) lam     (the product conj(d_hat_k) lam_hat)
//   v_k <- w_k - (clamp(v_k) - v_k)     (and, after the last iteration, z_k = rho (clamp(v_k) - v_k))
// so that only one 2-D transform pair per image and iteration is left of the K pairs the Fourier
// route takes. Both products are written as one correlation,
//   out(y, x) = sum_{a, b < F} g(a, b) in(y + a - c, x + b - c),   c = (F - 1) / 2,
// with every filter zero-padded to F x F = 11 x 11 about its centre (tap (ta, tb) of an fh x fw
// filter at (ta + c - (fh-1)/2, tb + c - (fw-1)/2)): g = the padded d_k for D^T, and the padded d_k
// flipped in both axes for D.
//
// Work item: one output tile of 32 rows x 64 columns of one image. 128 threads, each 4 rows x 4
// columns of outputs; the F x F taps of the current filter in registers; the input tile with its
// circular halo ((32 + F - 1) x (64 + F - 1) values) in shared memory, each thread reading its
// 4 + F - 1 input rows once (four 16-byte loads each) and using every row for all the output rows
// it reaches. D loops over the filters with the tile of u_k reloaded per filter and one accumulator
// per output; D^T loads the tile of lam once and runs the state update of each filter's outputs.
// Every sum runs in a fixed order: results are deterministic.
#include <cuda_runtime.h>

#include <algorithm>

#include "csc_internal.cuh"

namespace csc {
namespace usp {

constexpr int F = kUspF, C = (F - 1) / 2;
constexpr int TH = kUspTileH, TW = kUspTileW;
constexpr int NT = 128;                  // 16 x 8 threads, 4 x 4 outputs each
constexpr int IH = TH + F - 1;           // input tile rows
constexpr int IW = TW + F - 1;           // input tile columns
constexpr int IP = (IW + 3) / 4 * 4;     // input tile pitch (16-byte rows)
constexpr int GS = (F * F + 3) / 4 * 4;  // floats per padded filter in shared memory (16-byte aligned)
static_assert(4 + F - 1 <= 16, "a thread's input row segment is four 16-byte loads");
static_assert(IP >= 4 * 15 + 16, "the last thread's four loads stay inside the row");

__device__ __forceinline__ float uclamp(float v, float b) { return fminf(fmaxf(v, -b), b); }

// shared memory: padded filters [K][GS] | input tile [IH][IP] | halo row offsets [IH] | columns [IW]
// | the in-plane offset of every tile element [IH][IP] (0 for the pad columns IW..IP-1)
struct Smem {
  float* g;
  float* tile;
  long long* roff;
  int* cidx;
  int* gofs;
};
__device__ __forceinline__ Smem carve(float* sm, int K) {
  Smem s;
  s.g = sm;
  s.tile = sm + (size_t)K * GS;
  s.roff = reinterpret_cast<long long*>(s.tile + IH * IP);
  s.cidx = reinterpret_cast<int*>(s.roff + IH);
  s.gofs = s.cidx + IW;
  return s;
}

// the K filters padded to F x F (flipped for D), and the tile's circular halo indices
template <bool FLIP>
__device__ __forceinline__ void stage_filters_and_halo(const UspArgs& a, const Smem& s, int H, int W, int y0, int x0) {
  const int oh = C - (a.fh - 1) / 2, ow = C - (a.fw - 1) / 2;
  for (int i = threadIdx.x; i < a.K * GS; i += NT) {
    const int k = i / GS, t = i - k * GS;
    float val = 0.f;
    if (t < F * F) {
      int pa = t / F, pb = t - (t / F) * F;
      if (FLIP) { pa = F - 1 - pa; pb = F - 1 - pb; }
      const int ta = pa - oh, tb = pb - ow;
      if (ta >= 0 && ta < a.fh && tb >= 0 && tb < a.fw) val = a.d[((size_t)k * a.fh + ta) * a.fw + tb];
    }
    s.g[i] = val;
  }
  for (int i = threadIdx.x; i < IH; i += NT) s.roff[i] = (long long)((((y0 - C + i) % H) + H) % H) * W;
  for (int i = threadIdx.x; i < IW; i += NT) s.cidx[i] = (((x0 - C + i) % W) + W) % W;
}

// acc[i][c] += sum_{a, b} g(a, b) tile[4 ty + i + a][4 tx + c + b]
__device__ __forceinline__ void correlate(const float* __restrict__ tile, const float* __restrict__ gk, int ty, int tx,
                                          float (&acc)[4][4]) {
  float g[GS];
  const float4* g4 = reinterpret_cast<const float4*>(gk);
#pragma unroll
  for (int q = 0; q < GS / 4; ++q) {
    const float4 t = g4[q];
    g[4 * q] = t.x; g[4 * q + 1] = t.y; g[4 * q + 2] = t.z; g[4 * q + 3] = t.w;
  }
  // the taps stay in registers for the whole filter (not re-read from shared memory at each use)
#pragma unroll
  for (int t = 0; t < F * F; ++t) asm volatile("" : "+f"(g[t]));
#pragma unroll
  for (int r = 0; r < 4 + F - 1; ++r) {
    const float4* row = reinterpret_cast<const float4*>(tile + (4 * ty + r) * IP + 4 * tx);
    float in[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 t = row[q];
      in[4 * q] = t.x; in[4 * q + 1] = t.y; in[4 * q + 2] = t.z; in[4 * q + 3] = t.w;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ra = r - i;   // the filter row that input row r meets in output row i
      if (ra >= 0 && ra < F) {
#pragma unroll
        for (int b = 0; b < F; ++b)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(g[ra * F + b], in[c + b], acc[i][c]);
      }
    }
  }
}

// q = sum_k d_k * u_k - x / rho on one tile. The tile of v_{k+1} is loaded into registers while
// filter k's products run, and stored as u_{k+1} once every thread has finished reading tile k.
// Elements are taken in the tile's own order (pitch IP), their in-plane offsets from the table
// built once per tile (a plane is at most 1024 x 1024: int offsets).
constexpr int NPRE = (IH * IP + NT - 1) / NT;   // tile elements per thread
__global__ void __launch_bounds__(NT, 2) k_usp_conv(UspArgs a) {
  extern __shared__ __align__(16) float sm[];
  const UspTile tl = a.tiles[blockIdx.x];
  const BigImg im = a.img[tl.img];
  const int H = a.cls[im.cls].H, W = a.cls[im.cls].W;
  const Smem s = carve(sm, a.K);
  stage_filters_and_halo<true>(a, s, H, W, tl.y0, tl.x0);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const float beta = a.beta;
  float acc[4][4] = {};
  const size_t plane = (size_t)H * W;
  __syncthreads();   // the halo tables
  for (int i = threadIdx.x; i < IH * IP; i += NT) {
    const int r = i / IP, c = i - r * IP;
    s.gofs[i] = c < IW ? (int)(s.roff[r] + s.cidx[c]) : 0;
  }
  __syncthreads();
  float pre[NPRE];
  auto fetch = [&](int k) {
    const float* vk = a.v + im.v + (size_t)k * plane;
#pragma unroll
    for (int j = 0; j < NPRE; ++j) {
      const int i = threadIdx.x + j * NT;
      if (i < IH * IP) pre[j] = __ldg(vk + s.gofs[i]);
    }
  };
  fetch(0);
  for (int k = 0; k < a.K; ++k) {
    if (k > 0) __syncthreads();   // every thread's reads of tile k - 1
#pragma unroll
    for (int j = 0; j < NPRE; ++j) {
      const int i = threadIdx.x + j * NT;
      if (i < IH * IP) s.tile[i] = 2.f * uclamp(pre[j], beta) - pre[j];
    }
    __syncthreads();
    if (k + 1 < a.K) fetch(k + 1);
    correlate(s.tile, s.g + (size_t)k * GS, ty, tx, acc);
  }
  const float irho = 1.0f / a.rho;
  const float* xi = a.x + im.x;
  float* qi = a.q + im.x;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int y = tl.y0 + 4 * ty + i;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int x = tl.x0 + 4 * tx + c;
      if (y < H && x < W) qi[(size_t)y * W + x] = acc[i][c] - xi[(size_t)y * W + x] * irho;
    }
  }
}

// w_k = d_k (correlated with) lambda, the state update, and (last) the codes, on one tile
template <bool LAST>
__global__ void __launch_bounds__(NT, 2) k_usp_corr(UspArgs a) {
  extern __shared__ __align__(16) float sm[];
  const UspTile tl = a.tiles[blockIdx.x];
  const BigImg im = a.img[tl.img];
  const int H = a.cls[im.cls].H, W = a.cls[im.cls].W;
  const Smem s = carve(sm, a.K);
  stage_filters_and_halo<false>(a, s, H, W, tl.y0, tl.x0);
  __syncthreads();
  const float* lam = a.q + im.x;
  for (int i = threadIdx.x; i < IH * IW; i += NT) {
    const int r = i / IW, c = i - r * IW;
    s.tile[r * IP + c] = lam[s.roff[r] + s.cidx[c]];
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const float beta = a.beta, rho = a.rho;
  const size_t plane = (size_t)H * W;
  // this thread's outputs: in-image flags and offsets within a plane
  bool in[4][4];
  size_t off[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int y = tl.y0 + 4 * ty + i, x = tl.x0 + 4 * tx + c;
      in[i][c] = (y < H && x < W);
      off[i][c] = in[i][c] ? (size_t)y * W + x : 0;
    }
  for (int k = 0; k < a.K; ++k) {
    float* vk = a.v + im.v + (size_t)k * plane;
    float vo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) vo[i][c] = in[i][c] ? vk[off[i][c]] : 0.f;
    float acc[4][4] = {};
    correlate(s.tile, s.g + (size_t)k * GS, ty, tx, acc);
    float* zk = (LAST && a.z) ? a.z + im.v + (size_t)k * plane : nullptr;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (!in[i][c]) continue;
        const float v = vo[i][c];
        const float vn = acc[i][c] - (uclamp(v, beta) - v);
        vk[off[i][c]] = vn;
        if (zk) zk[off[i][c]] = rho * (uclamp(vn, beta) - vn);
      }
  }
}

}  // namespace usp

size_t usp_smem_bytes(int K) {
  using namespace usp;
  return ((size_t)K * GS + (size_t)IH * IP) * sizeof(float) + (size_t)IH * sizeof(long long) +
         (size_t)(IW + IH * IP) * sizeof(int);
}

cudaError_t launch_usp_conv(const UspArgs& a, cudaStream_t st) {
  const size_t smem = usp_smem_bytes(a.K);
  cudaError_t e = cudaFuncSetAttribute(usp::k_usp_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  usp::k_usp_conv<<<a.n_tiles, usp::NT, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_usp_corr(const UspArgs& a, bool last, cudaStream_t st) {
  const size_t smem = usp_smem_bytes(a.K);
  auto kern = last ? usp::k_usp_corr<true> : usp::k_usp_corr<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<a.n_tiles, usp::NT, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace csc
