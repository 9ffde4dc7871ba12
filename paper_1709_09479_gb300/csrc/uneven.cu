// Batched coding of images of different sizes in one persistent launch per ADMM iteration.
//
// The same dual ADMM sweep as geo_kernels.cuh (Eq. Inference_solution, one visit per map per
// iteration), over a batch whose images have their own H x W. Images of one size form a size class
// with its own FFT plan, twiddles, filter spectra d_hat and per-frequency system P. The N*K maps
// (image-major) are cut into G contiguous ranges of balanced pixel cost, one per CTA; a CTA meets
// each image of its range once, builds that image's lambda from the previous sweep's partial sums
// (slots of the covering CTAs in ascending order: deterministic), and streams the image's maps
// through shared memory with the run-time FFT plan of the image's class.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "csc_internal.cuh"

namespace csc {

__device__ __forceinline__ float uclamp(float v, float b) { return fminf(fmaxf(v, -b), b); }

// a complex value rounded to bfloat16 and back (operands of the mixed-precision contractions)
__device__ __forceinline__ float2 ubf16(float2 v) { return __bfloat1622float2(__floats2bfloat162_rn(v.x, v.y)); }

template <int MODE, int NT>
__global__ void __launch_bounds__(NT, 1) k_sweep_uneven(UnevenArgs a) {
  extern __shared__ float2 sm[];
  constexpr bool kLam = (MODE == kIter || MODE == kLast);
  constexpr bool kAcc = (MODE != kLast);
  const int J = a.J;
  float2* buf = sm;
  float2* lam = buf + a.buf_elems;
  float2* acc = lam + (kLam ? (size_t)J * a.max_omega : 0);
  float2* tws = acc + (kAcc ? (size_t)J * a.max_omega : 0);
  float* bf = reinterpret_cast<float*>(buf);
  const int cta = blockIdx.x;
  const long long m0 = a.mstart[cta], m1 = a.mstart[cta + 1];
  const float beta = a.beta;
  double l1 = 0.0;
  int cur_cls = -1;
  // the current size class's plan lives in shared memory: the transforms read it by reference
  __shared__ GeoRT g;
  Twiddles tw;

  for (long long n = m0 / a.K; n * a.K < m1; ++n) {
    const UImage im = a.img[n];
    if (im.cls != cur_cls) {
      __syncthreads();
      if (threadIdx.x == 0) g = a.cls[im.cls].g;
      __syncthreads();
      tw = stage_twiddles<GeoRT, NT>(g, tws, a.tw + a.cls[im.cls].tw);
      cur_cls = im.cls;
      __syncthreads();
    }
    const UClass& uc = a.cls[im.cls];
    const int W = g.W, P = g.P, Wc = g.Wc, Om = g.Omega, D = g.D;
    const int kb = (int)(max(m0, n * a.K) - n * a.K);
    const int ke = (int)(min(m1, (n + 1) * a.K) - n * a.K);
    const float2* dhat_c = a.dhat + uc.dhat;
    if (kLam) {
      const float irho = 1.0f / a.rho;
      const float2* xh = a.xhat + im.xh;
      const float* pd = a.pdiag + uc.pd;
      const float2* pmc = a.pmat + uc.pm;
      for (int o = threadIdx.x; o < Om; o += NT) {
        float2 r[kMaxJ];
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j) {
          if (j < J) {
            const float2 x = xh[(size_t)j * Om + o];
            float2 s = make_float2(-x.x * irho, -x.y * irho);
            for (int c = im.c0; c <= im.c1; ++c) s = cadd(s, a.part_in[a.slot[c + n] + (size_t)j * Om + o]);
            r[j] = s;
          }
        }
        if (J == 1) {
          lam[o] = cscale(r[0], pd[o]);
        } else {
          const float2* pm = pmc + (size_t)o * J * J;
#pragma unroll
          for (int i = 0; i < kMaxJ; ++i) {
            if (i < J) {
              float2 s = make_float2(0.f, 0.f);
#pragma unroll
              for (int j = 0; j < kMaxJ; ++j)
                if (j < J) s = cfma(pm[i * J + j], r[j], s);
              lam[(size_t)i * Om + o] = s;
            }
          }
        }
      }
    }
    if (kAcc)
      for (int i = threadIdx.x; i < J * Om; i += NT) acc[i] = make_float2(0.f, 0.f);

    for (int k = kb; k < ke; ++k) {
      const size_t moff = (size_t)im.v + (size_t)k * D;
      float* vk = a.v ? a.v + moff : nullptr;
      const float2* dk = dhat_c + (size_t)k * J * Om;
      // mixed precision: both operands of every complex product of the contractions in bfloat16
      const __nv_bfloat162* dk16 = a.dhat16 ? a.dhat16 + uc.dhat + (size_t)k * J * Om : nullptr;
      auto dval = [&](size_t i) { return dk16 ? __bfloat1622float2(dk16[i]) : __ldg(dk + i); };
      if (kLam) {
        for (int o = threadIdx.x; o < Om; o += NT) {
          float2 s = make_float2(0.f, 0.f);
#pragma unroll
          for (int j = 0; j < kMaxJ; ++j)
            if (j < J) {
              const float2 l = lam[(size_t)j * Om + o];
              s = cfmac(dval((size_t)j * Om + o), dk16 ? ubf16(l) : l, s);
            }
          const int h = o / Wc, c = o - h * Wc;
          buf[h * P + c] = s;
        }
        __syncthreads();
        irfft2<GeoRT, NT>(g, buf, tw);
        float* zk = (MODE == kLast && a.z) ? a.z + moff : nullptr;
        constexpr int U = 8;
        for (int p0 = threadIdx.x; p0 < D; p0 += NT * U) {
          float vv[U];
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (p0 + u * NT < D) vv[u] = __ldcs(vk + p0 + u * NT);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int p = p0 + u * NT;
            if (p < D) {
              const int h = p / W, x = p - h * W;
              float* cell = bf + 2 * P * h + x;
              const float vo = vv[u];
              const float vn = *cell - (uclamp(vo, beta) - vo);
              __stcs(vk + p, vn);
              const float cn = uclamp(vn, beta);
              if (MODE == kLast) {
                if (zk) __stcs(zk + p, a.rho * (cn - vn));
              } else {
                *cell = 2.f * cn - vn;
              }
            }
          }
        }
      } else {
        const float* src = (MODE == kPrologue) ? vk : a.z + moff;
        float l1f = 0.f;
        constexpr int U = 8;
        for (int p0 = threadIdx.x; p0 < D; p0 += NT * U) {
          float vv[U];
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (p0 + u * NT < D) vv[u] = __ldg(src + p0 + u * NT);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int p = p0 + u * NT;
            if (p < D) {
              const int h = p / W, x = p - h * W;
              const float t = vv[u];
              if (MODE == kPrologue) {
                bf[2 * P * h + x] = 2.f * uclamp(t, beta) - t;
              } else {
                l1f += fabsf(t);
                bf[2 * P * h + x] = t;
              }
            }
          }
        }
        l1 += (double)l1f;
      }
      if (kAcc) {
        __syncthreads();
        rfft2<GeoRT, NT>(g, buf, tw);
        for (int o = threadIdx.x; o < Om; o += NT) {
          const int h = o / Wc, c = o - h * Wc;
          const float2 uh = dk16 ? ubf16(buf[h * P + c]) : buf[h * P + c];
#pragma unroll
          for (int j = 0; j < kMaxJ; ++j)
            if (j < J) acc[(size_t)j * Om + o] = cfma(dval((size_t)j * Om + o), uh, acc[(size_t)j * Om + o]);
        }
      }
      __syncthreads();
    }
    if (kAcc) {
      float2* dst = a.part_out + a.slot[cta + n];
      for (int i = threadIdx.x; i < J * Om; i += NT) dst[i] = acc[i];
    }
  }
  if (MODE == kObjective) {
    __shared__ double red[NT / 32];
    for (int off = 16; off > 0; off >>= 1) l1 += __shfl_down_sync(0xffffffffu, l1, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l1;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < NT / 32; ++i) s += red[i];
      a.l1[cta] = s;
    }
  }
}

// per image: (1/D) sum_w weight(w) |sum of its slots - x_hat|^2 (Parseval on the half spectrum)
__global__ void k_objective_final_uneven(UnevenArgs a, double* out) {
  const int n = blockIdx.x;
  const UImage im = a.img[n];
  const UClass& uc = a.cls[im.cls];
  const int Om = uc.g.Omega, Wc = uc.g.Wc, W = uc.g.W;
  double s = 0.0;
  for (int j = 0; j < a.J; ++j) {
    const float2* xh = a.xhat + im.xh + (size_t)j * Om;
    for (int o = threadIdx.x; o < Om; o += blockDim.x) {
      float2 r = make_float2(-xh[o].x, -xh[o].y);
      for (int c = im.c0; c <= im.c1; ++c) r = cadd(r, a.part_in[a.slot[c + n] + (size_t)j * Om + o]);
      const int col = o % Wc;
      const float wgt = (col == 0 || (2 * col == W)) ? 1.f : 2.f;
      s += (double)(wgt * (r.x * r.x + r.y * r.y));
    }
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    out[n] = t / (double)uc.g.D;
  }
}

size_t uneven_smem_bytes(const UnevenLayout& L, int J, int mode) {
  const bool lam = (mode == kIter || mode == kLast);
  const bool acc = (mode != kLast);
  return ((size_t)L.buf_elems + (lam ? (size_t)J * L.max_omega : 0) + (acc ? (size_t)J * L.max_omega : 0) +
          (size_t)L.max_tw) * sizeof(float2);
}

template <int MODE, int NT>
static cudaError_t launch_uneven_mode(const UnevenArgs& a, int G, size_t smem, cudaStream_t st) {
  auto kern = k_sweep_uneven<MODE, NT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<G, NT, smem, st>>>(a);
  return cudaGetLastError();
}

template <int NT>
static cudaError_t launch_uneven_nt(int mode, const UnevenArgs& a, int G, size_t smem, cudaStream_t st) {
  switch (mode) {
    case kPrologue: return launch_uneven_mode<kPrologue, NT>(a, G, smem, st);
    case kIter: return launch_uneven_mode<kIter, NT>(a, G, smem, st);
    case kLast: return launch_uneven_mode<kLast, NT>(a, G, smem, st);
    default: return launch_uneven_mode<kObjective, NT>(a, G, smem, st);
  }
}

cudaError_t launch_sweep_uneven(const UnevenArgs& a, int mode, int G, int nt, size_t smem, cudaStream_t st) {
  return nt == 256 ? launch_uneven_nt<256>(mode, a, G, smem, st) : launch_uneven_nt<512>(mode, a, G, smem, st);
}

cudaError_t launch_objective_final_uneven(const UnevenArgs& a, double* out, cudaStream_t st) {
  k_objective_final_uneven<<<a.N, 512, 0, st>>>(a, out);
  return cudaGetLastError();
}

}  // namespace csc
