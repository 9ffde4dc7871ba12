// Per-map kernels (one CTA transforms one H x W map in shared memory), templated on the image
// geometry. Each geo_*.cu translation unit instantiates them for one geometry and exports the
// launchers through a GeoOps table, so the fixed sizes compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "csc_internal.cuh"

namespace csc {

__device__ __forceinline__ float clampb(float v, float b) { return fminf(fmaxf(v, -b), b); }

// a complex value rounded to bfloat16 and back (operands of the mixed-precision contractions)
__device__ __forceinline__ float2 round_bf16(float2 v) {
  return __bfloat1622float2(__floats2bfloat162_rn(v.x, v.y));
}

// bulk prefetch of a global range into L2 (address and size multiples of 16 bytes)
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------------------------
// batched forward transforms of real maps or of filters placed on the grid
// ---------------------------------------------------------------------------------------------
struct FftMapsArgs {
  const float* in;
  int nmaps;
  int filter_mode;   // 0: maps [m][H][W]; 1: filters [m][fh][fw] centred on the grid
  int fh, fw;
  float2* out;       // [m][Omega]
  const float2* tw;
};

template <class G, int NT>
__global__ void __launch_bounds__(NT) k_fft_maps(FftMapsArgs a, G g) {
  extern __shared__ float2 sm[];
  const int H = g.h(), W = g.w(), P = g.p(), Wc = g.wc(), Om = g.omega();
  float2* buf = sm;
  Twiddles tw = stage_twiddles<G, NT>(g, buf + H * P, a.tw);
  float* bf = reinterpret_cast<float*>(buf);
  for (int m = blockIdx.x; m < a.nmaps; m += gridDim.x) {
    __syncthreads();
    if (a.filter_mode) {
      for (int i = threadIdx.x; i < H * P; i += NT) buf[i] = make_float2(0.f, 0.f);
      __syncthreads();
      const int ch = (a.fh - 1) / 2, cw = (a.fw - 1) / 2;
      const float* f = a.in + (size_t)m * a.fh * a.fw;
      for (int t = threadIdx.x; t < a.fh * a.fw; t += NT) {
        const int ta = t / a.fw, tb = t - ta * a.fw;
        const int h = ((ta - ch) % H + H) % H, w = ((tb - cw) % W + W) % W;
        bf[2 * P * h + w] = f[t];
      }
    } else {
      const float* src = a.in + (size_t)m * H * W;
      for (int p = threadIdx.x; p < H * W; p += NT) {
        const int h = p / W, w = p - h * W;
        bf[2 * P * h + w] = src[p];
      }
    }
    __syncthreads();
    rfft2<G, NT>(g, buf, tw);
    float2* dst = a.out + (size_t)m * Om;
    for (int o = threadIdx.x; o < Om; o += NT) {
      const int h = o / Wc, c = o - h * Wc;
      dst[o] = buf[h * P + c];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// the fused coding sweep
// ---------------------------------------------------------------------------------------------
template <class G, int MODE, int NT>
__global__ void __launch_bounds__(NT, 1) k_sweep(SweepArgs a, G g) {
  extern __shared__ float2 sm[];
  constexpr bool kLam = (MODE == kIter || MODE == kLast);
  constexpr bool kAcc = (MODE != kLast);
  const int H = g.h(), W = g.w(), P = g.p(), Wc = g.wc(), Om = g.omega(), D = g.d();
  const int J = a.J;
  float2* buf = sm;
  float2* lam = buf + H * P;
  float2* acc = lam + (kLam ? J * Om : 0);
  float2* tws = acc + (kAcc ? J * Om : 0);
  const Twiddles tw = stage_twiddles<G, NT>(g, tws, a.tw);
  float* bf = reinterpret_cast<float*>(buf);
  __syncthreads();

  const long long NK = (long long)a.N * a.K;
  const int cta = blockIdx.x;
  const long long m0 = (long long)cta * NK / a.G, m1 = (long long)(cta + 1) * NK / a.G;
  const float beta = a.beta;
  double l1 = 0.0;

  for (long long n = m0 / a.K; n * a.K < m1; ++n) {
    const int kb = (int)(max(m0, n * a.K) - n * a.K);
    const int ke = (int)(min(m1, (n + 1) * a.K) - n * a.K);
    if (kLam) {
      // lambda_hat / D for image n from the previous sweep's partial sums (slot = cta' + n)
      const int c0 = (int)(((n * a.K + 1) * a.G - 1) / NK);
      const int c1 = (int)((((n + 1) * a.K) * a.G - 1) / NK);
      const float irho = 1.0f / a.rho;
      const float2* xh = a.xhat + (size_t)n * J * Om;
      bool bad = false;
      for (int o = threadIdx.x; o < Om; o += NT) {
        float2 r[kMaxJ];
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j) {
          if (j < J) {
            const float2 x = xh[(size_t)j * Om + o];
            r[j] = sum_slots_at(a.part_in + ((size_t)n * J + j) * Om + o, (size_t)J * Om, c0, c1,
                                make_float2(-x.x * irho, -x.y * irho));
          }
        }
        float2* ls = (a.lam_store && cta == c0) ? a.lam_store + (size_t)n * J * Om : nullptr;
        if (J == 1) {
          lam[o] = cscale(r[0], a.pdiag[o]);
          bad |= !(isfinite(lam[o].x) && isfinite(lam[o].y));
          if (ls) ls[o] = lam[o];
        } else {
          const float2* pm = a.pmat + (size_t)o * J * J;
#pragma unroll
          for (int i = 0; i < kMaxJ; ++i) {
            if (i < J) {
              float2 s = make_float2(0.f, 0.f);
#pragma unroll
              for (int j = 0; j < kMaxJ; ++j)
                if (j < J) s = cfma(pm[i * J + j], r[j], s);
              lam[(size_t)i * Om + o] = s;
              bad |= !(isfinite(s.x) && isfinite(s.y));
              if (ls) ls[(size_t)i * Om + o] = s;
            }
          }
        }
      }
      if (bad && a.err) atomicExch(a.err, (int)CSC_ERR_NONFINITE);
    }
    if (kAcc)
      for (int i = threadIdx.x; i < J * Om; i += NT) acc[i] = make_float2(0.f, 0.f);

    for (int k = kb; k < ke; ++k) {
      const size_t map = (size_t)n * a.K + k;
      float* vk = a.v ? a.v + map * D : nullptr;
      float* vw = a.v_out ? a.v_out + map * D : vk;   // where the new state goes
      const float2* dk = a.dhat + (size_t)k * J * Om;
      const __nv_bfloat162* dk16 = a.dhat16 ? a.dhat16 + (size_t)k * J * Om : nullptr;
      const bool tf = a.tf32 != 0;   // TF32 contraction operands
      // pull the next map's state (or codes) into L2 while this one is transformed
      if (a.vec4 && threadIdx.x < 4 && (long long)map + 1 < m1) {
        const float* nxt = (MODE == kObjective) ? a.z + (map + 1) * D : a.v + (map + 1) * D;
        prefetch_l2(nxt + threadIdx.x * (D / 4), (unsigned)D);
      }
      if (kLam) {
        // w_hat_k = sum_j conj(d_hat_jk) lam_j
        for (int o0 = threadIdx.x; o0 < Om; o0 += NT * 4) {
          float2 dv[4][kMaxJ];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int o = o0 + u * NT;
            if (o < Om)
#pragma unroll
              for (int j = 0; j < kMaxJ; ++j)
                if (j < J) dv[u][j] = dk16 ? __bfloat1622float2(dk16[(size_t)j * Om + o])
                                 : (tf ? tf32r2(__ldg(dk + (size_t)j * Om + o)) : __ldg(dk + (size_t)j * Om + o));
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int o = o0 + u * NT;
            if (o < Om) {
              float2 s = make_float2(0.f, 0.f);
#pragma unroll
              for (int j = 0; j < kMaxJ; ++j)
                if (j < J) {
                  const float2 l = lam[(size_t)j * Om + o];
                  s = cfmac(dv[u][j], dk16 ? round_bf16(l) : (tf ? tf32r2(l) : l), s);
                }
              const int h = o / Wc, c = o - h * Wc;
              buf[h * P + c] = s;
            }
          }
        }
        __syncthreads();
        irfft2<G, NT>(g, buf, tw);
        float* zk = (MODE == kLast && a.z) ? a.z + map * D : nullptr;
        if (a.vec4) {
          // 4 pixels per thread and step, all loads of a thread issued before any use
          constexpr int U = 8;
          const int n4 = D / 4;
          float4* v4 = reinterpret_cast<float4*>(vk);
          float4* vw4 = reinterpret_cast<float4*>(vw);
          float4* z4 = reinterpret_cast<float4*>(zk);
          for (int q0 = threadIdx.x; q0 < n4; q0 += NT * U) {
            float4 vv[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
              if (q0 + u * NT < n4) vv[u] = __ldcs(v4 + q0 + u * NT);
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int q = q0 + u * NT;
              if (q < n4) {
                const int p = 4 * q, h = p / W, x = p - h * W;
                float2* cell = reinterpret_cast<float2*>(bf + 2 * P * h + x);
                const float2 w01 = cell[0], w23 = cell[1];
                float4 vn;
                vn.x = w01.x - (clampb(vv[u].x, beta) - vv[u].x);
                vn.y = w01.y - (clampb(vv[u].y, beta) - vv[u].y);
                vn.z = w23.x - (clampb(vv[u].z, beta) - vv[u].z);
                vn.w = w23.y - (clampb(vv[u].w, beta) - vv[u].w);
                __stcs(vw4 + q, vn);
                if (MODE == kLast) {
                  if (zk) {
                    float4 zz;
                    zz.x = a.rho * (clampb(vn.x, beta) - vn.x);
                    zz.y = a.rho * (clampb(vn.y, beta) - vn.y);
                    zz.z = a.rho * (clampb(vn.z, beta) - vn.z);
                    zz.w = a.rho * (clampb(vn.w, beta) - vn.w);
                    __stcs(z4 + q, zz);
                  }
                } else {
                  cell[0] = make_float2(2.f * clampb(vn.x, beta) - vn.x, 2.f * clampb(vn.y, beta) - vn.y);
                  cell[1] = make_float2(2.f * clampb(vn.z, beta) - vn.z, 2.f * clampb(vn.w, beta) - vn.w);
                }
              }
            }
          }
        } else {
          for (int p = threadIdx.x; p < D; p += NT) {
            const int h = p / W, x = p - h * W;
            float* cell = bf + 2 * P * h + x;
            const float vo = vk[p];
            const float vn = *cell - (clampb(vo, beta) - vo);
            vw[p] = vn;
            const float cn = clampb(vn, beta);
            if (MODE == kLast) {
              if (zk) zk[p] = a.rho * (cn - vn);
            } else {
              *cell = 2.f * cn - vn;
            }
          }
        }
      } else {
        // prologue: u = 2 clamp(v) - v of the given state; objective: the codes themselves
        // (|z| summed in float32 per map, float64 across maps: the float64 rate is low)
        const float* src = (MODE == kPrologue) ? vk : a.z + map * D;
        float l1f = 0.f;
        if (a.vec4) {
          constexpr int U = 8;
          const int n4 = D / 4;
          const float4* s4 = reinterpret_cast<const float4*>(src);
          for (int q0 = threadIdx.x; q0 < n4; q0 += NT * U) {
            float4 vv[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
              if (q0 + u * NT < n4) vv[u] = __ldg(s4 + q0 + u * NT);
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int q = q0 + u * NT;
              if (q < n4) {
                const int p = 4 * q, h = p / W, x = p - h * W;
                float2* cell = reinterpret_cast<float2*>(bf + 2 * P * h + x);
                const float4 t = vv[u];
                if (MODE == kPrologue) {
                  cell[0] = make_float2(2.f * clampb(t.x, beta) - t.x, 2.f * clampb(t.y, beta) - t.y);
                  cell[1] = make_float2(2.f * clampb(t.z, beta) - t.z, 2.f * clampb(t.w, beta) - t.w);
                } else {
                  l1f += (fabsf(t.x) + fabsf(t.y)) + (fabsf(t.z) + fabsf(t.w));
                  cell[0] = make_float2(t.x, t.y);
                  cell[1] = make_float2(t.z, t.w);
                }
              }
            }
          }
        } else {
          for (int p = threadIdx.x; p < D; p += NT) {
            const int h = p / W, x = p - h * W;
            const float t = src[p];
            if (MODE == kPrologue) {
              bf[2 * P * h + x] = 2.f * clampb(t, beta) - t;
            } else {
              l1f += fabsf(t);
              bf[2 * P * h + x] = t;
            }
          }
        }
        l1 += (double)l1f;
      }
      if (kAcc) {
        __syncthreads();
        rfft2<G, NT>(g, buf, tw);
        for (int o0 = threadIdx.x; o0 < Om; o0 += NT * 4) {
          float2 dv[4][kMaxJ];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int o = o0 + u * NT;
            if (o < Om)
#pragma unroll
              for (int j = 0; j < kMaxJ; ++j)
                if (j < J) dv[u][j] = dk16 ? __bfloat1622float2(dk16[(size_t)j * Om + o])
                                 : (tf ? tf32r2(__ldg(dk + (size_t)j * Om + o)) : __ldg(dk + (size_t)j * Om + o));
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int o = o0 + u * NT;
            if (o < Om) {
              const int h = o / Wc, c = o - h * Wc;
              const float2 uh = dk16 ? round_bf16(buf[h * P + c]) : (tf ? tf32r2(buf[h * P + c]) : buf[h * P + c]);
#pragma unroll
              for (int j = 0; j < kMaxJ; ++j)
                if (j < J) acc[(size_t)j * Om + o] = cfma(dv[u][j], uh, acc[(size_t)j * Om + o]);
            }
          }
        }
      }
      __syncthreads();
    }
    if (kAcc) {
      float2* dst = a.part_out + (size_t)(cta + n) * J * Om;
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

// ---------------------------------------------------------------------------------------------
// b_kj = S F^{-1}( sum_n conj(z_hat_nk) x_hat_nj ) / D: one CTA per (k, j)
// ---------------------------------------------------------------------------------------------
struct RhsArgs {
  int N, K, J, fh, fw;
  const float2* zhat;  // [N][K][Omega]
  const float2* xhat;  // [N][J][Omega]
  float* b;            // [K][J][fh*fw]
  const float2* tw;
  const float2* spec;  // [K][J][Omega] precomputed sum_n conj(z_hat_nk) x_hat_nj, or null
};

template <class G, int NT>
__device__ __forceinline__ void crop_window(const G& g, const float* bf, int wa, int wb, int ca, int cb,
                                            float scale, float* out) {
  const int H = g.h(), W = g.w(), P = g.p();
  for (int t = threadIdx.x; t < wa * wb; t += NT) {
    const int ta = t / wb, tb = t - ta * wb;
    const int h = ((ta - ca) % H + H) % H, w = ((tb - cb) % W + W) % W;
    out[t] = bf[2 * P * h + w] * scale;
  }
}

template <class G, int NT>
__global__ void __launch_bounds__(NT) k_learn_rhs(RhsArgs a, G g) {
  extern __shared__ float2 sm[];
  const int H = g.h(), P = g.p(), Wc = g.wc(), Om = g.omega();
  float2* buf = sm;
  const Twiddles tw = stage_twiddles<G, NT>(g, buf + H * P, a.tw);
  const int k = blockIdx.x / a.J, j = blockIdx.x % a.J;
  for (int o = threadIdx.x; o < Om; o += NT) {
    float2 s = make_float2(0.f, 0.f);
    if (a.spec) s = a.spec[((size_t)k * a.J + j) * Om + o];
    else
      for (int n = 0; n < a.N; ++n)
        s = cfmac(a.zhat[((size_t)n * a.K + k) * Om + o], a.xhat[((size_t)n * a.J + j) * Om + o], s);
    const int h = o / Wc, c = o - h * Wc;
    buf[h * P + c] = s;
  }
  __syncthreads();
  irfft2<G, NT>(g, buf, tw);
  crop_window<G, NT>(g, reinterpret_cast<const float*>(buf), a.fh, a.fw, (a.fh - 1) / 2, (a.fw - 1) / 2,
                     1.0f / (float)g.d(), a.b + ((size_t)k * a.J + j) * a.fh * a.fw);
}

// ---------------------------------------------------------------------------------------------
// lags C_kk'(tau), tau in [-(fh-1), fh-1] x [-(fw-1), fw-1], one CTA per pair k <= k'
// ---------------------------------------------------------------------------------------------
struct LagsArgs {
  int K, fh, fw;
  const float2* gram;
  float* lags;   // [K][K][La][Lb]
  const float2* tw;
};

template <class G, int NT>
__global__ void __launch_bounds__(NT) k_learn_lags(LagsArgs a, G g) {
  extern __shared__ float2 sm[];
  const int H = g.h(), W = g.w(), P = g.p(), Wc = g.wc(), Om = g.omega();
  float2* buf = sm;
  const Twiddles tw = stage_twiddles<G, NT>(g, buf + H * P, a.tw);
  // pair index -> (k, k')
  int k = 0;
  long long rem = blockIdx.x;
  while (rem >= a.K - k) { rem -= a.K - k; ++k; }
  const int kp = k + (int)rem;
  const float2* src = a.gram + (size_t)blockIdx.x * Om;
  for (int o = threadIdx.x; o < Om; o += NT) {
    const int h = o / Wc, c = o - h * Wc;
    buf[h * P + c] = src[o];
  }
  __syncthreads();
  irfft2<G, NT>(g, buf, tw);
  const float* bf = reinterpret_cast<const float*>(buf);
  const int La = 2 * a.fh - 1, Lb = 2 * a.fw - 1;
  const float scale = 1.0f / (float)g.d();
  float* out = a.lags + ((size_t)k * a.K + kp) * La * Lb;
  float* outT = a.lags + ((size_t)kp * a.K + k) * La * Lb;
  for (int t = threadIdx.x; t < La * Lb; t += NT) {
    const int ta = t / Lb, tb = t - ta * Lb;
    const int h = ((ta - (a.fh - 1)) % H + H) % H, w = ((tb - (a.fw - 1)) % W + W) % W;
    const float val = bf[2 * P * h + w] * scale;
    if (k == kp) {
      // autocorrelation: C_kk(tau) = C_kk(-tau); store the symmetrised value so the matrix of the
      // normal equations is exactly symmetric (one writer per entry)
      const int hm = ((-(ta - (a.fh - 1))) % H + H) % H, wm = ((-(tb - (a.fw - 1))) % W + W) % W;
      out[t] = 0.5f * (val + bf[2 * P * hm + wm] * scale);
    } else {
      out[t] = val;
      outT[(La - 1 - ta) * Lb + (Lb - 1 - tb)] = val;   // C_k'k(tau) = C_kk'(-tau)
    }
  }
}


// ---------------------------------------------------------------------------------------------
// reverse mode through unrolled coding iterations (J = 1). With lam_s = lambda_hat / D stored by the
// forward sweeps, one reverse step t (incoming vbar = dL/dv^{t+1}) is, per image and map:
//   rbar_s = P/D * sum_k d_hat_k F(vbar_k)         (from the previous reverse sweep's partial sums)
//   ubar_k = F^{-1}( conj(d_hat_k) rbar_s )
//   vbar_k <- (1 - m) vbar_k + (2m - 1) ubar_k,     m = 1[|v^t_k| < beta]
//   G_nk  += conj(F u^t_k) rbar_s + conj(F vbar^t_k) lam_s^{t-1}      (filter-gradient spectra)
//   S_n   += D * 2 Re(conj(lam_s^t) rbar_s),  Xb_n -= rbar_s / rho       (once per image)
// and the partial sums d_hat_k F(vbar^t_k) feed the next reverse step. The seed sweep sets
// vbar^T = rho (m_T - 1) z_bar and G_nk = conj(F vbar^T_k) lam_s^{T-1}.
// ---------------------------------------------------------------------------------------------
template <class G, int MODE, int NT>
__global__ void __launch_bounds__(NT, 1) k_bwd_sweep(BwdArgs a, G g) {
  extern __shared__ float2 sm[];
  constexpr bool kR = (MODE != kBSeed);    // needs rbar_s
  constexpr bool kAcc = (MODE != kBLast);  // produces partial sums for the next reverse step
  const int H = g.h(), W = g.w(), P = g.p(), Wc = g.wc(), Om = g.omega(), D = g.d();
  float2* buf = sm;
  float2* rb = buf + H * P;
  float2* acc = rb + (kR ? Om : 0);
  float2* tws = acc + (kAcc ? Om : 0);
  const Twiddles tw = stage_twiddles<G, NT>(g, tws, a.tw);
  float* bf = reinterpret_cast<float*>(buf);
  __syncthreads();
  const long long NK = (long long)a.N * a.K;
  const int cta = blockIdx.x;
  const long long m0 = (long long)cta * NK / a.G, m1 = (long long)(cta + 1) * NK / a.G;
  const float beta = a.beta;
  for (long long n = m0 / a.K; n * a.K < m1; ++n) {
    const int kb = (int)(max(m0, n * a.K) - n * a.K);
    const int ke = (int)(min(m1, (n + 1) * a.K) - n * a.K);
    const int c0 = (int)(((n * a.K + 1) * a.G - 1) / NK);
    const int c1 = (int)((((n + 1) * a.K) * a.G - 1) / NK);
    if (kR) {
      const bool owner = (cta == c0);
      for (int o = threadIdx.x; o < Om; o += NT) {
        float2 s = make_float2(0.f, 0.f);
        for (int c = c0; c <= c1; ++c) s = cadd(s, a.part_in[(size_t)(c + n) * Om + o]);
        const float2 r = cscale(s, a.pdiag[o]);
        rb[o] = r;
        if (owner) {
          const float2 l = a.lam_t[(size_t)n * Om + o];
          a.S[(size_t)n * Om + o] += a.dsize * 2.f * (l.x * r.x + l.y * r.y);
          float2 xb = a.Xb[(size_t)n * Om + o];
          xb.x -= r.x / a.rho;
          xb.y -= r.y / a.rho;
          a.Xb[(size_t)n * Om + o] = xb;
        }
      }
    }
    if (kAcc)
      for (int o = threadIdx.x; o < Om; o += NT) acc[o] = make_float2(0.f, 0.f);
    const float2* lp = (MODE != kBLast) ? a.lam_prev + (size_t)n * Om : nullptr;
    for (int k = kb; k < ke; ++k) {
      const size_t map = (size_t)n * a.K + k;
      const float2* dk = a.dhat + (size_t)k * Om;
      float* vb = a.vbar + map * D;
      const float* vtk = a.vt + map * D;
      float2* gk = a.gspec + map * Om;
      if (MODE == kBSeed) {
        const float* gzk = a.gz + map * D;
        for (int p = threadIdx.x; p < D; p += NT) {
          const int h = p / W, x = p - h * W;
          const float v = vtk[p];
          const float m = (fabsf(v) < beta) ? 1.f : 0.f;
          const float b = a.rho * (m - 1.f) * gzk[p];
          vb[p] = b;
          bf[2 * P * h + x] = b;
        }
      } else {
        if (MODE == kBIter) {
          // ubar_k = F^{-1}(conj(d_hat_k) rbar_s)
          for (int o = threadIdx.x; o < Om; o += NT) {
            const int h = o / Wc, c = o - h * Wc;
            buf[h * P + c] = cfmac(__ldg(dk + o), rb[o], make_float2(0.f, 0.f));
          }
          __syncthreads();
          irfft2<G, NT>(g, buf, tw);
          // vbar update in HBM; then u^t into the buffer
          for (int p = threadIdx.x; p < D; p += NT) {
            const int h = p / W, x = p - h * W;
            float* cell = bf + 2 * P * h + x;
            const float v = vtk[p];
            const float m = (fabsf(v) < beta) ? 1.f : 0.f;
            vb[p] = (1.f - m) * vb[p] + (2.f * m - 1.f) * (*cell);
            *cell = 2.f * clampb(v, beta) - v;
          }
        } else {
          for (int p = threadIdx.x; p < D; p += NT) {
            const int h = p / W, x = p - h * W;
            const float v = vtk[p];
            bf[2 * P * h + x] = 2.f * clampb(v, beta) - v;
          }
        }
        __syncthreads();
        rfft2<G, NT>(g, buf, tw);
        // G_nk += conj(F u^t) rbar_s
        for (int o = threadIdx.x; o < Om; o += NT) {
          const int h = o / Wc, c = o - h * Wc;
          gk[o] = cfmac(buf[h * P + c], rb[o], gk[o]);
        }
        __syncthreads();
        if (MODE == kBIter) {
          for (int p = threadIdx.x; p < D; p += NT) {
            const int h = p / W, x = p - h * W;
            bf[2 * P * h + x] = vb[p];
          }
        }
      }
      if (kAcc) {
        __syncthreads();
        rfft2<G, NT>(g, buf, tw);
        // partial sums for the next reverse step, and G_nk (+)= conj(F vbar) lam_s^{t-1}
        for (int o = threadIdx.x; o < Om; o += NT) {
          const int h = o / Wc, c = o - h * Wc;
          const float2 vh = buf[h * P + c];
          acc[o] = cfma(__ldg(dk + o), vh, acc[o]);
          const float2 base = (MODE == kBSeed) ? make_float2(0.f, 0.f) : gk[o];
          gk[o] = cfmac(vh, lp[o], base);
        }
      }
      __syncthreads();
    }
    if (kAcc) {
      float2* dst = a.part_out + (size_t)(cta + n) * Om;
      for (int o = threadIdx.x; o < Om; o += NT) dst[o] = acc[o];
    }
  }
}

// spectra [m][Omega] -> real maps [m][H][W] (scaled), one CTA per map; optional per-map source
// sum: out = scale * F^{-1}(src[m]) (+ nothing else)
struct SpecMapsArgs {
  int nmaps;
  const float2* spec;  // [m][Omega]
  float* out;          // [m][D]
  float scale;
  const float2* tw;
};

template <class G, int NT>
__global__ void __launch_bounds__(NT) k_spec_to_maps(SpecMapsArgs a, G g) {
  extern __shared__ float2 sm[];
  const int H = g.h(), W = g.w(), P = g.p(), Wc = g.wc(), Om = g.omega();
  float2* buf = sm;
  const Twiddles tw = stage_twiddles<G, NT>(g, buf + H * P, a.tw);
  const float* bf = reinterpret_cast<const float*>(buf);
  for (int m = blockIdx.x; m < a.nmaps; m += gridDim.x) {
    __syncthreads();
    const float2* src = a.spec + (size_t)m * Om;
    for (int o = threadIdx.x; o < Om; o += NT) {
      const int h = o / Wc, c = o - h * Wc;
      buf[h * P + c] = src[o];
    }
    __syncthreads();
    irfft2<G, NT>(g, buf, tw);
    float* dst = a.out + (size_t)m * H * W;
    for (int p = threadIdx.x; p < H * W; p += NT) {
      const int h = p / W, x = p - h * W;
      dst[p] = bf[2 * P * h + x] * a.scale;
    }
  }
}

// filter gradient: gd_k = S F^{-1}( sum_n G_nk - d_hat_k sum_n S_n ), one CTA per filter
struct DgradArgs {
  int N, K, fh, fw;
  const float2* gspec;  // [N][K][Omega]
  const float* S;       // [N][Omega]
  const float2* dhat;   // [K][Omega]
  float* gd;            // [K][fh*fw]
  const float2* tw;
};

template <class G, int NT>
__global__ void __launch_bounds__(NT) k_bwd_dgrad(DgradArgs a, G g) {
  extern __shared__ float2 sm[];
  const int H = g.h(), P = g.p(), Wc = g.wc(), Om = g.omega();
  float2* buf = sm;
  const Twiddles tw = stage_twiddles<G, NT>(g, buf + H * P, a.tw);
  const int k = blockIdx.x;
  for (int o = threadIdx.x; o < Om; o += NT) {
    float2 s = make_float2(0.f, 0.f);
    float st = 0.f;
    for (int n = 0; n < a.N; ++n) {
      s = cadd(s, a.gspec[((size_t)n * a.K + k) * Om + o]);
      st += a.S[(size_t)n * Om + o];
    }
    const float2 dk = a.dhat[(size_t)k * Om + o];
    s.x -= dk.x * st;
    s.y -= dk.y * st;
    const int h = o / Wc, c = o - h * Wc;
    buf[h * P + c] = s;
  }
  __syncthreads();
  irfft2<G, NT>(g, buf, tw);
  crop_window<G, NT>(g, reinterpret_cast<const float*>(buf), a.fh, a.fw, (a.fh - 1) / 2, (a.fw - 1) / 2,
                     1.0f, a.gd + (size_t)k * a.fh * a.fw);
}

// out_nk = scale * F^{-1}( conj(d_hat_k) spec_n ) for every map (D^T applied to per-image spectra)
struct ExpandArgs {
  int N, K;
  const float2* dhat;  // [K][Omega]
  const float2* spec;  // [N][Omega]
  float scale;
  float* out;          // [N][K][D]
  const float2* tw;
};

template <class G, int NT>
__global__ void __launch_bounds__(NT) k_expand(ExpandArgs a, G g) {
  extern __shared__ float2 sm[];
  const int H = g.h(), W = g.w(), P = g.p(), Wc = g.wc(), Om = g.omega(), D = g.d();
  float2* buf = sm;
  const Twiddles tw = stage_twiddles<G, NT>(g, buf + H * P, a.tw);
  const float* bf = reinterpret_cast<const float*>(buf);
  const long long NK = (long long)a.N * a.K;
  for (long long m = blockIdx.x; m < NK; m += gridDim.x) {
    const int n = (int)(m / a.K), k = (int)(m % a.K);
    __syncthreads();
    const float2* dk = a.dhat + (size_t)k * Om;
    const float2* sp = a.spec + (size_t)n * Om;
    for (int o = threadIdx.x; o < Om; o += NT) {
      const int h = o / Wc, c = o - h * Wc;
      buf[h * P + c] = cscale(cfmac(__ldg(dk + o), sp[o], make_float2(0.f, 0.f)), a.scale);
    }
    __syncthreads();
    irfft2<G, NT>(g, buf, tw);
    float* dst = a.out + (size_t)m * D;
    for (int p = threadIdx.x; p < D; p += NT) {
      const int h = p / W, x = p - h * W;
      dst[p] = bf[2 * P * h + x];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// launchers for one geometry
// ---------------------------------------------------------------------------------------------
inline size_t map_smem_bytes(const Geometry& g) {
  return ((size_t)g.H * g.P + (size_t)(g.Wh + g.H + g.Wc)) * sizeof(float2);
}

template <class GEO>
struct GeoLaunch {
  static GEO geo(const Ctx& c) {
    if constexpr (std::is_same<GEO, GeoRT>::value) return c.g.rt;
    else return GEO{};
  }

  static cudaError_t fft_maps(const Ctx& c, const float* in, int nmaps, int filter_mode, float2* out) {
    if (nmaps <= 0) return cudaSuccess;
    FftMapsArgs a{in, nmaps, filter_mode, c.fh, c.fw, out, c.tw};
    const size_t smem = map_smem_bytes(c.g);
    const int grid = std::min(nmaps, c.nsm * 4);
    auto kern = k_fft_maps<GEO, kNT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kNT, smem, c.stream>>>(a, geo(c));
    return cudaGetLastError();
  }

  template <int MODE>
  static cudaError_t sweep_mode(const Ctx& c, const SweepArgs& a) {
    auto kern = k_sweep<GEO, MODE, kNTSweep>;
    const size_t smem = sweep_smem_bytes(c.g, c.J, MODE);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<c.G, kNTSweep, smem, c.stream>>>(a, geo(c));
    return cudaGetLastError();
  }

  static cudaError_t sweep(const Ctx& c, int mode, const SweepArgs& a) {
    switch (mode) {
      case kPrologue: return sweep_mode<kPrologue>(c, a);
      case kIter: return sweep_mode<kIter>(c, a);
      case kLast: return sweep_mode<kLast>(c, a);
      default: return sweep_mode<kObjective>(c, a);
    }
  }

  static cudaError_t rhs(const Ctx& c, const float2* spec) { return rhs_run(c, c.L.zhat, c.xhat, c.L.b, spec); }

  static cudaError_t rhs_ex(const Ctx& c, const float2* zhat, const float2* xhat, float* out) {
    return rhs_run(c, zhat, xhat, out, nullptr);
  }

  static cudaError_t rhs_run(const Ctx& c, const float2* zhat, const float2* xhat, float* out, const float2* spec) {
    RhsArgs a{c.N, c.K, c.J, c.fh, c.fw, zhat, xhat, out, c.tw, spec};
    const size_t smem = map_smem_bytes(c.g);
    auto kern = k_learn_rhs<GEO, kNT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<c.K * c.J, kNT, smem, c.stream>>>(a, geo(c));
    return cudaGetLastError();
  }

  static cudaError_t lags(const Ctx& c) {
    LagsArgs a{c.K, c.fh, c.fw, c.L.gram, c.L.lags, c.tw};
    const size_t smem = map_smem_bytes(c.g);
    const int npairs = c.K * (c.K + 1) / 2;
    auto kern = k_learn_lags<GEO, kNT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<npairs, kNT, smem, c.stream>>>(a, geo(c));
    return cudaGetLastError();
  }

  template <int MODE>
  static cudaError_t bwd_mode(const Ctx& c, const BwdArgs& a) {
    auto kern = k_bwd_sweep<GEO, MODE, kNTSweep>;
    const size_t smem = bwd_smem_bytes(c.g, MODE != kBSeed, MODE != kBLast);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<c.G, kNTSweep, smem, c.stream>>>(a, geo(c));
    return cudaGetLastError();
  }

  static cudaError_t bwd(const Ctx& c, int mode, const BwdArgs& a) {
    switch (mode) {
      case kBSeed: return bwd_mode<kBSeed>(c, a);
      case kBIter: return bwd_mode<kBIter>(c, a);
      default: return bwd_mode<kBLast>(c, a);
    }
  }

  static cudaError_t spec_maps(const Ctx& c, const float2* spec, int nmaps, float scale, float* out) {
    if (nmaps <= 0) return cudaSuccess;
    SpecMapsArgs a{nmaps, spec, out, scale, c.tw};
    const size_t smem = map_smem_bytes(c.g);
    auto kern = k_spec_to_maps<GEO, kNT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<std::min(nmaps, c.nsm * 4), kNT, smem, c.stream>>>(a, geo(c));
    return cudaGetLastError();
  }

  static cudaError_t dgrad(const Ctx& c, const float2* gspec, const float* S, float* gd) {
    DgradArgs a{c.N, c.K, c.fh, c.fw, gspec, S, c.dhat, gd, c.tw};
    const size_t smem = map_smem_bytes(c.g);
    auto kern = k_bwd_dgrad<GEO, kNT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<c.K, kNT, smem, c.stream>>>(a, geo(c));
    return cudaGetLastError();
  }

  static cudaError_t expand(const Ctx& c, const float2* spec, float scale, float* out) {
    ExpandArgs a{c.N, c.K, c.dhat, spec, scale, out, c.tw};
    const size_t smem = map_smem_bytes(c.g);
    auto kern = k_expand<GEO, kNT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long NK = (long long)c.N * c.K;
    kern<<<(int)std::min<long long>(NK, (long long)c.nsm * 4), kNT, smem, c.stream>>>(a, geo(c));
    return cudaGetLastError();
  }

  static const GeoOps& ops() {
    static const GeoOps o{&fft_maps, &sweep, &rhs, &lags, &bwd, &spec_maps, &dgrad, &rhs_ex, &expand};
    return o;
  }
};

}  // namespace csc
