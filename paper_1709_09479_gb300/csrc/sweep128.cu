// The coding sweep for grey 128 x 128 images, with the 2-D FFTs fused into the ADMM steps.
//
// Same arithmetic as k_sweep (Eq. Inference_solution: per map, w_k = F^-1(conj(d_hat_k) lambda_hat),
// the state update, u_k = 2 clamp(v_k) - v_k and the accumulation of d_hat_k F(u_k)), with one
// map's spectrum in shared memory, transformed by the per-thread passes of f128_common.cuh: the
// state update and u sit between the last inverse and the first forward column pass (registers,
// coalesced 8-byte loads and stores of v), and conj(d_hat_k) lambda_hat, the inverse split, the
// forward split and the accumulation of d_hat_k u_hat_k run on each thread's own 16 (+2) bins.
// A map visit takes six block barriers.
//
// Per-thread frequency data (d_hat, lambda_hat, the accumulator) use the thread-major slot order
// of f128_common.cuh; d_hat is copied into that order once per set of filter spectra
// (k_permute_dhat), scaled by 1/2, and lambda_hat is held scaled by 2: the products
// conj(d_hat) lambda_hat are unchanged and the forward split's 1/2 is absorbed (all exact). The
// passes are the packed-pair versions of f128x2.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "csc_internal.cuh"
#include "f128_common.cuh"
#include "f128x2.cuh"

namespace csc {
namespace f128 {

// a complex value rounded to bfloat16 and back (operands of the mixed-precision contractions)
__device__ __forceinline__ float2 to_bf16(float2 v) { return __bfloat1622float2(__floats2bfloat162_rn(v.x, v.y)); }

// PREC 0: float32. PREC 1 (CSC_MIXED_BF16): d_hat comes in bfloat16 (dhatp16, thread-major) and both
// operands of every complex product of the contractions are bfloat16 values, accumulated in float32.
// PREC 2 (CSC_MIXED_TF32): both operands rounded to TF32, accumulated in float32.
template <int MODE, int PREC>
__global__ void __launch_bounds__(NT, 1) k_sweep_f128(SweepArgs a, const float2* __restrict__ dhatp,
                                                      const __nv_bfloat162* __restrict__ dhatp16) {
  extern __shared__ float2 sm[];
  constexpr bool BF = (PREC == 1), TF = (PREC == 2);
  constexpr bool kLam = (MODE == kIter || MODE == kLast);
  constexpr bool kAcc = (MODE != kLast);
  float2* buf = sm;                                   // [128][P]
  float2* lam = buf + H * P;                          // [OM] thread-major
  const int t = threadIdx.x;
  const Tw T{nullptr, nullptr};   // the passes read their twiddles from constant memory

  const Roles R = roles_of(t);
  const int wc = R.wc, g = R.g;
  const bool nyq = R.nyq;

  const long long NK = (long long)a.N * a.K;
  const int cta = blockIdx.x;
  const long long m0 = (long long)cta * NK / a.G, m1 = (long long)(cta + 1) * NK / a.G;
  const float beta = a.beta;
  double l1 = 0.0;
  __syncthreads();

  for (long long n = m0 / a.K; n * a.K < m1; ++n) {
    const int kb = (int)(max(m0, n * a.K) - n * a.K);
    const int ke = (int)(min(m1, (n + 1) * a.K) - n * a.K);
    if (kLam) {
      // lambda_hat / D of image n at this thread's frequencies (slots of the previous sweep)
      const int c0 = (int)(((n * a.K + 1) * a.G - 1) / NK);
      const int c1 = (int)((((n + 1) * a.K) * a.G - 1) / NK);
      const float irho = 1.0f / a.rho;
      const float2* xh = a.xhat + (size_t)n * OM;
      float2* ls = (a.lam_store && cta == c0) ? a.lam_store + (size_t)n * OM : nullptr;
      bool bad = false;
#pragma unroll 2
      for (int s = 0; s < 18; ++s) {
        if (s >= 16 && !nyq) break;
        const int p = slot_pos(s, t);
        const int o = canonical_of(p);
        const float2 x = xh[o];
        const float2 acc2 = sum_slots_at(a.part_in + (size_t)n * OM + o, OM, c0, c1,
                                         make_float2(-x.x * irho, -x.y * irho));
        const float2 l = cscale(acc2, a.pdiag[o]);
        lam[p] = make_float2(2.f * l.x, 2.f * l.y);
        bad |= !(isfinite(l.x) && isfinite(l.y));
        if (ls) ls[o] = l;
      }
      if (bad && a.err) atomicExch(a.err, (int)CSC_ERR_NONFINITE);
    }
    // sum_k d_hat_k u_hat_k of this image at the thread's 16 (+2) bins, in registers
    float2 acc[18];
#pragma unroll
    for (int s = 0; s < 18; ++s) acc[s] = make_float2(0.f, 0.f);

    for (int k = kb; k < ke; ++k) {
      const size_t map = (size_t)n * a.K + k;
      const float2* dk = dhatp + (size_t)k * OM;
      const __nv_bfloat162* dk16 = BF ? dhatp16 + (size_t)k * OM : nullptr;
      auto dval = [&](int p) { return BF ? __bfloat1622float2(dk16[p]) : TF ? tf32r2(__ldg(dk + p)) : __ldg(dk + p); };
      if (threadIdx.x < 4 && (long long)map + 1 < m1) {
        const float* nxt = (MODE == kObjective) ? a.z + (map + 1) * D : a.v + (map + 1) * D;
        prefetch_l2_f128(nxt + threadIdx.x * (D / 4), (unsigned)D);
      }
      float2 zc[16];   // column phase registers: rows h = g + 8 j of column wc
      if (kLam) {
        if (!kAcc) __syncthreads();   // the previous map's column reads precede these writes
        // w_hat = conj(d_hat_k) lambda_hat at this thread's bins, inverse split, first row pass
        inv_rows1_x2(buf, T, R, [&](int s) {
          const int p = slot_pos(s, t);
          return cmulc(BF ? to_bf16(lam[p]) : TF ? tf32r2(lam[p]) : lam[p], dval(p));
        });
        __syncthreads();
        inv_rows2_x2(buf, R);
        __syncthreads();
        inv_cols1_x2(buf, T, R);
        __syncthreads();
        float2 vv[16];   // the state, loaded while the last inverse column pass runs
        const float* vk = a.v + map * D;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          vv[j] = __ldcs(reinterpret_cast<const float2*>(vk + (g + 8 * j) * W + 2 * wc));
        inv_cols2_x2(buf, R, zc);
        // zc[out_slot<16>(j)] is w at rows h = g + 8 j: state update (and codes on the last sweep),
        // two pixels per packed operation
        float* vw = (a.v_out ? a.v_out : a.v) + map * D;
        float* zk = (MODE == kLast && a.z) ? a.z + map * D : nullptr;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float2 w = zc[out_slot<16>(j)];
          const float2 vo = vv[j];
          const float2 vn = pk_sub(w, pk_sub(pk_clamp(vo, beta), vo));   // w - (clamp(v) - v)
          __stcs(reinterpret_cast<float2*>(vw + (g + 8 * j) * W + 2 * wc), vn);
          const float2 cn = pk_clamp(vn, beta);
          if (MODE == kLast) {
            if (zk)
              __stcs(reinterpret_cast<float2*>(zk + (g + 8 * j) * W + 2 * wc),
                     pk_mul(make_float2(a.rho, a.rho), pk_sub(cn, vn)));
          } else {
            vv[j] = pk_fma(vn, make_float2(-1.f, -1.f), pk_add(cn, cn));   // u = 2 clamp(v) - v
          }
        }
        if (kAcc) {
#pragma unroll
          for (int j = 0; j < 16; ++j) zc[j] = vv[j];
        }
      } else {
        // prologue: u = 2 clamp(v) - v; objective: the codes themselves. The previous map's row
        // reads precede these writes.
        __syncthreads();
        const float* src = ((MODE == kPrologue) ? a.v : a.z) + map * D;
        float l1f = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          zc[j] = __ldcs(reinterpret_cast<const float2*>(src + (g + 8 * j) * W + 2 * wc));
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float2 x = zc[j];
          if (MODE == kPrologue) {
            const float2 cx = pk_clamp(x, beta);
            zc[j] = pk_fma(x, make_float2(-1.f, -1.f), pk_add(cx, cx));
          } else {
            l1f += fabsf(x.x) + fabsf(x.y);
          }
        }
        l1 += (double)l1f;
      }

      if (kAcc) {
        fwd_cols1_x2(buf, T, R, zc);
        __syncthreads();
        fwd_cols2_x2(buf, R);
        __syncthreads();
        fwd_rows1_x2(buf, T, R);
        __syncthreads();
        // second forward row pass, split, accumulate d_hat_k u_hat. The d_hat values of the first
        // bin pairs (three in float32: slots 0-2 and 13-15) are loaded before the row transforms,
        // the rest where they are used (registers allow no more in flight)
        constexpr int kPre = (PREC == 0) ? 3 : 1;   // the rounding modes need the registers
        float2 dpre[2 * kPre];
#pragma unroll
        for (int i = 0; i < kPre; ++i) {
          dpre[i] = dval(i * NT + t);
          dpre[kPre + i] = dval((15 - i) * NT + t);
        }
        fwd_rows2_split_x2(buf, T, R, [&](int s, float2 x, bool cj) {
          const float2 xx = BF ? to_bf16(x) : TF ? tf32r2(x) : x;
          const float2 dv = (s < kPre) ? dpre[s] : (s > 15 - kPre && s < 16) ? dpre[kPre + 15 - s] : dval(slot_pos(s, t));
          acc[s] = cj ? make_float2(fmaf(dv.x, xx.x, fmaf(dv.y, xx.y, acc[s].x)),
                                    fmaf(dv.y, xx.x, fmaf(-dv.x, xx.y, acc[s].y)))   // + d conj(x)
                      : cfma(dv, xx, acc[s]);
        });
      }
    }
    if (kAcc) {
      float2* dst = a.part_out + (size_t)(cta + n) * OM;
#pragma unroll
      for (int s = 0; s < 18; ++s)
        if (s < 16 || nyq) dst[canonical_of(slot_pos(s, t))] = acc[s];
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

// out[k][p] = scale * in[k][canonical_of(p)]: spectra into the sweep's thread order
__global__ void k_permute_dhat(const float2* __restrict__ in, float2* __restrict__ out, int K, float scale) {
  const size_t n = (size_t)K * OM;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t k = i / OM;
    const int p = (int)(i - k * OM);
    const float2 v = in[k * OM + canonical_of(p)];
    out[i] = make_float2(scale * v.x, scale * v.y);
  }
}

size_t smem_bytes(int mode) {
  const bool lam = (mode == kIter || mode == kLast);
  return ((size_t)H * P + (lam ? OM : 0)) * sizeof(float2);
}

template <int MODE, int PREC>
cudaError_t launch_mode(const Ctx& c, const SweepArgs& a) {
  auto kern = k_sweep_f128<MODE, PREC>;
  const size_t smem = smem_bytes(MODE);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<c.G, NT, smem, c.stream>>>(a, c.dhatp, c.dhatp16);
  return cudaGetLastError();
}

}  // namespace f128

// the constant-memory twiddle tables of the 128 x 128 sweep on the current device (float64 then
// rounded once); every 128 x 128 context writes the same values
cudaError_t upload_f128_twiddles() {
  const double pi2 = 6.283185307179586476925286766559;
  auto w = [&](int m) {
    return make_float2((float)std::cos(pi2 * m / 128.0), (float)-std::sin(pi2 * m / 128.0));
  };
  float4 q4[128], s4[32];
  for (int a = 0; a < 16; ++a)
    for (int i = 0; i < 8; ++i) {
      const float2 w0 = w((a * (2 * i)) & 127), w1 = w((a * (2 * i + 1)) & 127);
      q4[8 * a + i] = make_float4(w0.x, w0.y, w1.x, w1.y);
    }
  for (int k = 0; k < 8; ++k)
    for (int i = 0; i < 4; ++i) {
      const float2 w0 = w(k + 8 * (2 * i)), w1 = w(k + 8 * (2 * i + 1));
      s4[4 * k + i] = make_float4(w0.x, w0.y, w1.x, w1.y);
    }
  cudaError_t e = cudaMemcpyToSymbol(f128::c_twq4, q4, sizeof(q4));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(f128::c_tws4, s4, sizeof(s4));
  return e;
}

bool fused128_applies(const Ctx& c, const SweepArgs& a) {
  return c.dhatp && c.g.ct_id == 1 && c.J == 1 && a.vec4 && (a.dhat16 == nullptr || c.dhatp16 != nullptr);
}

// a.dhat16 set: mixed precision, with the context's thread-major bf16 copy of d_hat; a.tf32: TF32
// contraction operands
cudaError_t launch_sweep_fused128(const Ctx& c, int mode, const SweepArgs& a) {
  const int prec = (a.dhat16 != nullptr && c.dhatp16 != nullptr) ? 1 : a.tf32 ? 2 : 0;
  switch (mode) {
    case kPrologue:
      return prec == 1 ? f128::launch_mode<kPrologue, 1>(c, a)
                       : prec == 2 ? f128::launch_mode<kPrologue, 2>(c, a) : f128::launch_mode<kPrologue, 0>(c, a);
    case kIter:
      return prec == 1 ? f128::launch_mode<kIter, 1>(c, a)
                       : prec == 2 ? f128::launch_mode<kIter, 2>(c, a) : f128::launch_mode<kIter, 0>(c, a);
    case kLast:
      return prec == 1 ? f128::launch_mode<kLast, 1>(c, a)
                       : prec == 2 ? f128::launch_mode<kLast, 2>(c, a) : f128::launch_mode<kLast, 0>(c, a);
    default: return f128::launch_mode<kObjective, 0>(c, a);
  }
}

cudaError_t launch_permute_f128(const float2* in, float2* out, int nmaps, const Ctx& c) {
  const size_t n = (size_t)nmaps * f128::OM;
  const int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)c.nsm * 8);
  f128::k_permute_dhat<<<grid, 256, 0, c.stream>>>(in, out, nmaps, 1.0f);
  c.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_permute_dhat128(const Ctx& c) {
  const size_t n = (size_t)c.K * f128::OM;
  const int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)c.nsm * 8);
  f128::k_permute_dhat<<<grid, 256, 0, c.stream>>>(c.dhat, c.dhatp, c.K, 0.5f);   // d_hat / 2 (exact)
  c.launches += 1;
  return cudaGetLastError();
}

}  // namespace csc
