// Coding of video tensors (the higher-order extension of Sec. 3.3 with a time axis): J channels x
// T frames x 128 x 128, K filters of support ft x fh x fw per channel, 3-D DFTs.
//
// The 3-D transform is taken as a 2-D transform of every frame followed by a T-point transform
// along time at every 2-D bin. A map's 3-D half spectrum (T x 8320 bins) does not fit in shared
// memory, so one ADMM iteration (Eq. Inference_solution, in the v-state form) is two launches that
// share the array S[N][K][T][8320] of per-frame 2-D spectra in HBM:
//   k_video_bins   (per image, per block of 8 of the 8320 2-D bins): with S = F2(u) of every frame,
//                  r_j(t) = sum_k (D2_jk *_t S_k)(t) in the time domain (a filter has ft time taps,
//                  so the contraction over k needs no time transform), r_hat = F_t r - x_hat / rho,
//                  lambda_hat = P r_hat (J x J per 3-D frequency), lambda = F_t^-1 lambda_hat, and
//                  S_k <- sum_j (conj D2_jk correlated with lambda_j)(t) = F2(w_k) per frame;
//   k_video_frames (per frame): w = F2^-1 S, v <- w - (clamp(v) - v), u = 2 clamp(v) - v and
//                  S <- F2(u), with the fused 128 x 128 passes of f128_common.cuh.
// D2_jk(t', .) is the 2-D spectrum of the filter's time tap t' (offset t' - (ft-1)/2, centred like
// the spatial taps); x_hat and P are per 3-D frequency. All per-bin arrays use the thread-major
// slot order of f128_common.cuh, so both launches read and write them coalesced.
#include <cuda_runtime.h>

#include <algorithm>

#include "csc_internal.cuh"
#include "f128_common.cuh"

namespace csc {
namespace f128 {

constexpr int kVidMaxT = 64;
constexpr int kBinTile = 8;    // 2-D bins per CTA of k_video_bins
constexpr int kBinNT = 256;

// ---------------------------------------------------------------------------------------------
// per frame: F2^-1, state update, F2 (modes as the coding sweep)
// ---------------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(NT, 1) k_video_frames(VideoArgs a) {
  extern __shared__ float2 sm[];
  constexpr bool kInv = (MODE == kIter || MODE == kLast);
  constexpr bool kFwd = (MODE != kLast);
  float2* buf = sm;            // [128][P]
  float2* T = buf + H * P;     // [128]
  const int t = threadIdx.x;
  for (int i = t; i < H; i += NT) T[i] = a.tw[W / 2 + i];
  const Roles R = roles_of(t);
  const int wc = R.wc, g = R.g;
  const long long nf = (long long)a.N * a.K * a.T;
  const long long f0 = (long long)blockIdx.x * nf / gridDim.x, f1 = (long long)(blockIdx.x + 1) * nf / gridDim.x;
  const float beta = a.beta;
  double l1 = 0.0;
  __syncthreads();
  for (long long f = f0; f < f1; ++f) {
    float2* Sf = a.S + (size_t)f * OM;
    if (threadIdx.x < 4 && f + 1 < f1) {
      const float* nxt = (MODE == kObjective) ? a.z + (f + 1) * D : a.v + (f + 1) * D;
      prefetch_l2_f128(nxt + threadIdx.x * (D / 4), (unsigned)D);
      if (kInv) prefetch_l2_f128(Sf + OM + threadIdx.x * (OM / 4), (unsigned)(OM / 4 * sizeof(float2)));
    }
    float2 zc[16];
    if (kInv) {
      if (!kFwd) __syncthreads();   // the previous frame's column reads precede these writes
      inv_rows1(buf, T, R, [&](int s) { return __ldcs(Sf + slot_pos(s, t)); });
      __syncthreads();
      inv_rows2(buf, R);
      __syncthreads();
      inv_cols1(buf, T, R);
      __syncthreads();
      float2 vv[16];
      const float* vk = a.v + f * D;
#pragma unroll
      for (int j = 0; j < 16; ++j) vv[j] = __ldcs(reinterpret_cast<const float2*>(vk + (g + 8 * j) * W + 2 * wc));
      inv_cols2(buf, R, zc);
      float* vw = a.v + f * D;
      float* zk = (MODE == kLast && a.z) ? a.z + f * D : nullptr;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float2 w = zc[out_slot<16>(j)];
        const float2 vo = vv[j];
        float2 vn;
        vn.x = w.x - (clampb(vo.x, beta) - vo.x);
        vn.y = w.y - (clampb(vo.y, beta) - vo.y);
        __stcs(reinterpret_cast<float2*>(vw + (g + 8 * j) * W + 2 * wc), vn);
        if (MODE == kLast) {
          if (zk)
            __stcs(reinterpret_cast<float2*>(zk + (g + 8 * j) * W + 2 * wc),
                   make_float2(a.rho * (clampb(vn.x, beta) - vn.x), a.rho * (clampb(vn.y, beta) - vn.y)));
        } else {
          vv[j] = make_float2(2.f * clampb(vn.x, beta) - vn.x, 2.f * clampb(vn.y, beta) - vn.y);
        }
      }
      if (kFwd) {
#pragma unroll
        for (int j = 0; j < 16; ++j) zc[j] = vv[j];
      }
    } else {
      __syncthreads();   // the previous frame's row reads precede these writes
      const float* src = ((MODE == kPrologue) ? a.v : a.z) + f * D;
      float l1f = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) zc[j] = __ldcs(reinterpret_cast<const float2*>(src + (g + 8 * j) * W + 2 * wc));
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float2 x = zc[j];
        if (MODE == kPrologue) zc[j] = make_float2(2.f * clampb(x.x, beta) - x.x, 2.f * clampb(x.y, beta) - x.y);
        else l1f += fabsf(x.x) + fabsf(x.y);
      }
      l1 += (double)l1f;
    }
    if (kFwd) {
      fwd_cols1(buf, T, R, zc);
      __syncthreads();
      fwd_cols2(buf, R);
      __syncthreads();
      fwd_rows1(buf, T, R);
      __syncthreads();
      fwd_rows2_split(buf, T, R, [&](int s, float2 x) { __stcs(Sf + slot_pos(s, t), x); });
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
      a.l1[blockIdx.x] = s;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// per block of 2-D bins: the contraction over filters, the per-frequency solve and the products
// with conj(d_hat), all along time; or (objective) the residual's energy by Parseval
// ---------------------------------------------------------------------------------------------
template <int MODE, int JT>
__global__ void __launch_bounds__(kBinNT) k_video_bins(VideoArgs a) {
  constexpr int J = JT;
  __shared__ float2 sS[4][kVidMaxT][kBinTile];        // S_k tiles of 4 filters
  __shared__ float2 sD[4][J][8][kBinTile];            // their time taps (ft <= 8)
  __shared__ float2 sr[J][kVidMaxT][kBinTile];         // r, then lambda
  __shared__ float2 sx[J][kVidMaxT][kBinTile];         // r_hat, lambda_hat
  __shared__ float2 tw[kVidMaxT];                      // exp(-2 pi i m / T)
  __shared__ double red[kBinNT / 32];
  const int T = a.T, K = a.K, ft = a.ft, oc = (a.ft - 1) / 2;
  const int n = blockIdx.y;
  const int p0 = blockIdx.x * kBinTile;
  const int tid = threadIdx.x;
  const int pp = tid % kBinTile;                       // bin of the tile
  for (int i = tid; i < T; i += kBinNT) {
    float s, c;
    sincospif(2.0f * (float)i / (float)T, &s, &c);
    tw[i] = make_float2(c, -s);
  }
  // ---- r_j(t) = sum_k sum_t' D2_jk(t') S_k(t - o(t')) -------------------------------------
  // thread e = (j, t, pp) accumulates outputs e, e + 256, ... (J * T * 8 <= 3 * 64 * 8)
  constexpr int kOut = (J * kVidMaxT * kBinTile + kBinNT - 1) / kBinNT;
  float2 acc[kOut];
#pragma unroll
  for (int u = 0; u < kOut; ++u) acc[u] = make_float2(0.f, 0.f);
  const int nout = J * T * kBinTile;
  for (int k0 = 0; k0 < K; k0 += 4) {
    const int nk = min(4, K - k0);
    __syncthreads();
    for (int i = tid; i < nk * T * kBinTile; i += kBinNT) {
      const int kk = i / (T * kBinTile), rem = i - kk * T * kBinTile, tt = rem / kBinTile, b = rem - tt * kBinTile;
      const size_t fr = ((size_t)n * K + k0 + kk) * T + tt;
      sS[kk][tt][b] = __ldcs(a.S + fr * OM + p0 + b);
    }
    for (int i = tid; i < nk * J * ft * kBinTile; i += kBinNT) {
      const int kk = i / (J * ft * kBinTile), rem = i - kk * J * ft * kBinTile;
      const int j = rem / (ft * kBinTile), rem2 = rem - j * ft * kBinTile, tp = rem2 / kBinTile, b = rem2 - tp * kBinTile;
      sD[kk][j][tp][b] = __ldg(a.d2 + (((size_t)(k0 + kk) * J + j) * ft + tp) * OM + p0 + b);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kOut; ++u) {
      const int e = tid + u * kBinNT;
      if (e < nout) {
        const int j = e / (T * kBinTile), rem = e - j * T * kBinTile, tt = rem / kBinTile, b = rem - tt * kBinTile;
        float2 s = acc[u];
        for (int kk = 0; kk < nk; ++kk)
          for (int tp = 0; tp < ft; ++tp) {
            int ts = tt - (tp - oc);
            ts = ts < 0 ? ts + T : (ts >= T ? ts - T : ts);
            s = cfma(sD[kk][j][tp][b], sS[kk][ts][b], s);
          }
        acc[u] = s;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kOut; ++u) {
    const int e = tid + u * kBinNT;
    if (e < nout) {
      const int j = e / (T * kBinTile), rem = e - j * T * kBinTile, tt = rem / kBinTile, b = rem - tt * kBinTile;
      sr[j][tt][b] = acc[u];
    }
  }
  __syncthreads();
  // ---- r_hat = F_t r - x_hat / rho (iterate) or - x_hat (objective) ------------------------
  const float xs = (MODE == kObjective) ? 1.f : 1.f / a.rho;
  for (int e = tid; e < nout; e += kBinNT) {
    const int j = e / (T * kBinTile), rem = e - j * T * kBinTile, tau = rem / kBinTile, b = rem - tau * kBinTile;
    float2 s = make_float2(0.f, 0.f);
    int m = 0;
    for (int tt = 0; tt < T; ++tt) {
      s = cfma(sr[j][tt][b], tw[m], s);
      m += tau;
      if (m >= T) m -= T;
    }
    const float2 xh = a.xh3[(((size_t)n * J + j) * T + tau) * OM + p0 + b];
    sx[j][tau][b] = make_float2(s.x - xs * xh.x, s.y - xs * xh.y);
  }
  __syncthreads();
  if (MODE == kObjective) {
    // sum_{tau, bins} wt |r_hat|^2 / (T H W), wt = 1 on the kw = 0 and kw = 64 columns, else 2
    double e2 = 0.0;
    for (int e = tid; e < nout; e += kBinNT) {
      const int j = e / (T * kBinTile), rem = e - j * T * kBinTile, tau = rem / kBinTile, b = rem - tau * kBinTile;
      const int kw = canonical_of(p0 + b) % 65;
      const float wt = (kw == 0 || kw == 64) ? 1.f : 2.f;
      const float2 v = sx[j][tau][b];
      e2 += (double)(wt * (v.x * v.x + v.y * v.y));
    }
    for (int off = 16; off > 0; off >>= 1) e2 += __shfl_down_sync(0xffffffffu, e2, off);
    if ((tid & 31) == 0) red[tid >> 5] = e2;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int i = 0; i < kBinNT / 32; ++i) s += red[i];
      a.objpart[(size_t)n * gridDim.x + blockIdx.x] = s / ((double)T * D);
    }
    return;
  }
  // ---- lambda_hat = P r_hat; lambda = F_t^-1 lambda_hat (P carries 1/(H W)) -----------------
  for (int e = tid; e < T * kBinTile; e += kBinNT) {
    const int tau = e / kBinTile, b = e - tau * kBinTile;
    const float2* Pm = a.p3 + ((size_t)tau * OM + p0 + b) * J * J;
    float2 rv[J];
#pragma unroll
    for (int j = 0; j < J; ++j) rv[j] = sx[j][tau][b];
#pragma unroll
    for (int i = 0; i < J; ++i) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < J; ++j) s = cfma(__ldg(Pm + i * J + j), rv[j], s);
      sr[i][tau][b] = s;   // lambda_hat
    }
  }
  __syncthreads();
  const float iT = 1.f / (float)T;
  for (int e = tid; e < nout; e += kBinNT) {
    const int j = e / (T * kBinTile), rem = e - j * T * kBinTile, tt = rem / kBinTile, b = rem - tt * kBinTile;
    float2 s = make_float2(0.f, 0.f);
    int m = 0;
    for (int tau = 0; tau < T; ++tau) {
      s = cfmac(tw[m], sr[j][tau][b], s);   // exp(+2 pi i tau t / T) lambda_hat
      m += tt;
      if (m >= T) m -= T;
    }
    sx[j][tt][b] = cscale(s, iT);   // lambda
  }
  __syncthreads();
  // ---- S_k(t) <- sum_j sum_t' conj(D2_jk(t')) lambda_j(t + o(t')) ---------------------------
  for (int k0 = 0; k0 < K; k0 += 4) {
    const int nk = min(4, K - k0);
    __syncthreads();
    for (int i = tid; i < nk * J * ft * kBinTile; i += kBinNT) {
      const int kk = i / (J * ft * kBinTile), rem = i - kk * J * ft * kBinTile;
      const int j = rem / (ft * kBinTile), rem2 = rem - j * ft * kBinTile, tp = rem2 / kBinTile, b = rem2 - tp * kBinTile;
      sD[kk][j][tp][b] = __ldg(a.d2 + (((size_t)(k0 + kk) * J + j) * ft + tp) * OM + p0 + b);
    }
    __syncthreads();
    for (int i = tid; i < nk * T * kBinTile; i += kBinNT) {
      const int kk = i / (T * kBinTile), rem = i - kk * T * kBinTile, tt = rem / kBinTile, b = rem - tt * kBinTile;
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < J; ++j)
        for (int tp = 0; tp < ft; ++tp) {
          int ts = tt + (tp - oc);
          ts = ts < 0 ? ts + T : (ts >= T ? ts - T : ts);
          s = cfmac(sD[kk][j][tp][b], sx[j][ts][b], s);
        }
      const size_t fr = ((size_t)n * K + k0 + kk) * T + tt;
      __stcs(a.S + fr * OM + p0 + b, s);
    }
  }
}

// x_hat3[n][j][tau][p] = sum_t exp(-2 pi i tau t / T) F2(x_njt)[canonical_of(p)]
__global__ void k_video_xhat(VideoArgs a, const float2* __restrict__ x2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int nj = blockIdx.y, tau = blockIdx.z;
  if (p >= OM) return;
  const int o = canonical_of(p);
  const int T = a.T;
  float2 s = make_float2(0.f, 0.f);
  for (int tt = 0; tt < T; ++tt) {
    float sn, cs;
    sincospif(2.0f * (float)((tau * tt) % T) / (float)T, &sn, &cs);
    s = cfma(x2[((size_t)nj * T + tt) * OM + o], make_float2(cs, -sn), s);
  }
  a.xh3[((size_t)nj * T + tau) * OM + p] = s;
}

// P(tau, p) = (A + I / rho)^{-1} / (H W), A_ij = sum_k d_hat_ik conj(d_hat_jk) at the 3-D frequency,
// d_hat_jk(tau, p) = sum_t' exp(-2 pi i tau o(t') / T) D2_jk(t', p); float64, Gauss-Jordan
template <int JT>
__global__ void k_video_prep(VideoArgs a) {
  constexpr int J = JT;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int tau = blockIdx.y;
  if (p >= OM) return;
  const int T = a.T, ft = a.ft, oc = (a.ft - 1) / 2;
  double re[J][2 * J], im[J][2 * J];
#pragma unroll
  for (int i = 0; i < J; ++i)
#pragma unroll
    for (int j = 0; j < 2 * J; ++j) { re[i][j] = 0.0; im[i][j] = 0.0; }
  for (int k = 0; k < a.K; ++k) {
    double dr[J], di[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      dr[j] = 0.0;
      di[j] = 0.0;
      for (int tp = 0; tp < ft; ++tp) {
        const int m = ((tau * (tp - oc)) % T + T) % T;
        double sn, cs;
        sincospi(2.0 * (double)m / (double)T, &sn, &cs);
        const float2 v = a.d2[(((size_t)k * J + j) * ft + tp) * OM + p];
        dr[j] += (double)v.x * cs + (double)v.y * sn;    // v * exp(-i phi)
        di[j] += (double)v.y * cs - (double)v.x * sn;
      }
    }
#pragma unroll
    for (int i = 0; i < J; ++i)
#pragma unroll
      for (int j = 0; j < J; ++j) {
        re[i][j] += dr[i] * dr[j] + di[i] * di[j];
        im[i][j] += di[i] * dr[j] - dr[i] * di[j];
      }
  }
#pragma unroll
  for (int i = 0; i < J; ++i) { re[i][i] += 1.0 / a.rho; re[i][J + i] = 1.0; }
#pragma unroll
  for (int c = 0; c < J; ++c) {
    const double pr = re[c][c], pi = im[c][c];
    const double den = pr * pr + pi * pi;
    const double ir = pr / den, ii = -pi / den;
#pragma unroll
    for (int j = 0; j < 2 * J; ++j) {
      const double xr = re[c][j], xi = im[c][j];
      re[c][j] = xr * ir - xi * ii;
      im[c][j] = xr * ii + xi * ir;
    }
#pragma unroll
    for (int i = 0; i < J; ++i) {
      if (i == c) continue;
      const double fr = re[i][c], fi = im[i][c];
#pragma unroll
      for (int j = 0; j < 2 * J; ++j) {
        re[i][j] -= fr * re[c][j] - fi * im[c][j];
        im[i][j] -= fr * im[c][j] + fi * re[c][j];
      }
    }
  }
  const double sc = 1.0 / (double)D;
  float2* out = a.p3 + ((size_t)tau * OM + p) * J * J;
#pragma unroll
  for (int i = 0; i < J; ++i)
#pragma unroll
    for (int j = 0; j < J; ++j) out[i * J + j] = make_float2((float)(re[i][J + j] * sc), (float)(im[i][J + j] * sc));
}

template <int MODE>
cudaError_t launch_frames_mode(const VideoArgs& a, int G, cudaStream_t st) {
  auto kern = k_video_frames<MODE>;
  const size_t smem = ((size_t)H * P + H) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<G, NT, smem, st>>>(a);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_bins_mode(const VideoArgs& a, cudaStream_t st) {
  dim3 grid(OM / kBinTile, a.N);
  switch (a.J) {
    case 1: k_video_bins<MODE, 1><<<grid, kBinNT, 0, st>>>(a); break;
    case 2: k_video_bins<MODE, 2><<<grid, kBinNT, 0, st>>>(a); break;
    default: k_video_bins<MODE, 3><<<grid, kBinNT, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

}  // namespace f128

size_t video_frames_smem_bytes() { return ((size_t)f128::H * f128::P + f128::H) * sizeof(float2); }
int video_max_T() { return f128::kVidMaxT; }
int video_bin_blocks() { return f128::OM / f128::kBinTile; }

cudaError_t launch_video_frames(const VideoArgs& a, int mode, int G, cudaStream_t st) {
  switch (mode) {
    case kPrologue: return f128::launch_frames_mode<kPrologue>(a, G, st);
    case kIter: return f128::launch_frames_mode<kIter>(a, G, st);
    case kLast: return f128::launch_frames_mode<kLast>(a, G, st);
    default: return f128::launch_frames_mode<kObjective>(a, G, st);
  }
}

cudaError_t launch_video_bins(const VideoArgs& a, int mode, cudaStream_t st) {
  return mode == kObjective ? f128::launch_bins_mode<kObjective>(a, st) : f128::launch_bins_mode<kIter>(a, st);
}

cudaError_t launch_video_setup(const VideoArgs& a, const float2* x2, cudaStream_t st) {
  dim3 gx((f128::OM + 255) / 256, a.N * a.J, a.T);
  f128::k_video_xhat<<<gx, 256, 0, st>>>(a, x2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 gp((f128::OM + 127) / 128, a.T);
  switch (a.J) {
    case 1: f128::k_video_prep<1><<<gp, 128, 0, st>>>(a); break;
    case 2: f128::k_video_prep<2><<<gp, 128, 0, st>>>(a); break;
    default: f128::k_video_prep<3><<<gp, 128, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

}  // namespace csc
