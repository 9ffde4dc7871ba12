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
constexpr int kBinTile = 32;   // 2-D bins per CTA of k_video_bins (one warp's lanes)
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
  const int t = threadIdx.x;
  const Tw T = build_tw<NT>(buf + H * P, a.tw + W / 2);
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
// Thread layout: lane = bin of a 32-bin tile (every load and store of S, D2, x_hat and P moves
// 256 contiguous bytes per warp), warp = row of work. The two convolutions along time are register
// blocked over four consecutive frames (and, for r, over all channels), so a staged S or lambda
// value is loaded once per four outputs. Shared memory (dynamic, sized by T): S tiles of KS
// filters, their time taps, and two J x T x 32 work arrays.
constexpr int kKS = 4;
constexpr int kTB = 4;   // frames per register block
template <int J>
__host__ __device__ constexpr size_t bins_smem_floats(int T) {
  return 2 * ((size_t)kKS * T * kBinTile + (size_t)kKS * J * 8 * kBinTile + 2 * (size_t)J * T * kBinTile + T);
}

template <int MODE, int JT, int FT>
__global__ void __launch_bounds__(kBinNT) k_video_bins(VideoArgs a) {
  constexpr int J = JT;
  constexpr int KS = kKS;
  constexpr int B = kBinTile;                          // 32 bins = one warp's lanes
  constexpr int NW = kBinNT / 32;                      // 8 warps
  constexpr int OC = (FT - 1) / 2;
  constexpr int WIN = kTB + FT - 1;                    // frames a block of four outputs reads
  extern __shared__ float2 vsm[];
  const int T = a.T, K = a.K;
  float2* sS = vsm;                                    // [KS][T][B]
  float2* sD = sS + (size_t)KS * T * B;                // [KS][J][8][B]
  float2* sr = sD + (size_t)KS * J * 8 * B;            // [J][T][B]: r, then lambda_hat
  float2* sx = sr + (size_t)J * T * B;                 // [J][T][B]: r_hat, then lambda
  float2* tw = sx + (size_t)J * T * B;                 // [T] exp(-2 pi i m / T)
  __shared__ double red[NW];
  const int n = blockIdx.y;
  const int p0 = blockIdx.x * B;
  const int tid = threadIdx.x;
  const int b = tid & 31, w = tid >> 5;
  for (int i = tid; i < T; i += kBinNT) {
    float s, c;
    sincospif(2.0f * (float)i / (float)T, &s, &c);
    tw[i] = make_float2(c, -s);
  }
  const int nblk = (T + kTB - 1) / kTB;                // frame blocks (T <= 64: <= 16)
  const int nout = J * T;
  const size_t fbase = (size_t)n * K * T;
  auto wrap = [T](int t) {   // t mod T for any t (windows may extend more than T past the ends when T < 4)
    t %= T;
    return t < 0 ? t + T : t;
  };
  // ---- r_j(t) = sum_k sum_t' D2_jk(t') S_k(t - o(t')): warp w, frame blocks w and w + 8 -------
  float2 acc[2][J][kTB];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int i = 0; i < kTB; ++i) acc[h][j][i] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < K; k0 += KS) {
    const int nk = min(KS, K - k0);
    __syncthreads();
    for (int e = w; e < nk * T; e += NW) {
      const int kk = e / T, tt = e - kk * T;
      sS[((size_t)kk * T + tt) * B + b] = __ldcs(a.S + (fbase + (size_t)(k0 + kk) * T + tt) * OM + p0 + b);
    }
    for (int e = w; e < nk * J * FT; e += NW) {
      const int kk = e / (J * FT), rem = e - kk * J * FT, j = rem / FT, tp = rem - j * FT;
      sD[(((size_t)kk * J + j) * 8 + tp) * B + b] = __ldg(a.d2 + (((size_t)(k0 + kk) * J + j) * FT + tp) * OM + p0 + b);
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int blk = w + NW * h;
      if (blk < nblk) {
        const int t0 = kTB * blk;
        for (int kk = 0; kk < nk; ++kk) {
          // S_k(t0 + i - tp + OC) for i < 4, tp < FT: window index wi = i - tp + FT - 1
          float2 win[WIN];
#pragma unroll
          for (int wi = 0; wi < WIN; ++wi) win[wi] = sS[((size_t)kk * T + wrap(t0 + wi - (FT - 1) + OC)) * B + b];
#pragma unroll
          for (int j = 0; j < J; ++j) {
            float2 dv[FT];
#pragma unroll
            for (int tp = 0; tp < FT; ++tp) dv[tp] = sD[(((size_t)kk * J + j) * 8 + tp) * B + b];
#pragma unroll
            for (int i = 0; i < kTB; ++i)
#pragma unroll
              for (int tp = 0; tp < FT; ++tp) acc[h][j][i] = cfma(dv[tp], win[i - tp + FT - 1], acc[h][j][i]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int blk = w + NW * h;
    if (blk < nblk)
#pragma unroll
      for (int j = 0; j < J; ++j)
#pragma unroll
        for (int i = 0; i < kTB; ++i)
          if (kTB * blk + i < T) sr[((size_t)j * T + kTB * blk + i) * B + b] = acc[h][j][i];
  }
  __syncthreads();
  // ---- r_hat = F_t r - x_hat / rho (iterate) or - x_hat (objective) ------------------------
  const float xs = (MODE == kObjective) ? 1.f : 1.f / a.rho;
  for (int e = w; e < nout; e += NW) {
    const int j = e / T, tau = e - j * T;
    const float2* rj = sr + (size_t)j * T * B + b;
    float2 s = make_float2(0.f, 0.f);
    int m = 0;
    for (int tt = 0; tt < T; ++tt) {
      s = cfma(rj[tt * B], tw[m], s);
      m += tau;
      if (m >= T) m -= T;
    }
    const float2 xh = a.xh3[(((size_t)n * J + j) * T + tau) * OM + p0 + b];
    sx[(size_t)e * B + b] = make_float2(s.x - xs * xh.x, s.y - xs * xh.y);
  }
  __syncthreads();
  if (MODE == kObjective) {
    // sum_{tau, bins} wt |r_hat|^2 / (T H W), wt = 1 on the kw = 0 and kw = 64 columns, else 2
    const int kw = canonical_of(p0 + b) % 65;
    const float wt = (kw == 0 || kw == 64) ? 1.f : 2.f;
    double e2 = 0.0;
    for (int e = w; e < nout; e += NW) {
      const float2 v = sx[(size_t)e * B + b];
      e2 += (double)(wt * (v.x * v.x + v.y * v.y));
    }
    for (int off = 16; off > 0; off >>= 1) e2 += __shfl_down_sync(0xffffffffu, e2, off);
    if (b == 0) red[w] = e2;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int i = 0; i < NW; ++i) s += red[i];
      a.objpart[(size_t)n * gridDim.x + blockIdx.x] = s / ((double)T * D);
    }
    return;
  }
  // ---- lambda_hat = P r_hat (P carries 1/(H W)) ---------------------------------------------
  for (int tau = w; tau < T; tau += NW) {
    const float2* Pm = a.p3 + ((size_t)tau * OM + p0 + b) * J * J;
    float2 rv[J];
#pragma unroll
    for (int j = 0; j < J; ++j) rv[j] = sx[((size_t)j * T + tau) * B + b];
#pragma unroll
    for (int i = 0; i < J; ++i) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < J; ++j) s = cfma(__ldg(Pm + i * J + j), rv[j], s);
      sr[((size_t)i * T + tau) * B + b] = s;
    }
  }
  __syncthreads();
  // ---- lambda = F_t^-1 lambda_hat ------------------------------------------------------------
  const float iT = 1.f / (float)T;
  for (int e = w; e < nout; e += NW) {
    const int j = e / T, tt = e - j * T;
    const float2* lj = sr + (size_t)j * T * B + b;
    float2 s = make_float2(0.f, 0.f);
    int m = 0;
    for (int tau = 0; tau < T; ++tau) {
      s = cfmac(tw[m], lj[tau * B], s);   // exp(+2 pi i tau t / T) lambda_hat
      m += tt;
      if (m >= T) m -= T;
    }
    sx[(size_t)e * B + b] = cscale(s, iT);
  }
  // ---- S_k(t) <- sum_j sum_t' conj(D2_jk(t')) lambda_j(t + o(t')): (filter, frame block) rows --
  for (int k0 = 0; k0 < K; k0 += KS) {
    const int nk = min(KS, K - k0);
    __syncthreads();
    for (int e = w; e < nk * J * FT; e += NW) {
      const int kk = e / (J * FT), rem = e - kk * J * FT, j = rem / FT, tp = rem - j * FT;
      sD[(((size_t)kk * J + j) * 8 + tp) * B + b] = __ldg(a.d2 + (((size_t)(k0 + kk) * J + j) * FT + tp) * OM + p0 + b);
    }
    __syncthreads();
    for (int e = w; e < nk * nblk; e += NW) {
      const int kk = e / nblk, blk = e - kk * nblk, t0 = kTB * blk;
      float2 o4[kTB];
#pragma unroll
      for (int i = 0; i < kTB; ++i) o4[i] = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < J; ++j) {
        // lambda_j(t0 + i + tp - OC): window index wi = i + tp
        float2 win[WIN];
#pragma unroll
        for (int wi = 0; wi < WIN; ++wi) win[wi] = sx[((size_t)j * T + wrap(t0 + wi - OC)) * B + b];
#pragma unroll
        for (int tp = 0; tp < FT; ++tp) {
          const float2 dv = sD[(((size_t)kk * J + j) * 8 + tp) * B + b];
#pragma unroll
          for (int i = 0; i < kTB; ++i) o4[i] = cfmac(dv, win[i + tp], o4[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < kTB; ++i)
        if (t0 + i < T) __stcs(a.S + (fbase + (size_t)(k0 + kk) * T + t0 + i) * OM + p0 + b, o4[i]);
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
// d_hat_jk(tau, p) = sum_t' exp(-2 pi i tau o(t') / T) D2_jk(t', p) (float32, ft terms); A is summed
// over filters in float32 with Kahan-Babuska compensation and inverted (Gauss-Jordan) in float64
template <int JT>
__global__ void k_video_prep(VideoArgs a) {
  constexpr int J = JT;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int tau = blockIdx.y;
  if (p >= OM) return;
  const int T = a.T, ft = a.ft, oc = (a.ft - 1) / 2;
  float2 ph[8];   // exp(-2 pi i tau o(t') / T), t' < ft <= 7
#pragma unroll
  for (int tp = 0; tp < 8; ++tp) {
    const int m = ((tau * (tp - oc)) % T + T) % T;
    float sn, cs;
    sincospif(2.0f * (float)m / (float)T, &sn, &cs);
    ph[tp] = make_float2(cs, -sn);
  }
  // A summed over filters in float32 with compensation (the float64 rate is low), inverted in float64
  float ar[J][J], ai[J][J], cr[J][J], ci[J][J];
#pragma unroll
  for (int i = 0; i < J; ++i)
#pragma unroll
    for (int j = 0; j < J; ++j) { ar[i][j] = ai[i][j] = cr[i][j] = ci[i][j] = 0.f; }
  auto kadd = [](float& s, float& c, float v) {   // Kahan-Babuska step
    const float t = s + v;
    c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
    s = t;
  };
  for (int k = 0; k < a.K; ++k) {
    float2 dk[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      float2 sacc = make_float2(0.f, 0.f);
#pragma unroll
      for (int tp = 0; tp < 8; ++tp)
        if (tp < ft) sacc = cfma(a.d2[(((size_t)k * J + j) * ft + tp) * OM + p], ph[tp], sacc);
      dk[j] = sacc;
    }
#pragma unroll
    for (int i = 0; i < J; ++i)
#pragma unroll
      for (int j = 0; j < J; ++j) {
        kadd(ar[i][j], cr[i][j], dk[i].x * dk[j].x + dk[i].y * dk[j].y);
        kadd(ai[i][j], ci[i][j], dk[i].y * dk[j].x - dk[i].x * dk[j].y);
      }
  }
  double re[J][2 * J], im[J][2 * J];
#pragma unroll
  for (int i = 0; i < J; ++i)
#pragma unroll
    for (int j = 0; j < J; ++j) {
      re[i][j] = (double)ar[i][j] + (double)cr[i][j];
      im[i][j] = (double)ai[i][j] + (double)ci[i][j];
      re[i][J + j] = 0.0;
      im[i][J + j] = 0.0;
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
  const size_t smem = ((size_t)H * P + kTwEntries) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<G, NT, smem, st>>>(a);
  return cudaGetLastError();
}

template <int MODE, int J, int FT>
cudaError_t launch_bins_mjf(const VideoArgs& a, cudaStream_t st) {
  auto kern = k_video_bins<MODE, J, FT>;
  const size_t smem = bins_smem_floats<J>(a.T) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(OM / kBinTile, a.N);
  kern<<<grid, kBinNT, smem, st>>>(a);
  return cudaGetLastError();
}

template <int MODE, int J>
cudaError_t launch_bins_mj(const VideoArgs& a, cudaStream_t st) {
  switch (a.ft) {
    case 1: return launch_bins_mjf<MODE, J, 1>(a, st);
    case 3: return launch_bins_mjf<MODE, J, 3>(a, st);
    case 5: return launch_bins_mjf<MODE, J, 5>(a, st);
    default: return launch_bins_mjf<MODE, J, 7>(a, st);
  }
}

template <int MODE>
cudaError_t launch_bins_mode(const VideoArgs& a, cudaStream_t st) {
  switch (a.J) {
    case 1: return launch_bins_mj<MODE, 1>(a, st);
    case 2: return launch_bins_mj<MODE, 2>(a, st);
    default: return launch_bins_mj<MODE, 3>(a, st);
  }
}

}  // namespace f128

size_t video_frames_smem_bytes() { return ((size_t)f128::H * f128::P + f128::kTwEntries) * sizeof(float2); }
int video_max_T() { return f128::kVidMaxT; }
int video_bin_blocks() { return f128::OM / f128::kBinTile; }
size_t video_bins_smem_bytes(int J, int T) {
  return (J == 1 ? f128::bins_smem_floats<1>(T) : J == 2 ? f128::bins_smem_floats<2>(T) : f128::bins_smem_floats<3>(T)) * sizeof(float);
}

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
