// The learning subproblem (Sec. 3.2, Eqs. Learning_new .. mu_update) on video tensors (the
// higher-order extension of Sec. 3.3 with a time axis): J channels x T frames x 128 x 128, filters
// ft x fh x fw per channel, one mu_k and one unit norm per filter over all its channels and taps.
//
// Same route as the 2-D learning: the filter-space normal equations
//     (S Z^T Z S^T + 2 diag(mu)) d_j = S Z^T x_j        (one system per channel, shared matrix)
// with the matrix the code cross-correlation on the (2ft-1) x (2fh-1) x (2fw-1) lag window, formed once
// per call from the per-frequency Gram of the codes' 3-D spectra:
//   1. per-frame 2-D spectra of the codes and images (the fused 128 x 128 passes), then the T-point
//      DFT along time (k_dft_time): z_hat_nk(tau, w), x_hat_nj(tau, w);
//   2. frequency-major copy of z_hat and the tensor-core Gram over the T x 8320 frequencies
//      (k_gram_tc, shared with the 2-D path), the right-hand-side spectra as its J extra columns;
//   3. the lag window C_kk'(tau) = F^-1 G_kk' / D and the right-hand side b = crop F^-1(R) / D as
//      direct partial sums: over w (65 -> Lb) and h (128 -> La) per time frequency (k_vl_rows), then
//      over the time frequency (k_vl_time);
//   4. lag spectra C_hat on the window grid (k_vl_lagspec), separable DFTs;
//   5. preconditioned CG per learning step, the operator in the Fourier domain of the lag grid:
//      taps -> bins (k_vl_t2b), y_hat_k = sum_k' C_hat_kk' p_hat_k' (k_vl_prod), bins -> taps
//      (k_vl_b2t; the direction update rides on k_vl_t2b and the p . Ap partials on k_vl_b2t), and the
//      x, r, z updates with float64 dot products over all SMs (k_vl_it_upd, k_vl_it_scal); Jacobi
//      preconditioner 1 / (C_kk(0) + 2 mu_k); then mu_k <- max(mu_k ||d_k||, floor) (k_vl_step_end),
//      and after the last step d_k <- d_k / max(1, ||d_k||).
// Filters whose codes are all zero keep d_k and mu_k. The host drives the CG iterations in batches
// of 8 iterations (a CUDA graph recorded once per call) and reads the device's convergence flag
// between batches.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "csc_internal.cuh"

namespace csc {
namespace vl {

constexpr int H = 128, W = 128, Wc = 65, OM = H * Wc;
constexpr int kMaxL = 24;           // lag / support window per spatial axis (filters up to 12 taps)
constexpr int kRowsPairs = 8, kRowsSub = 16, kRowsNT = kRowsPairs * kRowsSub, kRowsStages = 4;
constexpr int kCgNT = 1024;

__device__ __forceinline__ float2 root(long long m, int L, float sign) {   // exp(sign 2 pi i m / L)
  int r = (int)(m % L);
  if (r < 0) r += L;
  float s, c;
  sincospif(2.0f * (float)r / (float)L, &s, &c);
  return make_float2(c, sign * s);
}

__device__ __forceinline__ int imod(int m, int L) {
  const int r = m % L;
  return r < 0 ? r + L : r;
}

// tab[m] = exp(sign 2 pi i m / L), m < L, built by the whole block (no barrier inside)
__device__ __forceinline__ void build_roots(float2* tab, int L, float sign) {
  for (int i = threadIdx.x; i < L; i += blockDim.x) tab[i] = root(i, L, sign);
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}

// ---- 1. out[m][tau][o] = sum_t exp(-2 pi i tau t / T) in[m][t][o] ---------------------------------
__global__ void k_dft_time(const float2* __restrict__ in, float2* __restrict__ out, int T) {
  __shared__ float2 tw[64];
  for (int i = threadIdx.x; i < T; i += blockDim.x) tw[i] = root(i, T, -1.f);
  __syncthreads();
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t m = blockIdx.y;
  if (o >= OM) return;
  const float2* src = in + m * T * OM + o;
  for (int tau = 0; tau < T; ++tau) {
    float2 s = make_float2(0.f, 0.f);
    int ph = 0;
    for (int t = 0; t < T; ++t) {
      s = cfma(src[(size_t)t * OM], tw[ph], s);
      ph += tau;
      if (ph >= T) ph -= T;
    }
    out[(m * T + tau) * OM + o] = s;
  }
}

// ---- 3. partial inverse DFTs of a frequency-major spectrum set --------------------------------
// gT[(tau * OM + kh * 65 + kw) * np + p]; per time frequency tau and item p:
//   U[tau][p][ha][wb] = sum_kh e^{2 pi i kh (ha - offa) / H} sum_kw c(kw) gT[..] e^{2 pi i kw (wb - offb) / W}
struct RowsArgs {
  const float2* gT;
  int np, T, La, Lb, offa, offb;
  float2* U;           // [T][np][La * Lb]
  const float2* tab;   // [Wc][Lb] c(kw) e^{2 pi i kw (wb - offb) / W}, then [H][La] e^{2 pi i kh (ha - offa) / H}
};

__global__ void k_vl_tables(RowsArgs a, float2* tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Wc * a.Lb) {
    const int kw = i / a.Lb, wi = i - kw * a.Lb;
    const float2 r = root((long long)kw * (wi - a.offb), W, 1.f);
    const float wt = (kw == 0 || 2 * kw == W) ? 1.f : 2.f;
    tab[i] = make_float2(wt * r.x, wt * r.y);
  } else if (i < Wc * a.Lb + H * a.La) {
    const int j = i - Wc * a.Lb;
    const int kh = j / a.La, hi = j - kh * a.La;
    tab[i] = root((long long)kh * (hi - a.offa), H, 1.f);
  }
}

__global__ void __launch_bounds__(kRowsNT) k_vl_rows(RowsArgs a) {
  extern __shared__ float2 sm[];
  float2* e1 = sm;                       // [Wc][Lb]
  float2* e2 = e1 + Wc * a.Lb;           // [H][La]
  float2* ring = e2 + H * a.La;          // [kRowsStages][Wc][kRowsPairs]
  for (int i = threadIdx.x; i < Wc * a.Lb + H * a.La; i += kRowsNT) e1[i] = a.tab[i];   // e1 then e2
  const int tau = blockIdx.y;
  const int p0 = blockIdx.x * kRowsPairs;
  const int q = threadIdx.x / kRowsSub, sub = threadIdx.x % kRowsSub;
  const int tile = Wc * kRowsPairs;
  auto issue = [&](int kh) {
    if (kh < H) {
      float2* dst = ring + (kh % kRowsStages) * tile;
      const float2* src = a.gT + ((size_t)tau * OM + (size_t)kh * Wc) * a.np + p0;
      for (int i = threadIdx.x; i < tile; i += kRowsNT) {
        const int kw = i / kRowsPairs, qq = i - kw * kRowsPairs;
        const bool v = p0 + qq < a.np;
        cp_async8(dst + i, src + (size_t)kw * a.np + (v ? qq : 0), v);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  for (int r = 0; r < kRowsStages - 1; ++r) issue(r);
  float2 acc[2][kMaxL];
#pragma unroll
  for (int w = 0; w < 2; ++w)
#pragma unroll
    for (int h = 0; h < kMaxL; ++h) acc[w][h] = make_float2(0.f, 0.f);
  for (int kh = 0; kh < H; ++kh) {
    issue(kh + kRowsStages - 1);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kRowsStages - 1) : "memory");
    __syncthreads();
    const float2* g = ring + (kh % kRowsStages) * tile + q;
    float2 t[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    for (int kw = 0; kw < Wc; ++kw) {
      const float2 gv = g[kw * kRowsPairs];
      const float2* e = e1 + kw * a.Lb + sub;
#pragma unroll
      for (int w = 0; w < 2; ++w)
        if (sub + kRowsSub * w < a.Lb) t[w] = cfma(gv, e[kRowsSub * w], t[w]);
    }
    const float2* e = e2 + kh * a.La;
#pragma unroll
    for (int w = 0; w < 2; ++w)
#pragma unroll
      for (int h = 0; h < kMaxL; ++h)
        if (h < a.La) acc[w][h] = cfma(t[w], e[h], acc[w][h]);
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  const int p = p0 + q;
  if (p >= a.np) return;
  const int LL = a.La * a.Lb;
  float2* out = a.U + ((size_t)tau * a.np + p) * LL;
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    const int wi = sub + kRowsSub * w;
    if (wi >= a.Lb) continue;
#pragma unroll
    for (int h = 0; h < kMaxL; ++h)
      if (h < a.La) out[h * a.Lb + wi] = acc[w][h];
  }
}

// The same partial inverse DFTs with the per-frequency products formed on the fly from the 3-D
// spectra instead of read from a materialised Gram (for the video workload the Gram is [T x 8320
// frequencies][2080 pairs]: 4.4 GB written and read again): per (tau, kh) the block stages the rows
// z_hat_nk(tau, kh, .) it needs (the distinct k of its items, all n) and forms
//     g[kw][q] = sum_n conj(A_nq(tau, kh, kw)) B_nq(tau, kh, kw)
// with (A, B) = (z_hat_k, z_hat_k') for the pair items of the lag window (column order
// k'(k'+1)/2 + k, mode 0) or (z_hat_k, x_hat_j) for the right-hand-side items k J + j (mode 1).
// The first partial DFT pairs the outputs w = offb + m and offb - m: with g = gr + i gi and
// e = c(kw) e^{2 pi i kw m / W} = ec + i es, the four sums of gr ec, gi es, gr es, gi ec give both,
//     T(+m) = (A - B) + i (C + D),   T(-m) = (A + B) + i (D - C),
// so a thread (item q, m = sub) does four FMAs and two shared-memory reads per kw for two outputs.
struct RowsZArgs {
  const float2* z3;    // [N][K][T][OM]
  const float2* x3;    // [N][J][T][OM]
  int N, K, J, np, T, La, Lb, offa, offb, mode;
  int ns, ni;          // threads per item (m = 0 .. ns - 1), items per block
  float2* U;           // [T][np][La * Lb]
  const float2* tab;   // as RowsArgs
};
// items per block, staged rows (each item needs at most two), ring depth; the twiddles of both partial
// DFTs come from one 128-entry table (H = W = 128): 41 KB of shared memory for one video, four blocks
// per SM
constexpr int kRowsZMaxN = 2, kRowsZItems = 11, kRowsZRows = 2 * kRowsZItems, kRowsZStages = 3;

__host__ __device__ inline size_t rowsz_smem(int N) {
  return ((size_t)W + (size_t)kRowsZStages * kRowsZRows * N * Wc + (size_t)Wc * kRowsZItems) * sizeof(float2);
}

__global__ void __launch_bounds__(kRowsNT, 4) k_vl_rows_z(RowsZArgs a) {
  extern __shared__ float2 sm[];
  __shared__ const float2* rowp[kRowsZRows];   // row r: its map at n = 0 (tau and kh added per stage)
  __shared__ size_t rown[kRowsZRows];          // row r: the map stride of n
  __shared__ int qa[kRowsZItems], qb[kRowsZItems], s_nr;
  float2* w128 = sm;                                // e^{2 pi i m / 128}
  float2* ring = w128 + W;                          // [kRowsZStages][nr][N][Wc]
  float2* gt = ring + kRowsZStages * kRowsZRows * a.N * Wc;   // [Wc][ni]
  for (int i = threadIdx.x; i < W; i += kRowsNT) w128[i] = root(i, W, 1.f);
  const int tau = blockIdx.y, ni = a.ni, ns = a.ns;
  const int p0 = blockIdx.x * ni;
  const size_t map = (size_t)a.T * OM;
  if (threadIdx.x == 0) {   // the distinct rows of the block's items
    int nr = 0;
    auto slot = [&](const float2* base, size_t nstride) {
      for (int r = 0; r < nr; ++r)
        if (rowp[r] == base) return r;
      rowp[nr] = base;
      rown[nr] = nstride;
      return nr++;
    };
    for (int q = 0; q < ni; ++q) {
      const int p = min(p0 + q, a.np - 1);
      if (a.mode == 0) {
        int kp = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
        while (kp * (kp + 1) / 2 > p) --kp;
        while ((kp + 1) * (kp + 2) / 2 <= p) ++kp;
        qa[q] = slot(a.z3 + (size_t)(p - kp * (kp + 1) / 2) * map, (size_t)a.K * map);
        qb[q] = slot(a.z3 + (size_t)kp * map, (size_t)a.K * map);
      } else {
        const int k = p / a.J;
        qa[q] = slot(a.z3 + (size_t)k * map, (size_t)a.K * map);
        qb[q] = slot(a.x3 + (size_t)(p - k * a.J) * map, (size_t)a.J * map);
      }
    }
    s_nr = nr;
  }
  __syncthreads();
  const int nr = s_nr, NW = a.N * Wc, stage = nr * NW;
  const int q = threadIdx.x / ns, sub = threadIdx.x - q * ns;
  const bool live = q < ni;
  const int wp = a.offb + sub, wm = a.offb - sub;   // the thread's outputs w = offb + m, offb - m
  const bool hp = live && wp < a.Lb, hm = live && sub > 0 && wm >= 0;
  auto issue = [&](int kh) {
    if (kh < H) {
      float2* dst = ring + (kh % kRowsZStages) * kRowsZRows * NW;
      const size_t off = (size_t)tau * OM + (size_t)kh * Wc;
      for (int i = threadIdx.x; i < stage; i += kRowsNT) {
        const int r = i / NW, rem = i - r * NW, n = rem / Wc, kw = rem - n * Wc;
        cp_async8(dst + i, rowp[r] + n * rown[r] + off + kw, true);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  for (int r = 0; r < kRowsZStages - 1; ++r) issue(r);
  float2 acc[2][kMaxL];
#pragma unroll
  for (int w = 0; w < 2; ++w)
#pragma unroll
    for (int h = 0; h < kMaxL; ++h) acc[w][h] = make_float2(0.f, 0.f);
  for (int kh = 0; kh < H; ++kh) {
    issue(kh + kRowsZStages - 1);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kRowsZStages - 1) : "memory");
    __syncthreads();
    const float2* rs = ring + (kh % kRowsZStages) * kRowsZRows * NW;
    for (int i = threadIdx.x; i < Wc * ni; i += kRowsNT) {   // g[kw][qq], n in order
      const int kw = i / ni, qq = i - kw * ni;
      const float2* A = rs + qa[qq] * NW + kw;
      const float2* B = rs + qb[qq] * NW + kw;
      float2 g = make_float2(0.f, 0.f);
      for (int n = 0; n < a.N; ++n) g = cfmac(A[n * Wc], B[n * Wc], g);
      gt[i] = g;
    }
    __syncthreads();
    if (live) {
      const float2* g = gt + q;
      // c(kw) e^{2 pi i kw m / W} (c = 1 at kw = 0 and W / 2, else 2)
      float sA = 0.f, sB = 0.f, sC = 0.f, sD = 0.f;
      int m = 0;
      for (int kw = 0; kw < Wc; ++kw) {
        const float2 gv = g[kw * ni];
        const float cw = (kw == 0 || 2 * kw == W) ? 1.f : 2.f;
        const float2 ev = make_float2(cw * w128[m].x, cw * w128[m].y);
        m = (m + sub) & (W - 1);
        sA = fmaf(gv.x, ev.x, sA);
        sB = fmaf(gv.y, ev.y, sB);
        sC = fmaf(gv.x, ev.y, sC);
        sD = fmaf(gv.y, ev.x, sD);
      }
      const float2 t[2] = {make_float2(sA - sB, sC + sD), make_float2(sA + sB, sD - sC)};
      // e^{2 pi i kh (h - offa) / H}
      int m2 = (int)(((long long)kh * (H - a.offa)) & (H - 1));
#pragma unroll
      for (int h = 0; h < kMaxL; ++h)
        if (h < a.La) {
          const float2 e = w128[m2];
          m2 = (m2 + kh) & (H - 1);
#pragma unroll
          for (int w = 0; w < 2; ++w) acc[w][h] = cfma(t[w], e, acc[w][h]);
        }
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  const int p = p0 + q;
  if (!live || p >= a.np) return;
  const int LL = a.La * a.Lb;
  float2* out = a.U + ((size_t)tau * a.np + p) * LL;
#pragma unroll
  for (int h = 0; h < kMaxL; ++h) {
    if (h >= a.La) continue;
    if (hp) out[h * a.Lb + wp] = acc[0][h];
    if (hm) out[h * a.Lb + wm] = acc[1][h];
  }
}

// block shape of k_vl_rows_z for an output window of Lb columns around offb
static void rowsz_shape(int Lb, int offb, int& ns, int& ni) {
  ns = std::max(offb, Lb - 1 - offb) + 1;
  ni = std::min(kRowsZItems, kRowsNT / ns);
}

// C(ti, i) = (1/D) sum_tau Re(U[tau][p][i] e^{2 pi i tau (ti - offt) / T}); the same operations in the
// same order for every (p, ti, i), so C(tau) is bitwise the same whichever thread forms it
__device__ __forceinline__ float time_sum(const float2* U, const float2* twT, int np, int LL, int T, int p, int i,
                                          int ti, int offt, float invD) {
  float s = 0.f;
  const int step = imod(ti - offt, T);
  int m = 0;
  for (int tau = 0; tau < T; ++tau) {
    const float2 u = U[((size_t)tau * np + p) * LL + i];
    const float2 e = twT[m];
    s = fmaf(u.x, e.x, fmaf(-u.y, e.y, s));
    m += step;
    if (m >= T) m -= T;
  }
  return s * invD;
}

struct TimeArgs {
  const float2* U;
  int np, T, Lt, LL, offt, K, J;
  float invD;
  int lags;        // 1: pairs in column order k'(k'+1)/2 + k -> lags [K][K][Lt][LL]; 0: items k J + j -> out [K J][Lt][LL]
  float* out;
};

__global__ void k_vl_time(TimeArgs a) {
  __shared__ float2 twT[64];   // exp(+2 pi i m / T)
  build_roots(twT, a.T, 1.f);
  __syncthreads();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)a.np * a.LL) return;
  const int p = (int)(e / a.LL), i = (int)(e - (long long)p * a.LL);
  const int LLL = a.Lt * a.LL;
  if (!a.lags) {
    for (int ti = 0; ti < a.Lt; ++ti)
      a.out[(size_t)p * LLL + ti * a.LL + i] = time_sum(a.U, twT, a.np, a.LL, a.T, p, i, ti, a.offt, a.invD);
    return;
  }
  int kp = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
  while (kp * (kp + 1) / 2 > p) --kp;
  while ((kp + 1) * (kp + 2) / 2 <= p) ++kp;
  const int k = p - kp * (kp + 1) / 2;
  float* outp = a.out + ((size_t)k * a.K + kp) * LLL;
  float* outT = a.out + ((size_t)kp * a.K + k) * LLL;
  for (int ti = 0; ti < a.Lt; ++ti) {
    const float v = time_sum(a.U, twT, a.np, a.LL, a.T, p, i, ti, a.offt, a.invD);
    const int idx = ti * a.LL + i;
    if (k == kp) {
      // C_kk(tau) = C_kk(-tau): the writers of tau and -tau add the same two values
      const float m = time_sum(a.U, twT, a.np, a.LL, a.T, p, a.LL - 1 - i, a.Lt - 1 - ti, a.offt, a.invD);
      outp[idx] = 0.5f * (v + m);
    } else {
      outp[idx] = v;
      outT[LLL - 1 - idx] = v;   // C_k'k(tau) = C_kk'(-tau)
    }
  }
}

// ---- 4. lag spectra: C_hat(f) = sum_tau C(tau) e^{-2 pi i f . tau / L} / (Lt La Lb), f in
// [Lt][La][fw] (half spectrum along the last axis), one block per pair k <= k' -----------------
struct SpecArgs {
  const float* lags;   // [K][K][Lt][La][Lb]
  int K, Lt, La, Lb, fw, ft, fh;
  float2* chat;        // [NF][K][K]: [f][k'][k] = C_hat_kk'(f) (both triangles, the input filter k' major)
};

__global__ void __launch_bounds__(256) k_vl_lagspec(SpecArgs a) {
  extern __shared__ float2 ss[];
  const int Lt = a.Lt, La = a.La, Lb = a.Lb, fw = a.fw;
  float* C = reinterpret_cast<float*>(ss);                 // [Lt][La][Lb]
  float2* R1 = ss + (Lt * La * Lb + 1) / 2;                // [Lt][La][fw]
  float2* R2 = R1 + Lt * La * fw;                          // [Lt][La][fw]
  float2* tb_ = R2 + Lt * La * fw;                         // exp(-2 pi i m / Lb), / La, / Lt
  float2* ta_ = tb_ + Lb;
  float2* tt_ = ta_ + La;
  build_roots(tb_, Lb, -1.f);
  build_roots(ta_, La, -1.f);
  build_roots(tt_, Lt, -1.f);
  int k = 0, rem = blockIdx.x;
  while (rem >= a.K - k) { rem -= a.K - k; ++k; }
  const int kp = k + rem;
  const float* src = a.lags + ((size_t)k * a.K + kp) * Lt * La * Lb;
  for (int i = threadIdx.x; i < Lt * La * Lb; i += blockDim.x) C[i] = src[i];
  __syncthreads();
  for (int e = threadIdx.x; e < Lt * La * fw; e += blockDim.x) {
    const int w2 = e % fw, row = e / fw;
    float2 s = make_float2(0.f, 0.f);
    for (int tb = 0; tb < Lb; ++tb) {
      const float2 r = tb_[imod(w2 * (tb - (a.fw - 1)), Lb)];
      const float cv = C[row * Lb + tb];
      s.x = fmaf(cv, r.x, s.x);
      s.y = fmaf(cv, r.y, s.y);
    }
    R1[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < Lt * La * fw; e += blockDim.x) {
    const int w2 = e % fw, w1 = (e / fw) % La, tt = e / (fw * La);
    float2 s = make_float2(0.f, 0.f);
    for (int ta = 0; ta < La; ++ta) s = cfma(R1[(tt * La + ta) * fw + w2], ta_[imod(w1 * (ta - (a.fh - 1)), La)], s);
    R2[e] = s;
  }
  __syncthreads();
  const int K = a.K;
  const float sc = 1.0f / (float)(Lt * La * Lb);
  for (int e = threadIdx.x; e < Lt * La * fw; e += blockDim.x) {
    const int w2 = e % fw, w1 = (e / fw) % La, w0 = e / (fw * La);
    float2 s = make_float2(0.f, 0.f);
    for (int tt = 0; tt < Lt; ++tt) s = cfma(R2[(tt * La + w1) * fw + w2], tt_[imod(w0 * (tt - (a.ft - 1)), Lt)], s);
    s = cscale(s, sc);
    float2* cf = a.chat + (size_t)e * K * K;
    cf[(size_t)kp * K + k] = s;                                      // C_hat_kk'
    if (kp != k) cf[(size_t)k * K + kp] = make_float2(s.x, -s.y);    // C_hat_k'k = conj C_hat_kk'
  }
}

// ---- 5. CG operator on the lag grid ----------------------------------------------------------
struct OpArgs {
  int K, J, ft, fh, fw, Lt, La, Lb, S3, NF;
  const float* p;      // [K][J][S3] taps (qt, qa, qb)
  float2* phat;        // [K][J][NF]
  float2* yhat;        // [K][J][NF]
  float* y;            // [K][J][S3]
  const float2* chat;  // [NF][K][K], [f][k'][k] = C_hat_kk'(f)
  const int* done;     // all channels converged: skip
  // inside CG iterations (null otherwise): k_vl_t2b first forms p <- beta_j p + z on its (k, j) and
  // stores it (the direction update of the previous iteration); k_vl_b2t forms the (k, j) partial of
  // p . Ap with Ap = y + 2 mu_k p
  float* pw;
  const float* zv;
  const float* beta;   // [kMaxJ]
  const int* active;   // [K]
  const float* fscal;  // [2][K]: 2 mu_k, Jacobi inverse
  double* pap;         // [K][J]
};

// p_hat(f) = sum_q p(q) e^{-2 pi i (w0 qt / Lt + w1 qa / La + w2 qb / Lb)}, separable, one block per (k, j)
__global__ void __launch_bounds__(256) k_vl_t2b(OpArgs a) {
  if (a.done && *a.done) return;
  extern __shared__ float2 so[];
  const int ft = a.ft, fh = a.fh, fw = a.fw, La = a.La, Lt = a.Lt;
  float* P = reinterpret_cast<float*>(so);           // [ft][fh][fw]
  float2* Q1 = so + (a.S3 + 1) / 2;                  // [ft][fh][fw']  (w2 < fw)
  float2* Q2 = Q1 + ft * fh * fw;                    // [ft][La][fw]
  float2* tb_ = Q2 + ft * La * fw;                   // exp(-2 pi i m / Lb), / La, / Lt
  float2* ta_ = tb_ + a.Lb;
  float2* tt_ = ta_ + La;
  build_roots(tb_, a.Lb, -1.f);
  build_roots(ta_, La, -1.f);
  build_roots(tt_, Lt, -1.f);
  const size_t kj = blockIdx.x;
  if (a.pw) {
    const int j = (int)(kj % a.J);
    const bool act = a.active[kj / a.J] != 0;
    const float bj = a.beta[j];
    for (int i = threadIdx.x; i < a.S3; i += blockDim.x) {
      const size_t q = kj * a.S3 + i;
      float pv = a.pw[q];
      if (act) {
        pv = fmaf(bj, pv, a.zv[q]);
        a.pw[q] = pv;
      }
      P[i] = pv;
    }
  } else {
    for (int i = threadIdx.x; i < a.S3; i += blockDim.x) P[i] = a.p[kj * a.S3 + i];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ft * fh * fw; e += blockDim.x) {
    const int w2 = e % fw, row = e / fw;
    float2 s = make_float2(0.f, 0.f);
    for (int qb = 0; qb < fw; ++qb) {
      const float2 r = tb_[(w2 * qb) % a.Lb];
      const float pv = P[row * fw + qb];
      s.x = fmaf(pv, r.x, s.x);
      s.y = fmaf(pv, r.y, s.y);
    }
    Q1[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ft * La * fw; e += blockDim.x) {
    const int w2 = e % fw, w1 = (e / fw) % La, qt = e / (fw * La);
    float2 s = make_float2(0.f, 0.f);
    for (int qa = 0; qa < fh; ++qa) s = cfma(Q1[(qt * fh + qa) * fw + w2], ta_[(w1 * qa) % La], s);
    Q2[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < a.NF; e += blockDim.x) {
    const int w2 = e % fw, w1 = (e / fw) % La, w0 = e / (fw * La);
    float2 s = make_float2(0.f, 0.f);
    for (int qt = 0; qt < ft; ++qt) s = cfma(Q2[(qt * La + w1) * fw + w2], tt_[(w0 * qt) % Lt], s);
    a.phat[kj * a.NF + e] = s;
  }
}

// y_hat_kj(f) = sum_k' C_hat_kk'(f) p_hat_k'j(f); the lanes of a warp share the bin (p_hat loads are
// broadcasts) and take consecutive filters (C_hat loads are contiguous: [f][k'][k])
__global__ void k_vl_prod(OpArgs a) {
  if (a.done && *a.done) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)a.NF * a.K) return;
  const int f = (int)(e / a.K), k = (int)(e - (long long)f * a.K);
  const int K = a.K, J = a.J;
  const float2* __restrict__ cf = a.chat + (size_t)f * K * K + k;
  const float2* __restrict__ ph = a.phat + f;
  float2 acc[kMaxJ];
#pragma unroll
  for (int j = 0; j < kMaxJ; ++j) acc[j] = make_float2(0.f, 0.f);
#pragma unroll 8
  for (int kp = 0; kp < K; ++kp) {
    const float2 c = __ldg(cf + (size_t)kp * K);
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j)
      if (j < J) acc[j] = cfma(c, __ldg(ph + ((size_t)kp * J + j) * a.NF), acc[j]);
  }
#pragma unroll
  for (int j = 0; j < kMaxJ; ++j)
    if (j < J) a.yhat[((size_t)k * J + j) * a.NF + f] = acc[j];
}

// y(q) = sum_f wt(w2) Re(y_hat(f) e^{+2 pi i (w0 qt / Lt + w1 qa / La + w2 qb / Lb)}), one block per (k, j)
__global__ void __launch_bounds__(256) k_vl_b2t(OpArgs a) {
  if (a.done && *a.done) return;
  extern __shared__ float2 so[];
  const int ft = a.ft, fh = a.fh, fw = a.fw, La = a.La, Lt = a.Lt;
  float2* Y = so;                        // [Lt][La][fw]
  float2* Q2 = Y + a.NF;                 // [ft][La][fw]
  float2* Q1 = Q2 + ft * La * fw;        // [ft][fh][fw]
  float2* tb_ = Q1 + ft * fh * fw;       // exp(+2 pi i m / Lb), / La, / Lt
  float2* ta_ = tb_ + a.Lb;
  float2* tt_ = ta_ + La;
  build_roots(tb_, a.Lb, 1.f);
  build_roots(ta_, La, 1.f);
  build_roots(tt_, Lt, 1.f);
  const size_t kj = blockIdx.x;
  for (int i = threadIdx.x; i < a.NF; i += blockDim.x) Y[i] = a.yhat[kj * a.NF + i];
  __syncthreads();
  for (int e = threadIdx.x; e < ft * La * fw; e += blockDim.x) {
    const int w2 = e % fw, w1 = (e / fw) % La, qt = e / (fw * La);
    float2 s = make_float2(0.f, 0.f);
    for (int w0 = 0; w0 < Lt; ++w0) s = cfma(Y[(w0 * La + w1) * fw + w2], tt_[(w0 * qt) % Lt], s);
    Q2[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ft * fh * fw; e += blockDim.x) {
    const int w2 = e % fw, qa = (e / fw) % fh, qt = e / (fw * fh);
    float2 s = make_float2(0.f, 0.f);
    for (int w1 = 0; w1 < La; ++w1) s = cfma(Q2[(qt * La + w1) * fw + w2], ta_[(w1 * qa) % La], s);
    Q1[e] = s;
  }
  __syncthreads();
  double pap = 0.0;
  const int k = (int)(kj / a.J);
  const bool act = a.pap && a.active[k];
  const float mu2 = a.pap ? a.fscal[k] : 0.f;
  for (int e = threadIdx.x; e < a.S3; e += blockDim.x) {
    const int qb = e % fw, row = e / fw;
    float s = 0.f;
    for (int w2 = 0; w2 < fw; ++w2) {
      const float2 v = Q1[row * fw + w2];
      const float2 r = tb_[(w2 * qb) % a.Lb];
      s = fmaf(w2 == 0 ? 1.f : 2.f, v.x * r.x - v.y * r.y, s);
    }
    a.y[kj * a.S3 + e] = s;
    if (act) {
      const float pv = a.pw[kj * a.S3 + e];
      pap += (double)pv * (s + mu2 * pv);
    }
  }
  if (a.pap) {   // block sum in a fixed order: warps, then warp totals in warp order
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) pap += __shfl_down_sync(0xffffffffu, pap, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = pap;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      a.pap[kj] = t;
    }
  }
}

// ---- CG vectors and scalars: one block ---------------------------------------------------------
struct CgState {
  double rz[kMaxJ], rr[kMaxJ], bb[kMaxJ];
  int done_j[kMaxJ];
  int done;     // every channel converged
  int iters;    // iterations of the current step
};

struct VecArgs {
  int K, J, S3, cg_max;
  double tol2, mu_floor;
  const float* b;      // [K][J][S3]
  float* x;            // [K][J][S3] the filters (warm start, solution)
  float* r;
  float* z;
  float* p;
  const float* y;      // operator output (C part) for the vector the step applied it to
  double* mu;          // [K]
  const float* lags;   // [K][K][LLL]: C_kk at the zero lag
  int zero_lag;        // index of the zero lag in a [Lt][La][Lb] window
  int LLL;
  const int* active;   // [K]
  float* fscal;        // [2][K]: 2 mu_k and the Jacobi inverse 1 / (C_kk(0) + 2 mu_k) (0 if inactive), float
  CgState* st;
  int* iters_out;      // [steps]
  int step;
};

template <int N>
__device__ void block_sum(double (&v)[N], double* red) {
  for (int i = 0; i < N; ++i) {
    double s = v[i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[(threadIdx.x >> 5) * N + i] = s;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    double s = 0.0;
    for (int w = 0; w < kCgNT / 32; ++w) s += red[w * N + threadIdx.x];
    red[kCgNT / 32 * N + threadIdx.x] = s;
  }
  __syncthreads();
  for (int i = 0; i < N; ++i) v[i] = red[kCgNT / 32 * N + i];
  __syncthreads();
}

// (the per-filter float scalars of a step are formed once per filter in float64 and stored as floats:
// the device's float64 rate is low, so no element of the vector loops touches float64 arithmetic)
// phase 0: the step's scalars; r = b - (y + 2 mu x) with y = C x, z = M^-1 r, p = z; rz, rr, bb
__global__ void __launch_bounds__(kCgNT) k_vl_cg_init(VecArgs a) {
  __shared__ double red[(kCgNT / 32 + 1) * 3 * kMaxJ];
  __shared__ float s2mu[128], sinv[128];
  for (int k = threadIdx.x; k < a.K; k += kCgNT) {
    const double c0 = (double)a.lags[((size_t)k * a.K + k) * a.LLL + a.zero_lag];
    s2mu[k] = a.fscal[k] = (float)(2.0 * a.mu[k]);
    sinv[k] = a.fscal[a.K + k] = a.active[k] ? (float)(1.0 / (c0 + 2.0 * a.mu[k])) : 0.f;
  }
  __syncthreads();
  const int JS = a.J * a.S3, n = a.K * JS;
  double s[3 * kMaxJ] = {};
  for (int i = threadIdx.x; i < n; i += kCgNT) {
    const int k = i / JS, j = (i - k * JS) / a.S3;
    if (!a.active[k]) { a.r[i] = a.z[i] = a.p[i] = 0.f; continue; }
    const float rv = a.b[i] - (a.y[i] + s2mu[k] * a.x[i]);
    const float zv = rv * sinv[k];
    a.r[i] = rv; a.z[i] = zv; a.p[i] = zv;
    s[j] += (double)rv * zv;
    s[kMaxJ + j] += (double)rv * rv;
    s[2 * kMaxJ + j] += (double)a.b[i] * a.b[i];
  }
  block_sum<3 * kMaxJ>(s, red);
  if (threadIdx.x == 0) {
    int all = 1;
    for (int j = 0; j < a.J; ++j) {
      a.st->rz[j] = s[j];
      a.st->rr[j] = s[kMaxJ + j];
      a.st->bb[j] = s[2 * kMaxJ + j];
      a.st->done_j[j] = !(a.st->rr[j] > a.tol2 * a.st->bb[j]) || !(a.st->rz[j] > 0.0);
      all = all && a.st->done_j[j];
    }
    a.st->done = all || a.cg_max < 1;
    a.st->iters = 0;
  }
}

// one iteration over G blocks (after y = C p), four launches: partial p . Ap per block; alpha from
// the partials (summed in block order) and the updates of x, r, z with partial r . z, r . r; the
// scalars (one block: beta, convergence, the iteration count); p = z + beta p
constexpr int kVecNT = 256;
struct IterArgs {
  VecArgs v;
  int G;
  double* part;    // [K][J]: p . Ap partials of k_vl_b2t
  double* part2;   // [G][2 kMaxJ]: r . z, r . r
  float* beta;     // [kMaxJ]
};

template <int N>
__device__ void block_sum_small(double (&v)[N], double* red) {   // kVecNT threads; result in thread 0
  for (int i = 0; i < N; ++i) {
    double s = v[i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[(threadIdx.x >> 5) * N + i] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 0; i < N; ++i) {
      double s = 0.0;
      for (int w = 0; w < kVecNT / 32; ++w) s += red[w * N + i];
      v[i] = s;
    }
}

__device__ __forceinline__ void block_range(int n, int G, int& i0, int& i1) {
  i0 = (int)((long long)blockIdx.x * n / G);
  i1 = (int)((long long)(blockIdx.x + 1) * n / G);
}

__global__ void __launch_bounds__(kVecNT) k_vl_it_upd(IterArgs a) {
  const VecArgs& v = a.v;
  if (v.st->done) return;
  __shared__ double red[(kVecNT / 32) * 2 * kMaxJ];
  __shared__ float s_alpha[kMaxJ];
  if (threadIdx.x < 32) {
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j) {
      double t = 0.0;
      if (j < v.J)
        for (int k = threadIdx.x; k < v.K; k += 32) t += a.part[k * v.J + j];   // p . Ap partials [K][J]
      for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
      if (threadIdx.x == 0)
        s_alpha[j] = (j < v.J && !v.st->done_j[j] && t > 0.0) ? (float)(v.st->rz[j] / t) : 0.f;
    }
  }
  __syncthreads();
  const int JS = v.J * v.S3, n = v.K * JS;
  int i0, i1;
  block_range(n, a.G, i0, i1);
  double s[2 * kMaxJ] = {};
  for (int i = i0 + threadIdx.x; i < i1; i += kVecNT) {
    const int k = i / JS, j = (i - k * JS) / v.S3;
    if (!v.active[k]) continue;
    const float al = s_alpha[j];
    const float pv = v.p[i];
    const float apv = v.y[i] + v.fscal[k] * pv;
    v.x[i] = fmaf(al, pv, v.x[i]);
    const float rv = fmaf(-al, apv, v.r[i]);
    v.r[i] = rv;
    const float zv = rv * v.fscal[v.K + k];
    v.z[i] = zv;
    s[j] += (double)rv * zv;
    s[kMaxJ + j] += (double)rv * rv;
  }
  block_sum_small<2 * kMaxJ>(s, red);
  if (threadIdx.x == 0)
    for (int u = 0; u < 2 * kMaxJ; ++u) a.part2[blockIdx.x * 2 * kMaxJ + u] = s[u];
}

__global__ void k_vl_it_scal(IterArgs a) {   // one warp
  const VecArgs& v = a.v;
  if (v.st->done) return;
  double sums[2 * kMaxJ];
#pragma unroll
  for (int u = 0; u < 2 * kMaxJ; ++u) {
    double t = 0.0;
    for (int g = threadIdx.x; g < a.G; g += 32) t += a.part2[g * 2 * kMaxJ + u];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    sums[u] = t;
  }
  if (threadIdx.x != 0) return;
  int all = 1;
  for (int j = 0; j < v.J; ++j) {
    const double rz = sums[j], rr = sums[kMaxJ + j];
    if (!v.st->done_j[j]) {
      a.beta[j] = v.st->rz[j] > 0.0 ? (float)(rz / v.st->rz[j]) : 0.f;
      v.st->rz[j] = rz;
      v.st->rr[j] = rr;
      v.st->done_j[j] = !(rr > v.tol2 * v.st->bb[j]) || !(rz > 0.0);
    } else {
      a.beta[j] = 0.f;
    }
    all = all && v.st->done_j[j];
  }
  v.st->iters += 1;
  v.st->done = all || v.st->iters >= v.cg_max;
}

// mu_k <- max(mu_k ||d_k||, floor) for active filters (norm over channels and taps); the step's
// iteration count; with last set, d_k <- d_k / max(1, ||d_k||) for every filter
__global__ void __launch_bounds__(kCgNT) k_vl_step_end(VecArgs a, int do_mu, int last) {
  __shared__ double sq[1];
  const int JS = a.J * a.S3;
  for (int k = 0; k < a.K; ++k) {
    double v[1] = {0.0};
    __shared__ double red[(kCgNT / 32 + 1)];
    for (int i = threadIdx.x; i < JS; i += kCgNT) {
      const double xv = a.x[(size_t)k * JS + i];
      v[0] += xv * xv;
    }
    block_sum<1>(v, red);
    if (threadIdx.x == 0) {
      const double nrm = sqrt(v[0]);
      if (do_mu && a.active[k]) a.mu[k] = fmax(a.mu[k] * nrm, a.mu_floor);
      sq[0] = nrm;
    }
    __syncthreads();
    if (last) {
      const float sc = (float)(1.0 / fmax(1.0, sq[0]));
      for (int i = threadIdx.x; i < JS; i += kCgNT) a.x[(size_t)k * JS + i] *= sc;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && do_mu && a.iters_out) a.iters_out[a.step] = a.st->iters;
}

// active[k] = any code of filter k nonzero
__global__ void k_vl_active(const float* z, long long per_filter, int N, int K, int* active) {
  const int k = blockIdx.x;
  int any = 0;
  for (int n = 0; n < N && !any; ++n) {
    const float* zk = z + ((size_t)n * K + k) * per_filter;
    for (long long i = threadIdx.x; i < per_filter; i += blockDim.x)
      if (zk[i] != 0.f) { any = 1; break; }
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) active[k] = any;
}

}  // namespace vl

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
static csc_status vl_fail(Ctx* c, csc_status s, const std::string& msg) {
  c->last_error = msg;
  return s;
}

static csc_status vl_cuda_fail(Ctx* c, cudaError_t e, const char* where) {
  return vl_fail(c, CSC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static bool vl_is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static cudaError_t vl_alloc(void** p, size_t bytes) {
  if (*p) return cudaSuccess;
  return cudaMalloc(p, std::max<size_t>(bytes, 16));
}

bool video_learn_shape_ok(const Ctx& c) {
  return 2 * c.fh - 1 <= vl::kMaxL && 2 * c.fw - 1 <= 2 * vl::kRowsSub && c.K + c.J <= 128 && c.T <= 64;
}

// x, z, d device arrays ([N][J][T][H][W], [N][K][T][H][W], [K][J][ft][fh][fw]); mu host or device;
// the steps' CG iteration counts to iters_dev ([steps], device). Synchronises the stream.
csc_status video_learn(Ctx* c, const float* x, const float* z, float* d, double* mu, int steps) {
  using namespace vl;
  VideoLearnBuffers& V = c->VL;
  const int N = c->N, K = c->K, J = c->J, T = c->T, ft = c->ft, fh = c->fh, fw = c->fw;
  const int Lt = 2 * ft - 1, La = 2 * fh - 1, Lb = 2 * fw - 1, S3 = ft * fh * fw, NF = Lt * La * fw;
  const int np = K * (K + 1) / 2, KJ = K * J;
  const size_t O3 = (size_t)T * OM;
  const size_t nvec = (size_t)KJ * S3;
  const int LLmax = La * Lb;
  const int npmax = std::max(np, KJ);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = vl_alloc(p, bytes); };
  // few videos: the per-frequency products are formed inside the partial inverse DFTs (k_vl_rows_z);
  // else the frequency-major Gram on the tensor cores and the right-hand-side spectra are materialised
  const bool fused = N <= kRowsZMaxN;
  A((void**)&V.z3, (size_t)N * K * O3 * sizeof(float2));
  A((void**)&V.x3, (size_t)N * J * O3 * sizeof(float2));
  if (!fused) {
    A((void**)&V.zt, (size_t)N * K * O3 * sizeof(float2));
    A((void**)&V.gram, O3 * np * sizeof(float2));
    A((void**)&V.rspec, (size_t)KJ * O3 * sizeof(float2));
    A((void**)&V.rspecT, (size_t)KJ * O3 * sizeof(float2));
  }
  A((void**)&V.U, (size_t)T * npmax * LLmax * sizeof(float2));
  A((void**)&V.lags, (size_t)K * K * Lt * La * Lb * sizeof(float));
  A((void**)&V.chat, (size_t)NF * K * K * sizeof(float2));
  A((void**)&V.vec, 5 * nvec * sizeof(float));
  A((void**)&V.phat, (size_t)KJ * NF * sizeof(float2));
  A((void**)&V.yhat, (size_t)KJ * NF * sizeof(float2));
  A((void**)&V.mu, (size_t)K * sizeof(double));
  A((void**)&V.active, (size_t)K * sizeof(int));
  A((void**)&V.fscal, (size_t)2 * K * sizeof(float));
  A((void**)&V.part, (size_t)(std::max(kMaxJ * c->nsm, KJ) + 2 * kMaxJ * c->nsm) * sizeof(double) +
                        kMaxJ * sizeof(float));
  A((void**)&V.st, sizeof(CgState));
  A((void**)&V.x2, (size_t)N * J * O3 * sizeof(float2));
  A((void**)&V.tab, ((size_t)Wc * 32 + (size_t)H * kMaxL) * sizeof(float2));
  if (e == cudaSuccess && steps > V.iters_cap) {
    if (V.iters) cudaFree(V.iters);
    V.iters = nullptr;
    e = cudaMalloc((void**)&V.iters, (size_t)steps * sizeof(int));
    if (e == cudaSuccess) V.iters_cap = steps;
  }
  if (e != cudaSuccess) { cudaGetLastError(); return vl_fail(c, CSC_ERR_WORKSPACE, "csc_learn: video workspace allocation failed"); }
  float* b = V.vec;
  float* r = b + nvec;
  float* zz = r + nvec;
  float* pvec = zz + nvec;
  float* y = pvec + nvec;
  cudaStream_t st = c->stream;
#define VL_CHECK(call, what)                          \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return vl_cuda_fail(c, e_, what); \
  } while (0)
  // 1. 3-D spectra: per frame, then along time
  VL_CHECK(launch_code_spectra(*c, z, N * K * T, c->vS), "code frame spectra");
  dim3 gt((OM + 127) / 128, N * K);
  k_dft_time<<<gt, 128, 0, st>>>(c->vS, V.z3, T);
  VL_CHECK(cudaGetLastError(), "time DFT");
  VL_CHECK(launch_code_spectra(*c, x, N * J * T, V.x2), "image frame spectra");
  dim3 gx((OM + 127) / 128, N * J);
  k_dft_time<<<gx, 128, 0, st>>>(V.x2, V.x3, T);
  VL_CHECK(cudaGetLastError(), "time DFT");
  // 2. frequency-major codes and the Gram over the 3-D frequencies
  if (!fused) {
    Ctx v = *c;
    v.g.Omega = (int)O3;
    v.L.zhat = V.z3;
    v.L.zt = V.zt;
    v.L.gram = V.gram;
    v.xhat = V.x3;
    VL_CHECK(launch_spectra_transpose(v, V.z3, N * K, V.zt), "code spectra transpose");
    VL_CHECK(launch_learn_gram_tc(v, CSC_FP32, V.rspec, c->err), "code Gram (tensor cores)");
    // right-hand-side spectra frequency-major: [O3][K J]
    Ctx vr = *c;
    vr.g.Omega = (int)O3;
    VL_CHECK(launch_spectra_transpose(vr, V.rspec, KJ, V.rspecT), "right-hand-side transpose");
  }
  // 3. lag window and right-hand side
  const size_t rsm = ((size_t)Wc * Lb + (size_t)H * La + (size_t)kRowsStages * Wc * kRowsPairs) * sizeof(float2);
  VL_CHECK(cudaFuncSetAttribute(k_vl_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm), "attribute");
  const float invD = 1.0f / (float)(O3 / Wc * W);   // 1 / (T H W)
  const size_t zsm = rowsz_smem(N);
  if (fused)
    VL_CHECK(cudaFuncSetAttribute(k_vl_rows_z, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsm), "attribute");
  {
    RowsArgs ra{V.gram, np, T, La, Lb, fh - 1, fw - 1, V.U, V.tab};
    k_vl_tables<<<(Wc * Lb + H * La + 255) / 256, 256, 0, st>>>(ra, V.tab);
    if (fused) {
      RowsZArgs rz{V.z3, V.x3, N, K, J, np, T, La, Lb, fh - 1, fw - 1, 0, 0, 0, V.U, V.tab};
      rowsz_shape(Lb, fw - 1, rz.ns, rz.ni);
      k_vl_rows_z<<<dim3((np + rz.ni - 1) / rz.ni, T), kRowsNT, zsm, st>>>(rz);
    } else {
      k_vl_rows<<<dim3((np + kRowsPairs - 1) / kRowsPairs, T), kRowsNT, rsm, st>>>(ra);
    }
    VL_CHECK(cudaGetLastError(), "lag window rows");
    TimeArgs ta{V.U, np, T, Lt, La * Lb, ft - 1, K, J, invD, 1, V.lags};
    const long long nt = (long long)np * La * Lb;
    k_vl_time<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(ta);
    VL_CHECK(cudaGetLastError(), "lag window time");
  }
  {
    RowsArgs ra{V.rspecT, KJ, T, fh, fw, (fh - 1) / 2, (fw - 1) / 2, V.U, V.tab};
    k_vl_tables<<<(Wc * fw + H * fh + 255) / 256, 256, 0, st>>>(ra, V.tab);
    if (fused) {
      RowsZArgs rz{V.z3, V.x3, N, K, J, KJ, T, fh, fw, (fh - 1) / 2, (fw - 1) / 2, 1, 0, 0, V.U, V.tab};
      rowsz_shape(fw, (fw - 1) / 2, rz.ns, rz.ni);
      k_vl_rows_z<<<dim3((KJ + rz.ni - 1) / rz.ni, T), kRowsNT, zsm, st>>>(rz);
    } else {
      k_vl_rows<<<dim3((KJ + kRowsPairs - 1) / kRowsPairs, T), kRowsNT, rsm, st>>>(ra);
    }
    VL_CHECK(cudaGetLastError(), "right-hand side rows");
    TimeArgs ta{V.U, KJ, T, ft, fh * fw, (ft - 1) / 2, K, J, invD, 0, b};
    const long long nt = (long long)KJ * fh * fw;
    k_vl_time<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(ta);
    VL_CHECK(cudaGetLastError(), "right-hand side time");
  }
  // 4. lag spectra
  {
    SpecArgs sa{V.lags, K, Lt, La, Lb, fw, ft, fh, V.chat};
    const size_t ssm = ((size_t)(Lt * La * Lb + 1) / 2 + 2 * (size_t)Lt * La * fw + Lt + La + Lb) * sizeof(float2);
    VL_CHECK(cudaFuncSetAttribute(k_vl_lagspec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm), "attribute");
    k_vl_lagspec<<<np, 256, ssm, st>>>(sa);
    VL_CHECK(cudaGetLastError(), "lag spectra");
  }
  // 5. CG steps
  VL_CHECK(cudaMemcpyAsync(V.mu, mu, K * sizeof(double), vl_is_device_ptr(mu) ? cudaMemcpyDeviceToDevice
                                                                             : cudaMemcpyHostToDevice, st), "mu copy");
  k_vl_active<<<K, 256, 0, st>>>(z, (long long)T * H * W, N, K, V.active);
  VL_CHECK(cudaGetLastError(), "activity");
  float* xdev = d;   // staged by the caller: device filters [K][J][ft][fh][fw]
  if (steps >= 0 && video_cg_applies(*c)) {
    // all learning steps in one persistent cooperative launch (video_cg.cu)
    A((void**)&V.words, video_cg_words(*c) * sizeof(unsigned long long));
    if (e != cudaSuccess) { cudaGetLastError(); return vl_fail(c, CSC_ERR_WORKSPACE, "csc_learn: video workspace allocation failed"); }
    VL_CHECK(launch_video_cg(*c, V.words, V.lags, V.chat, b, xdev, V.mu, V.active, V.iters, steps), "video CG");
    VL_CHECK(cudaMemcpyAsync(mu, V.mu, K * sizeof(double), vl_is_device_ptr(mu) ? cudaMemcpyDeviceToDevice
                                                                              : cudaMemcpyDeviceToHost, st), "mu copy");
    c->launches += 14;
    return CSC_OK;
  }
  OpArgs oa{K, J, ft, fh, fw, Lt, La, Lb, S3, NF, nullptr, V.phat, V.yhat, y, V.chat, nullptr};
  const size_t t2b_sm = ((size_t)(S3 + 1) / 2 + (size_t)ft * fh * fw + (size_t)ft * La * fw + Lt + La + Lb) * sizeof(float2);
  const size_t b2t_sm = ((size_t)NF + (size_t)ft * La * fw + (size_t)ft * fh * fw + Lt + La + Lb) * sizeof(float2);
  VL_CHECK(cudaFuncSetAttribute(k_vl_t2b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t2b_sm), "attribute");
  VL_CHECK(cudaFuncSetAttribute(k_vl_b2t, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b2t_sm), "attribute");
  auto apply_on = [&](const float* pv, const int* done, cudaStream_t s) -> cudaError_t {
    OpArgs o = oa;
    o.p = pv;
    o.done = done;
    k_vl_t2b<<<KJ, 256, t2b_sm, s>>>(o);
    k_vl_prod<<<(unsigned)(((long long)NF * K + 127) / 128), 128, 0, s>>>(o);
    k_vl_b2t<<<KJ, 256, b2t_sm, s>>>(o);
    return cudaGetLastError();
  };
  auto apply = [&](const float* pv, const int* done) { return apply_on(pv, done, st); };
  VecArgs va{K, J, S3, c->p.cg_max, c->p.cg_tol * c->p.cg_tol, kMuFloor, b, xdev, r, zz, pvec, y, V.mu, V.lags,
             ((ft - 1) * La + (fh - 1)) * Lb + (fw - 1), Lt * La * Lb, V.active, V.fscal,
             reinterpret_cast<CgState*>(V.st), V.iters, 0};
  int* done_dev = &reinterpret_cast<CgState*>(V.st)->done;
  IterArgs ia;
  ia.v = va;
  ia.G = (int)std::max<size_t>(1, std::min<size_t>((size_t)c->nsm, (nvec + kVecNT - 1) / kVecNT));
  const size_t part1 = (size_t)std::max(kMaxJ * c->nsm, KJ);
  ia.part = V.part;
  ia.part2 = V.part + part1;
  ia.beta = reinterpret_cast<float*>(V.part + part1 + (size_t)2 * kMaxJ * c->nsm);
  // one CG iteration; none of its kernels reads the step index, so a batch of kBatch iterations is
  // recorded once per call as a CUDA graph (on a private stream) and replayed between the host's
  // reads of the convergence flag
  constexpr int kBatch = 8;
  // an iteration: (p <- beta p + z, then the operator on p, with the p . Ap partials), the x, r, z
  // updates with their partial sums, the scalars
  OpArgs ob = oa;
  ob.p = pvec;
  ob.done = done_dev;
  ob.pw = pvec;
  ob.zv = zz;
  ob.beta = ia.beta;
  ob.active = V.active;
  ob.fscal = V.fscal;
  ob.pap = ia.part;
  auto iteration_on = [&](cudaStream_t s) -> cudaError_t {
    k_vl_t2b<<<KJ, 256, t2b_sm, s>>>(ob);
    k_vl_prod<<<(unsigned)(((long long)NF * K + 127) / 128), 128, 0, s>>>(ob);
    k_vl_b2t<<<KJ, 256, b2t_sm, s>>>(ob);
    k_vl_it_upd<<<ia.G, kVecNT, 0, s>>>(ia);
    k_vl_it_scal<<<1, 32, 0, s>>>(ia);
    return cudaGetLastError();
  };
  struct GraphGuard {
    cudaGraphExec_t g = nullptr;
    ~GraphGuard() { if (g) cudaGraphExecDestroy(g); }
  } guard;
  cudaGraphExec_t& batch_graph = guard.g;
  if (c->p.cg_max >= kBatch && steps > 0) {
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      c->cap_stream = nullptr;
    }
    cudaGraph_t gr = nullptr;
    if (c->cap_stream && cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t e = cudaSuccess;
      for (int u = 0; u < kBatch && e == cudaSuccess; ++u) e = iteration_on(c->cap_stream);
      const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &gr);
      if (e != cudaSuccess || e2 != cudaSuccess || !gr || cudaGraphInstantiate(&batch_graph, gr, 0) != cudaSuccess)
        batch_graph = nullptr;
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
    }
  }
  for (int s = 0; s < steps; ++s) {
    va.step = s;
    ia.v = va;
    VL_CHECK(apply(xdev, nullptr), "operator");
    k_vl_cg_init<<<1, kCgNT, 0, st>>>(va);
    VL_CHECK(cudaGetLastError(), "CG init");
    // the first iteration's direction update p <- 0 p + z keeps the initial p = z
    VL_CHECK(cudaMemsetAsync(ia.beta, 0, kMaxJ * sizeof(float), st), "beta reset");
    for (int it = 0; it < c->p.cg_max;) {
      const int batch = std::min(kBatch, c->p.cg_max - it);
      if (batch == kBatch && batch_graph) {
        VL_CHECK(cudaGraphLaunch(batch_graph, st), "CG iterations (graph)");
      } else {
        for (int u = 0; u < batch; ++u) VL_CHECK(iteration_on(st), "CG iteration");
      }
      it += batch;
      int hd = 0;
      VL_CHECK(cudaMemcpyAsync(&hd, done_dev, sizeof(int), cudaMemcpyDeviceToHost, st), "flag copy");
      VL_CHECK(cudaStreamSynchronize(st), "sync");
      if (hd) break;
    }
    k_vl_step_end<<<1, kCgNT, 0, st>>>(va, 1, s == steps - 1 ? 1 : 0);
    VL_CHECK(cudaGetLastError(), "step end");
  }
  if (steps == 0) {
    k_vl_step_end<<<1, kCgNT, 0, st>>>(va, 0, 1);
    VL_CHECK(cudaGetLastError(), "projection");
  }
  VL_CHECK(cudaMemcpyAsync(mu, V.mu, K * sizeof(double), vl_is_device_ptr(mu) ? cudaMemcpyDeviceToDevice
                                                                            : cudaMemcpyDeviceToHost, st), "mu copy");
#undef VL_CHECK
  c->launches += 12 + 2;
  return CSC_OK;
}

}  // namespace csc
