// Learning subproblem of Sec. 3.2 (Eqs. Learning_new .. mu_update) on the GPU.
//
// For fixed multipliers mu, Eq. Learning_new is a ridge problem in d whose dual is
// Eq. Learning_gamma; both give the same d(mu) (strong duality). The library solves the primal
// normal equations in filter space,
//     (S Z^T Z S^T + 2 diag(mu)) d = S Z^T x,
// whose matrix only involves the code cross-correlations on the (2fh-1) x (2fw-1) lag window:
//     C_kk'(tau) = sum_n sum_p z_nk(p) z_nk'(p + tau) = F^{-1}( sum_n conj(z_hat_nk) z_hat_nk' )(tau)
//     [S Z^T Z S^T d]_k(q) = sum_k' sum_q' C_kk'(q - q') d_k'(q').
// Pipeline per csc_learn call:
//   k_fft_maps          z_hat = F z for all N*K maps (coding.cu)
//   k_learn_rhs         b_kj = S F^{-1}( sum_n conj(z_hat_nk) x_hat_nj )
//   k_learn_gram        G_kk'(w) = sum_n conj(z_hat_nk(w)) z_hat_nk'(w), k <= k' (per-frequency
//                       K x N by N x K complex product)
//   k_learn_lags        C_kk' = crop of F^{-1} G_kk'
//   k_learn_cg          all learning steps in one persistent cooperative launch: Jacobi-
//                       preconditioned CG warm-started from the current d, then
//                       mu_k <- max(mu_k ||d_k||, floor) (Eq. mu_update); after the last step
//                       d_k <- d_k / max(1, ||d_k||).
#include <cuda_runtime.h>

#include <algorithm>

#include "csc_internal.cuh"
#include "cg_exchange.cuh"

namespace csc {

// ---------------------------------------------------------------------------------------------
// per-frequency Gram G_kk'(w) = sum_n conj(z_hat_nk(w)) z_hat_nk'(w), tiles of 32 frequencies x
// 16 k x 16 k' (upper tile triangle), float32 accumulation on the CUDA cores
// ---------------------------------------------------------------------------------------------
constexpr int kGramF = 32, kGramT = 16, kGramNT = 256;

struct GramArgs {
  int N, K, Omega, ntile;
  const float2* zhat;
  float2* gram;        // [npairs][Omega]
};

__device__ __forceinline__ long long pair_index(int k, int kp, int K) {
  return (long long)k * K - (long long)k * (k - 1) / 2 + (kp - k);
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}

__global__ void __launch_bounds__(kGramNT) k_learn_gram(GramArgs a) {
  // three-stage pipeline: the tiles of image n + 2 are copied (cp.async) while image n is used
  constexpr int kSt = 3;
  __shared__ __align__(16) float2 As[kSt][kGramT][kGramF];
  __shared__ __align__(16) float2 Bs[kSt][kGramT][kGramF];
  // tile pair (ti <= tj) from blockIdx.x
  int ti = 0, rem = blockIdx.x;
  while (rem >= a.ntile - ti) { rem -= a.ntile - ti; ++ti; }
  const int tj = ti + rem;
  const int o0 = blockIdx.y * kGramF;
  const int f = threadIdx.x % kGramF;
  const int grp = threadIdx.x / kGramF;   // 0..7
  const int kq = grp % 4, kpq = grp / 4;  // k rows 4kq..4kq+3, k' rows 8kpq..8kpq+7
  // this thread's share of a tile pair: elements e = threadIdx.x + 256 u of 16 x 32
  constexpr int kLd = kGramT * kGramF / kGramNT;   // 2
  int lr[kLd], lf[kLd];
  bool la[kLd], lb[kLd];
#pragma unroll
  for (int u = 0; u < kLd; ++u) {
    const int e = threadIdx.x + u * kGramNT;
    lr[u] = e / kGramF;
    lf[u] = e % kGramF;
    const int oo = o0 + lf[u];
    la[u] = (ti * kGramT + lr[u] < a.K) && oo < a.Omega;
    lb[u] = (tj * kGramT + lr[u] < a.K) && oo < a.Omega;
  }
  auto stage = [&](int n) {   // issue the copies of image n into buffer n % kSt (zero fill outside)
    const int bf = n % kSt;
#pragma unroll
    for (int u = 0; u < kLd; ++u) {
      const size_t base = (size_t)n * a.K;
      const float2* sa = la[u] ? a.zhat + (base + ti * kGramT + lr[u]) * a.Omega + o0 + lf[u] : a.zhat;
      const float2* sb = lb[u] ? a.zhat + (base + tj * kGramT + lr[u]) * a.Omega + o0 + lf[u] : a.zhat;
      cp_async8(&As[bf][lr[u]][lf[u]], sa, la[u]);
      cp_async8(&Bs[bf][lr[u]][lf[u]], sb, lb[u]);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  float2 acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) acc[i][jj] = make_float2(0.f, 0.f);
  const int o = o0 + f;
  stage(0);
  if (a.N > 1) stage(1);
  else asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int n = 0; n < a.N; ++n) {
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // image n has landed
    __syncthreads();                                          // ... for every thread; image n-1 is done
    if (n + 2 < a.N) stage(n + 2);
    else asm volatile("cp.async.commit_group;\n" ::: "memory");
    const int bf = n % kSt;
    float2 av[4], bv[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) av[i] = As[bf][4 * kq + i][f];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) bv[jj] = Bs[bf][8 * kpq + jj][f];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) acc[i][jj] = cfmac(av[i], bv[jj], acc[i][jj]);
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (o >= a.Omega) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = ti * kGramT + 4 * kq + i;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int kp = tj * kGramT + 8 * kpq + jj;
      if (k < a.K && kp < a.K && k <= kp) a.gram[pair_index(k, kp, a.K) * a.Omega + o] = acc[i][jj];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// lag spectra: the normal-equation product in the Fourier domain of the (2fh-1) x (2fw-1) lag grid
//
// For taps q, q' of an fh x fw filter the lags q - q' stay inside the La x Lb = (2fh-1) x (2fw-1)
// window, so the block Toeplitz product [S Z^T Z S^T p]_k(q) = sum_k' sum_q' C_kk'(q - q') p_k'(q')
// equals the circular correlation on the La x Lb grid, cropped to the taps:
//     y_k = crop( F^-1( sum_k' C_hat_kk' . F(p_k') ) ),   C_hat_kk' = F(C_kk') on the lag grid.
// C is real, so only the half spectrum w2 < fw is kept (NF = La * fw bins); C_hat_k'k = conj C_hat_kk'.
// chat[f][pair(k, k')] holds C_hat_kk'(f) / (La Lb) for k <= k' (pair_index order), f = w1 * fw + w2.
// ---------------------------------------------------------------------------------------------
struct LagSpecArgs {
  int K, fh, fw, La, Lb, NF;
  const float* lags;   // [K][K][La][Lb], lag (ta, tb) at ((ta + fh - 1) * Lb + tb + fw - 1)
  float2* chat;        // [NF][K(K+1)/2]
};

__device__ __forceinline__ float2 unit_root(int m, int L) {   // exp(-2 pi i m / L), 0 <= m < L
  float s, c;
  sincospif(2.0f * (float)m / (float)L, &s, &c);
  return make_float2(c, -s);
}

constexpr int kLagSpecNT = 256;

__global__ void __launch_bounds__(kLagSpecNT) k_lag_spectra(LagSpecArgs a) {
  extern __shared__ float2 ls2[];
  const int La = a.La, Lb = a.Lb, fw = a.fw, fh = a.fh, NF = a.NF, K = a.K;
  float2* R = ls2;                          // [La][fw] row transforms
  float2* twa = R + La * fw;                // [La]
  float2* twb = twa + La;                   // [Lb]
  float* C = reinterpret_cast<float*>(twb + Lb);   // [La][Lb]
  // pair (k <= kp) of this CTA
  int k = 0, rem = blockIdx.x;
  while (rem >= K - k) { rem -= K - k; ++k; }
  const int kp = k + rem;
  for (int i = threadIdx.x; i < La; i += kLagSpecNT) twa[i] = unit_root(i, La);
  for (int i = threadIdx.x; i < Lb; i += kLagSpecNT) twb[i] = unit_root(i, Lb);
  const float* src = a.lags + ((size_t)k * K + kp) * La * Lb;
  for (int i = threadIdx.x; i < La * Lb; i += kLagSpecNT) C[i] = src[i];
  __syncthreads();
  // over tb: R[ta][w2] = sum_tb C[ta][tb] exp(-2 pi i w2 (tb - fw + 1) / Lb)
  for (int e = threadIdx.x; e < La * fw; e += kLagSpecNT) {
    const int ta = e / fw, w2 = e - ta * fw;
    float2 s = make_float2(0.f, 0.f);
    for (int tb = 0; tb < Lb; ++tb) {
      const int m = ((w2 * (tb - fw + 1)) % Lb + Lb) % Lb;
      const float cv = C[ta * Lb + tb];
      s.x = fmaf(cv, twb[m].x, s.x);
      s.y = fmaf(cv, twb[m].y, s.y);
    }
    R[e] = s;
  }
  __syncthreads();
  // over ta, scaled by 1/(La Lb)
  const float sc = 1.0f / (float)(La * Lb);
  for (int f = threadIdx.x; f < NF; f += kLagSpecNT) {
    const int w1 = f / fw, w2 = f - w1 * fw;
    float2 s = make_float2(0.f, 0.f);
    for (int ta = 0; ta < La; ++ta) {
      const int m = ((w1 * (ta - fh + 1)) % La + La) % La;
      s = cfma(R[ta * fw + w2], twa[m], s);
    }
    s = cscale(s, sc);
    a.chat[(size_t)f * (K * (K + 1) / 2) + pair_index(k, kp, K)] = s;
  }
}

// ---------------------------------------------------------------------------------------------
// persistent CG over all learning steps
//
// One cooperative launch; CTA b owns the lag-grid bins [f0, f1) for the product and the filters
// k = b, b + G, ... for everything else. An iteration has two grid-wide exchanges:
//   A: after the product at its bins (y_hat to global) a CTA contributes its partial p . A p;
//   B: after x, r and z = M^-1 r of its filters (z to global) it contributes partial r . z, r . r.
// An exchange is a counter that every CTA increments with release semantics once its data (plain
// stores) and its partial sums (one slot per CTA, two banks alternating by exchange parity) are out;
// a reader polls the counter with acquire loads (bounded by the context's wait limit), then reads the
// slots and the data through L2 and sums the slots in a fixed order, so every CTA forms the same
// scalars (in float32: the device's float64 rate is a few operations per clock per SM).
// ---------------------------------------------------------------------------------------------
struct CgArgs {
  int K, J, fh, fw, S2, La, Lb, NF, G, steps, cg_max;
  double tol2, mu_floor;
  const float* lags;   // [K][K][La*Lb]: the zero lag of C_kk (activity) and the preconditioner blocks
  const float2* chat;  // [NF][K(K+1)/2] lag spectra / (La Lb), pairs k <= k'
  int chat_smem;       // the CTA's bins of chat are staged in shared memory
  float2* yv;          // [K][J][NF] y_hat, the product (written by the bins' CTAs)
  float* zv;           // [K][J][S2] z = M^-1 r (written by the filters' CTAs)
  const float* b;      // [K][J][S2]
  float* x;            // [K][J][S2]  d (in/out)
  double* mu;          // [K]
  float* slots;        // [2][G][kSlotWords] partial sums of the exchanges (bank = exchange parity)
  unsigned* arrivals;  // exchange counter: G arrivals per exchange, zeroed before the launch
  int* iters;          // [steps]
  int* err;
  long long spin;      // bound of every spin-wait, in SM clocks
};

// shared-memory layout of the CG kernel (float2 arrays first, then floats)
struct CgSmem {
  size_t ew, phat, red, yh, sc, twa, twb, cch, pp, own, total_floats;
  int nb, nown;
};
CSC_HD CgSmem cg_smem_layout(int K, int J, int S2, int NF, int fh, int fw, int La, int Lb, int NT, int G,
                             bool chat_smem) {
  CgSmem L;
  L.nb = (NF + G - 1) / G;        // bins per CTA (at most)
  L.nown = (K + G - 1) / G;       // filters per CTA (at most)
  const int red_items = L.nb * K < NT ? NT : L.nb * K;
  size_t o = 0;   // in floats
  L.ew = o;   o += 2 * (size_t)L.nb * S2;
  L.phat = o; o += 2 * (size_t)L.nb * K * J;
  L.red = o;  o += 2 * (size_t)red_items * J;
  L.yh = o;   o += 2 * (size_t)J * NF;
  L.sc = o;   o += 2 * (size_t)J * fw * fh;
  L.twa = o;  o += 2 * (size_t)La;
  L.twb = o;  o += 2 * (size_t)Lb;
  L.cch = o;  o += chat_smem ? 2 * (size_t)L.nb * (K * (K + 1) / 2) : 0;
  L.pp = o;   o += (size_t)K * J * S2;
  L.own = o;  o += 4 * (size_t)L.nown * J * S2;   // x, r, b, z of the CTA's filters
  L.total_floats = o;
  return L;
}

// dst[i] = src[i] + beta(i) * dst[i] over the whole vector, src written by other CTAs (read
// through L2); up to 24 loads per thread in flight before their use
template <int NT>
__device__ __forceinline__ void axpy_from_l2(float* dst, const float* src, int n, int JS, int S2,
                                             const double* beta, bool overwrite) {
  constexpr int U = 24;
  for (int i0 = threadIdx.x; i0 < n; i0 += U * NT) {
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = (i0 + u * NT < n) ? __ldcg(src + i0 + u * NT) : 0.f;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * NT;
      if (i < n) dst[i] = overwrite ? v[u] : fmaf((float)beta[JS == S2 ? 0 : (i % JS) / S2], dst[i], v[u]);
    }
  }
}

// thread 0: vals[0..n) into the CTA's slot of bank ep & 1, then release and count the arrival. The
// caller has synchronised the block since its data stores.
__device__ __forceinline__ void cg_arrive(const CgArgs& a, const float* vals, int n, unsigned ep) {
  if (threadIdx.x != 0) return;
  float* sl = a.slots + ((size_t)(ep & 1) * a.G + blockIdx.x) * kSlotWords;
  for (int i = 0; i < n; ++i) sl[i] = vals[i];
  asm volatile("fence.acq_rel.gpu;" ::: "memory");   // release
  atomicAdd(a.arrivals, 1u);
}

// Waits (thread 0, acquire, bounded) for the G arrivals of exchange ep, then loads the G x nw slot
// values into gv (one round trip, all threads) and forms their totals in a fixed order (one warp per
// value) into tot; then() runs on thread 0. Ends synchronised; false when the wait ran out or a CTA
// flagged an error (error word set).
template <int NT, class F>
__device__ bool cg_wait(const CgArgs& a, unsigned ep, int nw, float* gv, float* tot, int* fail, F then) {
  if (threadIdx.x == 0) {
    const unsigned target = ep * (unsigned)a.G;
    const long long t0 = clock64();
    unsigned v;
    for (;;) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a.arrivals) : "memory");
      if ((int)(v - target) >= 0) break;
      if (*(volatile int*)a.err) { *fail = 1; break; }
      if (clock64() - t0 > a.spin) {
        atomicCAS(a.err, 0, (int)CSC_ERR_TIMEOUT);
        *fail = 1;
        break;
      }
    }
  }
  __syncthreads();
  if (*fail) return false;
  const float* sb = a.slots + (size_t)(ep & 1) * a.G * kSlotWords;
  for (int i = threadIdx.x; i < a.G * nw; i += NT) gv[i] = __ldcg(sb + (size_t)(i / nw) * kSlotWords + i % nw);
  __syncthreads();
  sum_slots<NT>(gv, a.G, nw, nw, tot, then);
  return true;
}

// Lag-grid half spectrum of S Z^T Z S^T p at this CTA's bins, p (all filters) in shared memory:
// y_hat_kj(f) = sum_k' C_hat_kk'(f) p_hat_k'j(f) to a.yv (C_hat_kk' = conj C_hat_k'k for k > k'),
// and the partial Parseval sums of p . S Z^T Z S^T p over these bins (weight 2 for w2 > 0) into
// part[j]. ew[i][q] holds the tap twiddles of the CTA's bin f0 + i, cch the CTA's bins of chat (or
// null: read from global), both in pair_index order. Does not end synchronised.
template <int NT, int JT>
__device__ void product_bins(const CgArgs& a, int f0, int nbc, const float* pp, const float2* ew, float2* phat,
                             float2* red, const float2* cch, float (&part)[JT]) {
  constexpr int J = JT;
  const int K = a.K, S2 = a.S2, fw = a.fw, NF = a.NF;
  const int KJ = K * J;
  const int np = K * (K + 1) / 2;
  // p_hat of every filter at the CTA's bins: four lanes per (bin, filter, channel)
  {
    const int sub = threadIdx.x & 3;
    const int nit = nbc * KJ;
    for (int e0 = threadIdx.x >> 2; e0 < ((nit + 7) / 8) * 8; e0 += NT / 4) {
      const int e = e0 < nit ? e0 : nit - 1;
      const int bi = e / KJ, i = e - bi * KJ;
      const float* pr = pp + (size_t)i * S2;
      const float2* w = ew + (size_t)bi * S2;
      float2 s = make_float2(0.f, 0.f);
      for (int q = sub; q < S2; q += 4) {
        const float pv = pr[q];
        s.x = fmaf(pv, w[q].x, s.x);
        s.y = fmaf(pv, w[q].y, s.y);
      }
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 1);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 1);
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 2);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 2);
      if (sub == 0 && e0 < nit) phat[e] = s;
    }
  }
  __syncthreads();
  // partial products over k' ranges: item (bin, part, k). In pair_index order the entries
  // C_hat_k'k (k' < k, column k of the upper triangle) are K - k' - 1 apart, C_hat_kk' (k' >= k,
  // row k) are contiguous.
  const int PS = (nbc * K < NT) ? NT / (nbc * K) : 1;
  const int kchunk = (K + PS - 1) / PS;
  for (int e = threadIdx.x; e < nbc * PS * K; e += NT) {
    const int k = e % K, rest = e / K, pi = rest % PS, bi = rest / PS;
    const float2* cf = cch ? cch + (size_t)bi * np : a.chat + (size_t)(f0 + bi) * np;
    const float2* ph = phat + (size_t)bi * KJ;
    const int kp0 = pi * kchunk, kp1 = min(K, kp0 + kchunk);
    float2 acc[kMaxJ];
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j) acc[j] = make_float2(0.f, 0.f);
    // k' < k: conj of the stored C_hat_k'k
    const int ce = min(kp1, k);
    if (kp0 < ce) {
      int idx = kp0 * K - kp0 * (kp0 - 1) / 2 + (k - kp0);
      for (int kp = kp0; kp < ce; ++kp) {
        const float2 c = cf[idx];
        idx += K - kp - 1;
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j)
          if (j < J) acc[j] = cfmac(c, ph[kp * J + j], acc[j]);
      }
    }
    // k' >= k: the stored C_hat_kk'
    const int rs = max(kp0, k);
    if (rs < kp1) {
      const float2* row = cf + (k * K - k * (k - 1) / 2 - k);
#pragma unroll 4
      for (int kp = rs; kp < kp1; ++kp) {
        const float2 c = row[kp];
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j)
          if (j < J) acc[j] = cfma(c, ph[kp * J + j], acc[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j)
      if (j < J) red[(size_t)e * J + j] = acc[j];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nbc * KJ; e += NT) {
    const int bi = e / KJ, i = e - bi * KJ, k = i / J, j = i - k * J;
    const int f = f0 + bi, w2 = f % fw;
    float2 s = make_float2(0.f, 0.f);
    for (int pi = 0; pi < PS; ++pi) s = cadd(s, red[(((size_t)bi * PS + pi) * K + k) * J + j]);
    a.yv[(size_t)i * NF + f] = s;
    const float2 p = phat[e];
    add_at(part, j, (w2 == 0 ? 1.f : 2.f) * (p.x * s.x + p.y * s.y));
  }
}

// y = crop(F^-1 y_hat) on the taps for one filter, y_hat ([J][NF]) in shared memory and complete.
// Thread t gets y at taps o = t, t + NT, ... in out[o].
template <int NT>
__device__ void product_taps(const CgArgs& a, const float2* yh, float2* sc, const float2* twa, const float2* twb,
                             float* out) {
  const int J = a.J, NF = a.NF, fw = a.fw, fh = a.fh, La = a.La, Lb = a.Lb, S2 = a.S2;
  // over w1: sc[j][w2][qa] = sum_w1 y_hat[j][w1][w2] exp(+2 pi i w1 qa / La), four lanes per item
  {
    const int sub = threadIdx.x & 3;
    const int nit = J * fw * fh;
    for (int e0 = threadIdx.x >> 2; e0 < ((nit + 7) / 8) * 8; e0 += NT / 4) {
      const int e = e0 < nit ? e0 : nit - 1;
      const int j = e / (fw * fh), rem = e - j * fw * fh, w2 = rem / fh, qa = rem - w2 * fh;
      float2 s = make_float2(0.f, 0.f);
      int m = (sub * qa) % La;
      const int step = (4 * qa) % La;
      for (int w1 = sub; w1 < La; w1 += 4) {
        s = cfmac(twa[m], yh[(size_t)j * NF + w1 * fw + w2], s);
        m += step;
        if (m >= La) m -= La;
      }
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 1);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 1);
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 2);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 2);
      if (sub == 0 && e0 < nit) sc[e] = s;
    }
  }
  __syncthreads();
  // over w2: y[j][qa][qb] = sum_w2 wt(w2) Re(sc[j][w2][qa] exp(+2 pi i w2 qb / Lb))
  for (int o = threadIdx.x; o < J * S2; o += NT) {
    const int j = o / S2, q = o - j * S2, qa = q / fw, qb = q - qa * fw;
    float s = 0.f;
    int m = 0;
    for (int w2 = 0; w2 < fw; ++w2) {
      const float2 v = sc[((size_t)j * fw + w2) * fh + qa];
      const float2 e = twb[m];   // exp(-i .); Re(v conj(e))
      s = fmaf(w2 == 0 ? 1.f : 2.f, v.x * e.x + v.y * e.y, s);
      m += qb;
      if (m >= Lb) m -= Lb;
    }
    out[o] = s;
  }
}

// z = M_k^{-1} r for one filter (r complete in shared memory) with the Jacobi preconditioner
// M_k^{-1} = 1 / (C_kk(0) + 2 mu_k) of the current step, written to zo and to a.zv; the partial r . z
// into part[j]. (A block-Jacobi inverse of the filter's Toeplitz block, formed once per call, was
// tried: it goes stale as mu grows from step to step, and took more CG iterations than this one.)
template <int NT, int N>
__device__ __forceinline__ void precondition_k(const CgArgs& a, int k, bool act, float sjac, const float* r,
                                               float* zo, float (&part)[N]) {
  const int S2 = a.S2, JS = a.J * S2;
  for (int o = threadIdx.x; o < JS; o += NT) {
    const int j = o / S2;
    const float zv = act ? r[o] * sjac : 0.f;
    zo[o] = zv;
    a.zv[(size_t)k * JS + o] = zv;
    add_at(part, j, r[o] * zv);
  }
}

template <int NT, int JT>
__global__ void __launch_bounds__(NT, 1) k_learn_cg(CgArgs a) {
  extern __shared__ float smf[];
  __shared__ float scratch[(NT / 32) * kSlotWords];
  __shared__ float tot[kSlotWords];
  __shared__ float gvals[2 * NT];   // slot words of the current exchange [G][nw]
  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = 0;
  __shared__ float s_twomu[8], s_jac[8];
  // scalars of the CG iteration, formed by thread 0 in float64
  __shared__ float s_rz[kMaxJ], s_rr[kMaxJ], s_bb[kMaxJ];
  __shared__ float s_alpha[kMaxJ], s_beta[kMaxJ];
  __shared__ int s_done[kMaxJ], s_all;
  __shared__ int s_act[8];
  constexpr int J = JT;
  const int K = a.K, S2 = a.S2, G = a.G;
  const int JS = J * S2;
  const CgSmem Ls = cg_smem_layout(K, J, S2, a.NF, a.fh, a.fw, a.La, a.Lb, NT, G, a.chat_smem);
  float2* ew = reinterpret_cast<float2*>(smf + Ls.ew);
  float2* phat = reinterpret_cast<float2*>(smf + Ls.phat);
  float2* red = reinterpret_cast<float2*>(smf + Ls.red);
  float2* yh = reinterpret_cast<float2*>(smf + Ls.yh);
  float2* sc = reinterpret_cast<float2*>(smf + Ls.sc);
  float2* twa = reinterpret_cast<float2*>(smf + Ls.twa);
  float2* twb = reinterpret_cast<float2*>(smf + Ls.twb);
  float2* cch = a.chat_smem ? reinterpret_cast<float2*>(smf + Ls.cch) : nullptr;   // [nb][K(K+1)/2]
  float* pp = smf + Ls.pp;                       // [K][J][S2] the whole search direction
  float* ox = smf + Ls.own;                      // [nown][J][S2] x, r, b, z of the CTA's filters
  float* orr = ox + (size_t)Ls.nown * JS;
  float* ob = orr + (size_t)Ls.nown * JS;
  float* oz = ob + (size_t)Ls.nown * JS;
  const int nown = (blockIdx.x < K) ? (K - 1 - blockIdx.x) / G + 1 : 0;
  const int La = a.La, Lb = a.Lb, ctr = (a.fh - 1) * Lb + (a.fw - 1);   // lag tau = 0
  const int f0 = (int)((long long)blockIdx.x * a.NF / G), f1 = (int)((long long)(blockIdx.x + 1) * a.NF / G);
  const int nbc = f1 - f0;
  const float tol2f = (float)a.tol2;
  unsigned ep = 0;

  for (int i = threadIdx.x; i < La; i += NT) twa[i] = unit_root(i, La);
  for (int i = threadIdx.x; i < Lb; i += NT) twb[i] = unit_root(i, Lb);
  __syncthreads();
  // tap twiddles of the CTA's bins: exp(-2 pi i (w1 qa / La + w2 qb / Lb))
  for (int e = threadIdx.x; e < nbc * S2; e += NT) {
    const int bi = e / S2, q = e - bi * S2, f = f0 + bi;
    const int w1 = f / a.fw, w2 = f - w1 * a.fw, qa = q / a.fw, qb = q - qa * a.fw;
    ew[e] = cmul(twa[(w1 * qa) % La], twb[(w2 * qb) % Lb]);
  }
  // the CTA's bins of the lag spectra
  if (cch) {
    const size_t n = (size_t)nbc * (K * (K + 1) / 2);
    const float2* src = a.chat + (size_t)f0 * (K * (K + 1) / 2);
    for (size_t i = threadIdx.x; i < n; i += NT) cch[i] = __ldg(src + i);
  }
  // the CTA's filters: activity, x, b
  if (threadIdx.x < nown) {
    const int k = blockIdx.x + threadIdx.x * G;
    const float c0 = a.lags[((size_t)k * K + k) * La * Lb + ctr];   // sum of z_k^2 over all images
    s_act[threadIdx.x] = c0 > 0.f;
    if (!isfinite(c0)) atomicCAS(a.err, 0, (int)CSC_ERR_NONFINITE);   // a code was not finite
  }
  for (int i = 0; i < nown; ++i) {
    const int k = blockIdx.x + i * G;
    for (int o = threadIdx.x; o < JS; o += NT) {
      ox[(size_t)i * JS + o] = a.x[(size_t)k * JS + o];
      ob[(size_t)i * JS + o] = a.b[(size_t)k * JS + o];
    }
  }
  __syncthreads();


  const int NF = a.NF, nz = K * JS;
  // y_hat of the CTA's filter k into yh (read through L2 after an exchange)
  auto load_y = [&](int k) {
    const float2* src = a.yv + (size_t)k * J * NF;
    for (int i = threadIdx.x; i < J * NF; i += NT) yh[i] = __ldcg(src + i);
  };
  for (int step = 0; step < a.steps; ++step) {
    if (threadIdx.x < nown) {
      const int k = blockIdx.x + threadIdx.x * G;
      const double m2 = 2.0 * a.mu[k];
      s_twomu[threadIdx.x] = (float)m2;
      s_jac[threadIdx.x] = s_act[threadIdx.x] ? (float)(1.0 / ((double)a.lags[((size_t)k * K + k) * La * Lb + ctr] + m2)) : 0.f;
    }
    // ---- r = b - A x, z = M^{-1} r, p = z -----------------------------------------------
    axpy_from_l2<NT>(pp, a.x, K * JS, JS, S2, nullptr, true);
    __syncthreads();
    {
      float pa[J];
#pragma unroll
      for (int j = 0; j < J; ++j) pa[j] = 0.f;
      product_bins<NT, J>(a, f0, nbc, pp, ew, phat, red, cch, pa);
    }
    __syncthreads();
    cg_arrive(a, nullptr, 0, ++ep);   // no sums: an exchange of y_hat only
    if (!cg_wait<NT>(a, ep, 0, gvals, tot, &s_fail, [] {})) return;
    {
      float w3[3 * J];   // r . z, r . r, b . b
#pragma unroll
      for (int u = 0; u < 3 * J; ++u) w3[u] = 0.f;
      for (int i = 0; i < nown; ++i) {
        const int k = blockIdx.x + i * G;
        load_y(k);
        __syncthreads();
        float* r = orr + (size_t)i * JS;
        product_taps<NT>(a, yh, sc, twa, twb, r);   // r <- (S Z^T Z S^T x)_k
        const bool act = s_act[i];
        for (int o = threadIdx.x; o < JS; o += NT) {
          const int j = J == 1 ? 0 : o / S2;
          const float bv = ob[(size_t)i * JS + o];
          const float rv = act ? bv - fmaf(s_twomu[i], ox[(size_t)i * JS + o], r[o]) : 0.f;
          r[o] = rv;
          add_at(w3, J + j, rv * rv);
          if (act) add_at(w3, 2 * J + j, bv * bv);
        }
        __syncthreads();
        precondition_k<NT>(a, k, act, s_jac[i], r, oz + (size_t)i * JS, w3);
      }
      block_reduce_to0<NT>(w3, scratch);
      cg_arrive(a, w3, 3 * J, ++ep);
    }
    // all z (and the sums) of exchange ep: p = z
    if (!cg_wait<NT>(a, ep, 3 * J, gvals, tot, &s_fail, [&]() {
          int all = 1;
          bool nonfinite = false;
          for (int j = 0; j < J; ++j) {
            s_rz[j] = tot[j];
            s_rr[j] = tot[J + j];
            s_bb[j] = tot[2 * J + j];
            s_done[j] = !(s_rr[j] > tol2f * s_bb[j]) || !(s_rz[j] > 0.f);
            all = all && s_done[j];
            if (!isfinite(s_rr[j]) || !isfinite(s_rz[j]) || !isfinite(s_bb[j])) nonfinite = true;
          }
          if (nonfinite) {   // the same totals in every CTA: all of them stop here together
            if (blockIdx.x == 0) atomicCAS(a.err, 0, (int)CSC_ERR_NONFINITE);
            all = 1;
          }
          s_all = all;
        }))
      return;
    axpy_from_l2<NT>(pp, a.zv, nz, JS, S2, nullptr, true);
    __syncthreads();
    int it = 0;
    for (; it < a.cg_max; ++it) {
      if (s_all) break;   // the same totals in every CTA
      // ---- A p at this CTA's bins, p . A p (exchange A) -----------------------------------
      {
        float pa[J];
#pragma unroll
        for (int j = 0; j < J; ++j) pa[j] = 0.f;
        product_bins<NT, J>(a, f0, nbc, pp, ew, phat, red, cch, pa);
        for (int i = 0; i < nown; ++i) {
          if (!s_act[i]) continue;
          const int k = blockIdx.x + i * G;
          for (int o = threadIdx.x; o < JS; o += NT) {
            const float pv = pp[(size_t)k * JS + o];
            add_at(pa, J == 1 ? 0 : o / S2, s_twomu[i] * pv * pv);
          }
        }
        block_reduce_to0<NT>(pa, scratch);
        cg_arrive(a, pa, J, ++ep);
      }
      // ---- x += alpha p, r -= alpha A p, z = M^{-1} r (exchange B) ---------------------------
      if (!cg_wait<NT>(a, ep, J, gvals, tot, &s_fail, [&]() {
            for (int j = 0; j < J; ++j) {
              const float pap = tot[j];
              s_alpha[j] = (!s_done[j] && pap > 0.f) ? s_rz[j] / pap : 0.f;
            }
          }))
        return;
      {
        float w2[2 * J];   // r . z, r . r
#pragma unroll
        for (int u = 0; u < 2 * J; ++u) w2[u] = 0.f;
        for (int i = 0; i < nown; ++i) {
          const int k = blockIdx.x + i * G;
          if (!s_act[i]) continue;   // z_k stays 0
          load_y(k);
          __syncthreads();
          float* r = orr + (size_t)i * JS;
          float* yk = oz + (size_t)i * JS;   // A p of the filter, then z
          product_taps<NT>(a, yh, sc, twa, twb, yk);
          for (int o = threadIdx.x; o < JS; o += NT) {
            const int j = J == 1 ? 0 : o / S2;
            const float al = s_alpha[j];
            const float pv = pp[(size_t)k * JS + o];
            const float apv = fmaf(s_twomu[i], pv, yk[o]);
            ox[(size_t)i * JS + o] = fmaf(al, pv, ox[(size_t)i * JS + o]);
            const float rv = fmaf(-al, apv, r[o]);
            r[o] = rv;
            add_at(w2, J + j, rv * rv);
          }
          __syncthreads();
          precondition_k<NT>(a, k, true, s_jac[i], r, yk, w2);
        }
        block_reduce_to0<NT>(w2, scratch);
        cg_arrive(a, w2, 2 * J, ++ep);
      }
      // ---- p = z + beta p: every CTA keeps the whole search direction ------------------------
      if (!cg_wait<NT>(a, ep, 2 * J, gvals, tot, &s_fail, [&]() {
            int all = 1;
            bool nonfinite = false;
            for (int j = 0; j < J; ++j) {
              if (!s_done[j]) {
                s_beta[j] = s_rz[j] > 0.f ? tot[j] / s_rz[j] : 0.f;
                s_rz[j] = tot[j];
                s_rr[j] = tot[J + j];
                s_done[j] = !(s_rr[j] > tol2f * s_bb[j]) || !(s_rz[j] > 0.f);
                if (!isfinite(s_rr[j]) || !isfinite(s_rz[j])) nonfinite = true;
              } else {
                s_beta[j] = 0.f;
              }
              all = all && s_done[j];
            }
            if (nonfinite) {   // the same totals in every CTA: all of them stop here together
              if (blockIdx.x == 0) atomicCAS(a.err, 0, (int)CSC_ERR_NONFINITE);
              all = 1;
            }
            s_all = all;
          }))
        return;
      {
        constexpr int U = 24;   // z values per thread in flight
        for (int i0 = threadIdx.x; i0 < nz; i0 += U * NT) {
          float v[U];
#pragma unroll
          for (int u = 0; u < U; ++u) v[u] = (i0 + u * NT < nz) ? __ldcg(a.zv + i0 + u * NT) : 0.f;
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int idx = i0 + u * NT;
            if (idx < nz) pp[idx] = fmaf(s_beta[J == 1 ? 0 : (idx % JS) / S2], pp[idx], v[u]);
          }
        }
      }
      __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.iters) a.iters[step] = it;
    // ---- mu_k <- max(mu_k ||d_k||, floor) for active filters (Eq. mu_update); x to global -------
    for (int i = 0; i < nown; ++i) {
      const int k = blockIdx.x + i * G;
      float sq[1] = {0.f};
      for (int o = threadIdx.x; o < JS; o += NT) {
        const float xv = ox[(size_t)i * JS + o];
        sq[0] = fmaf(xv, xv, sq[0]);
        a.x[(size_t)k * JS + o] = xv;
      }
      block_reduce_to0<NT>(sq, scratch);
      if (threadIdx.x == 0 && s_act[i]) a.mu[k] = fmax(a.mu[k] * sqrt((double)sq[0]), a.mu_floor);
      __syncthreads();
    }
    __syncthreads();
    cg_arrive(a, nullptr, 0, ++ep);   // x (plain stores) complete everywhere before the next step
    if (!cg_wait<NT>(a, ep, 0, gvals, tot, &s_fail, [] {})) return;
  }
  // ---- d_k <- d_k / max(1, ||d_k||) ---------------------------------------------------------
  for (int i = 0; i < nown; ++i) {
    const int k = blockIdx.x + i * G;
    float sq[1] = {0.f};
    for (int o = threadIdx.x; o < JS; o += NT) {
      const float xv = ox[(size_t)i * JS + o];
      sq[0] = fmaf(xv, xv, sq[0]);
    }
    block_reduce_to0<NT>(sq, scratch);
    if (threadIdx.x == 0) scratch[0] = 1.0f / fmaxf(1.0f, sqrtf(sq[0]));
    __syncthreads();
    const float sc2 = scratch[0];
    for (int o = threadIdx.x; o < JS; o += NT) a.x[(size_t)k * JS + o] = ox[(size_t)i * JS + o] * sc2;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
cudaError_t launch_learn_rhs(const Ctx& c, const float2* spec) { return geo_ops(c).rhs(c, spec); }

cudaError_t launch_learn_gram(const Ctx& c) {
  const int ntile = (c.K + kGramT - 1) / kGramT;
  GramArgs a{c.N, c.K, c.g.Omega, ntile, c.L.zhat, c.L.gram};
  dim3 grid(ntile * (ntile + 1) / 2, (c.g.Omega + kGramF - 1) / kGramF);
  k_learn_gram<<<grid, kGramNT, 0, c.stream>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// lags from the frequency-major Gram of the tensor-core path, gramT[o][p], pairs in column order
// p = k'(k'+1)/2 + k (k <= k'), o = kh * Wc + kw. Only the La x Lb window of C_kk' = F^-1 G_kk' / D is
// needed, so the inverse transform is two direct partial sums (G is Hermitian: C is real):
//   T(kh, w) = sum_{kw < Wc} c(kw) G(kh, kw) e^{+2 pi i kw w / W},  c = 1 at kw = 0 and kw = W/2, else 2
//   C(h, w)  = (1/D) sum_kh Re[T(kh, w) e^{+2 pi i kh h / H}],        |h| < fh, |w| < fw
// with one thread per pair in both (coalesced over p), twiddles from exact integer phases.
// ---------------------------------------------------------------------------------------------
struct LagSepArgs {
  int K, H, W, Wc, fh, fw, La, Lb, np;
  const float2* gramT;   // [Omega][np]
  float2* T;             // [H][Lb][np]
  float* lags;           // [K][K][La][Lb]
  float invD;
};

constexpr int kLagSepNT = 128, kLagSepU = 24, kLagSepB = 4;

__device__ __forceinline__ float2 root_pos(long long m, int L) {   // exp(+2 pi i m / L)
  int r = (int)(m % L);
  if (r < 0) r += L;
  float s, c;
  sincospif(2.0f * (float)r / (float)L, &s, &c);
  return make_float2(c, s);
}

// one thread per (pair, row kh): up to kLagSepU values of w per pass over the row (one pass when
// 2 fw - 1 <= 24), the row's Gram values loaded kLagSepB at a time ahead of their use
__global__ void __launch_bounds__(kLagSepNT) k_lags_rows(LagSepArgs a) {
  extern __shared__ float2 e1[];   // [Wc][Lb]: c(kw) e^{2 pi i kw w / W}
  const int kh = blockIdx.y;
  for (int i = threadIdx.x; i < a.Wc * a.Lb; i += kLagSepNT) {
    const int kw = i / a.Lb, wi = i - kw * a.Lb;
    const float2 r = root_pos((long long)kw * (wi - (a.fw - 1)), a.W);
    const float wt = (kw == 0 || 2 * kw == a.W) ? 1.f : 2.f;
    e1[i] = make_float2(wt * r.x, wt * r.y);
  }
  __syncthreads();
  const int p = blockIdx.x * kLagSepNT + threadIdx.x;
  if (p >= a.np) return;
  const float2* g = a.gramT + (size_t)kh * a.Wc * a.np + p;
  for (int w0 = 0; w0 < a.Lb; w0 += kLagSepU) {
    float2 acc[kLagSepU];
#pragma unroll
    for (int j = 0; j < kLagSepU; ++j) acc[j] = make_float2(0.f, 0.f);
    for (int kw0 = 0; kw0 < a.Wc; kw0 += kLagSepB) {
      float2 gv[kLagSepB];
#pragma unroll
      for (int b = 0; b < kLagSepB; ++b)
        gv[b] = kw0 + b < a.Wc ? __ldg(g + (size_t)(kw0 + b) * a.np) : make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < kLagSepB; ++b) {
        if (kw0 + b >= a.Wc) break;
        const float2* e = e1 + (kw0 + b) * a.Lb + w0;
#pragma unroll
        for (int j = 0; j < kLagSepU; ++j)
          if (w0 + j < a.Lb) acc[j] = cfma(gv[b], e[j], acc[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < kLagSepU; ++j)
      if (w0 + j < a.Lb) a.T[((size_t)kh * a.Lb + w0 + j) * a.np + p] = acc[j];
  }
}

// acc[j] = C(h, w) for ta = h + fh - 1 = h0 + j (REV: ta = La - 1 - (h0 + j)) and the w of T column
// wt. Both orders form each value with the same operations in the same order, so C(tau) comes out
// bitwise the same whichever thread forms it.
template <bool REV>
__device__ __forceinline__ void lag_column(const LagSepArgs& a, const float2* e2, int p, int wt, int h0, float* acc) {
  const float2* t = a.T + (size_t)wt * a.np + p;
#pragma unroll
  for (int j = 0; j < kLagSepU; ++j) acc[j] = 0.f;
  for (int kh0 = 0; kh0 < a.H; kh0 += kLagSepB) {
    float2 tv[kLagSepB];
#pragma unroll
    for (int b = 0; b < kLagSepB; ++b)
      tv[b] = kh0 + b < a.H ? __ldg(t + (size_t)(kh0 + b) * a.Lb * a.np) : make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < kLagSepB; ++b) {
      if (kh0 + b >= a.H) break;
      const float2* e = e2 + (kh0 + b) * a.La;
#pragma unroll
      for (int j = 0; j < kLagSepU; ++j)
        if (h0 + j < a.La) {
          const float2 ev = e[REV ? a.La - 1 - (h0 + j) : h0 + j];
          acc[j] = fmaf(tv[b].x, ev.x, fmaf(-tv[b].y, ev.y, acc[j]));
        }
    }
  }
}

__global__ void __launch_bounds__(kLagSepNT) k_lags_cols(LagSepArgs a) {
  extern __shared__ float2 e2[];   // [H][La]: e^{2 pi i kh h / H} / D
  const int wi = blockIdx.y;
  for (int i = threadIdx.x; i < a.H * a.La; i += kLagSepNT) {
    const int kh = i / a.La, hi = i - kh * a.La;
    const float2 r = root_pos((long long)kh * (hi - (a.fh - 1)), a.H);
    e2[i] = make_float2(r.x * a.invD, r.y * a.invD);
  }
  __syncthreads();
  const int p = blockIdx.x * kLagSepNT + threadIdx.x;
  if (p >= a.np) return;
  // column-order pair p = k'(k'+1)/2 + k
  int kp = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
  while (kp * (kp + 1) / 2 > p) --kp;
  while ((kp + 1) * (kp + 2) / 2 <= p) ++kp;
  const int k = p - kp * (kp + 1) / 2;
  const int LL = a.La * a.Lb;
  float* out = a.lags + ((size_t)k * a.K + kp) * LL;
  float* outT = a.lags + ((size_t)kp * a.K + k) * LL;
  for (int h0 = 0; h0 < a.La; h0 += kLagSepU) {
    float acc[kLagSepU];
    lag_column<false>(a, e2, p, wi, h0, acc);
    if (k == kp) {
      // autocorrelation: C_kk(tau) = C_kk(-tau); store the symmetrised value so the matrix of the
      // normal equations is exactly symmetric (the writers of tau and -tau add the same two values)
      float m[kLagSepU];
      lag_column<true>(a, e2, p, a.Lb - 1 - wi, h0, m);
#pragma unroll
      for (int j = 0; j < kLagSepU; ++j) {
        const int hi = h0 + j;
        if (hi >= a.La) break;
        out[hi * a.Lb + wi] = 0.5f * (acc[j] + m[j]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < kLagSepU; ++j) {
        const int hi = h0 + j;
        if (hi >= a.La) break;
        out[hi * a.Lb + wi] = acc[j];
        outT[(a.La - 1 - hi) * a.Lb + (a.Lb - 1 - wi)] = acc[j];   // C_k'k(tau) = C_kk'(-tau)
      }
    }
  }
}

// Both partial sums in one kernel for windows up to 24 x 24 (filters up to 12 x 12): a CTA owns 8
// pairs; for each pair 8 threads own the w columns sub, sub + 8, sub + 16 and 4 thread groups split
// the H rows of the Gram (group g takes rows g, g + 4, ...), each group with a four-deep cp.async
// ring of its row tiles [Wc][8 pairs]. A thread forms T(kh, w) for its columns and adds
// Re[T e^{2 pi i kh h / H}] / D into its C(h, w) registers; the four groups' partial windows are
// then added in group order through shared memory. No T buffer.
constexpr int kLfPairs = 8, kLfSub = 8, kLfGroups = 4, kLfNT = kLfPairs * kLfSub * kLfGroups, kLfNW = 3, kLfNH = 24,
              kLfStages = 4;

__device__ __forceinline__ void cp_async8_lag(void* dst, const void* src, bool valid) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}

static size_t lags_fused_ring(const Ctx& c) {
  return (size_t)kLfGroups * kLfStages * c.g.Wc * kLfPairs * sizeof(float2);
}

size_t lags_fused_smem(const Ctx& c) {
  const int La = 2 * c.fh - 1, Lb = 2 * c.fw - 1;
  return ((size_t)c.g.Wc * Lb + (size_t)c.g.H * La) * sizeof(float2) + lags_fused_ring(c);
}

bool lags_fused_applies(const Ctx& c) {
  const int La = 2 * c.fh - 1, Lb = 2 * c.fw - 1;
  return La <= kLfNH && Lb <= kLfNW * kLfSub && lags_fused_smem(c) <= kSmemLimit &&
         (size_t)kLfGroups * kLfPairs * La * Lb * sizeof(float) <= lags_fused_ring(c);
}

__global__ void __launch_bounds__(kLfNT) k_lags_fused(LagSepArgs a) {
  extern __shared__ float2 lsm[];
  float2* e1 = lsm;                          // [Wc][Lb]: c(kw) e^{2 pi i kw w / W}
  float2* e2 = e1 + a.Wc * a.Lb;             // [H][La]: e^{2 pi i kh h / H} / D
  float2* gs = e2 + a.H * a.La;              // [kLfGroups][kLfStages][Wc][kLfPairs]
  for (int i = threadIdx.x; i < a.Wc * a.Lb; i += kLfNT) {
    const int kw = i / a.Lb, wi = i - kw * a.Lb;
    const float2 r = root_pos((long long)kw * (wi - (a.fw - 1)), a.W);
    const float wt = (kw == 0 || 2 * kw == a.W) ? 1.f : 2.f;
    e1[i] = make_float2(wt * r.x, wt * r.y);
  }
  for (int i = threadIdx.x; i < a.H * a.La; i += kLfNT) {
    const int kh = i / a.La, hi = i - kh * a.La;
    const float2 r = root_pos((long long)kh * (hi - (a.fh - 1)), a.H);
    e2[i] = make_float2(r.x * a.invD, r.y * a.invD);
  }
  const int p0 = blockIdx.x * kLfPairs;
  const int grp = threadIdx.x / (kLfPairs * kLfSub);        // row group
  const int gt = threadIdx.x % (kLfPairs * kLfSub);         // thread within the group
  const int q = gt / kLfSub, sub = gt % kLfSub;
  const int tile = a.Wc * kLfPairs;
  float2* ring = gs + (size_t)grp * kLfStages * tile;
  const int nrounds = (a.H + kLfGroups - 1) / kLfGroups;
  auto issue_row = [&](int r) {   // row kh = grp + kLfGroups r of this group into slot r % kLfStages
    const int kh = grp + kLfGroups * r;
    if (kh < a.H) {
      float2* dst = ring + (r % kLfStages) * tile;
      const float2* src = a.gramT + (size_t)kh * a.Wc * a.np + p0;
      for (int i = gt; i < tile; i += kLfPairs * kLfSub) {
        const int kw = i / kLfPairs, qq = i - kw * kLfPairs;
        const bool v = p0 + qq < a.np;
        cp_async8_lag(dst + i, src + (size_t)kw * a.np + (v ? qq : 0), v);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  for (int r = 0; r < kLfStages - 1; ++r) issue_row(r);
  float acc[kLfNW][kLfNH];
#pragma unroll
  for (int w = 0; w < kLfNW; ++w)
#pragma unroll
    for (int h = 0; h < kLfNH; ++h) acc[w][h] = 0.f;
  for (int r = 0; r < nrounds; ++r) {
    issue_row(r + kLfStages - 1);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kLfStages - 1) : "memory");
    __syncthreads();   // row r of every group (and, on the first pass, the twiddle tables) visible
    const int kh = grp + kLfGroups * r;
    if (kh < a.H) {
      const float2* g = ring + (r % kLfStages) * tile + q;
      float2 t[kLfNW];
#pragma unroll
      for (int w = 0; w < kLfNW; ++w) t[w] = make_float2(0.f, 0.f);
      for (int kw = 0; kw < a.Wc; ++kw) {
        const float2 gv = g[kw * kLfPairs];
        const float2* e = e1 + kw * a.Lb + sub;
#pragma unroll
        for (int w = 0; w < kLfNW; ++w)
          if (sub + kLfSub * w < a.Lb) t[w] = cfma(gv, e[kLfSub * w], t[w]);
      }
      const float2* e = e2 + kh * a.La;
#pragma unroll
      for (int w = 0; w < kLfNW; ++w)
#pragma unroll
        for (int h = 0; h < kLfNH; ++h)
          if (h < a.La) acc[w][h] = fmaf(t[w].x, e[h].x, fmaf(-t[w].y, e[h].y, acc[w][h]));
    }
    __syncthreads();   // every read of round r's slots precedes their refill
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  // the groups' partial windows through shared memory (the rings are free): [group][pair][La][Lb]
  float* xs = reinterpret_cast<float*>(gs);
  const int LL = a.La * a.Lb;
#pragma unroll
  for (int w = 0; w < kLfNW; ++w) {
    const int wi = sub + kLfSub * w;
    if (wi >= a.Lb) continue;
#pragma unroll
    for (int h = 0; h < kLfNH; ++h)
      if (h < a.La) xs[(grp * kLfPairs + q) * LL + h * a.Lb + wi] = acc[w][h];
  }
  __syncthreads();
  auto total = [&](int qq, int i) {   // the four groups' sum, always in group order
    float v = 0.f;
#pragma unroll
    for (int gg = 0; gg < kLfGroups; ++gg) v += xs[(gg * kLfPairs + qq) * LL + i];
    return v;
  };
  for (int e = threadIdx.x; e < kLfPairs * LL; e += kLfNT) {
    const int qq = e / LL, i = e - qq * LL;
    const int p = p0 + qq;
    if (p >= a.np) continue;
    int kp = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
    while (kp * (kp + 1) / 2 > p) --kp;
    while ((kp + 1) * (kp + 2) / 2 <= p) ++kp;
    const int k = p - kp * (kp + 1) / 2;
    const float v = total(qq, i);
    if (k == kp) {
      // autocorrelation: C_kk(tau) = C_kk(-tau); the writers of tau and -tau add the same two
      // values, so the normal-equation matrix is exactly symmetric
      a.lags[((size_t)k * a.K + kp) * LL + i] = 0.5f * (v + total(qq, LL - 1 - i));
    } else {
      a.lags[((size_t)k * a.K + kp) * LL + i] = v;
      a.lags[((size_t)kp * a.K + k) * LL + (LL - 1 - i)] = v;   // C_k'k(tau) = C_kk'(-tau)
    }
  }
}

size_t lag_sep_T_count(const Ctx& c) {
  if (lags_fused_applies(c)) return 1;   // the fused kernel keeps T in registers
  return (size_t)c.g.H * (2 * c.fw - 1) * ((size_t)c.K * (c.K + 1) / 2);
}


cudaError_t launch_learn_lags_sep(const Ctx& c) {
  const int La = 2 * c.fh - 1, Lb = 2 * c.fw - 1;
  const int np = c.K * (c.K + 1) / 2;
  LagSepArgs a{c.K, c.g.H, c.g.W, c.g.Wc, c.fh, c.fw, La, Lb, np, c.L.gram, c.L.lagT, c.L.lags,
               1.0f / (float)c.g.D};
  const size_t s1 = (size_t)c.g.Wc * Lb * sizeof(float2), s2 = (size_t)c.g.H * La * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_lags_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lags_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2);
  if (e != cudaSuccess) return e;
  if (lags_fused_applies(c)) {
    const size_t sf = lags_fused_smem(c);
    if ((e = cudaFuncSetAttribute(k_lags_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf)) != cudaSuccess)
      return e;
    k_lags_fused<<<(np + kLfPairs - 1) / kLfPairs, kLfNT, sf, c.stream>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    c.launches += 1;
    return launch_lag_spectra(c);
  }
  const int tiles = (np + kLagSepNT - 1) / kLagSepNT;
  k_lags_rows<<<dim3(tiles, c.g.H), kLagSepNT, s1, c.stream>>>(a);
  k_lags_cols<<<dim3(tiles, Lb), kLagSepNT, s2, c.stream>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  c.launches += 2;
  return launch_lag_spectra(c);
}

cudaError_t launch_learn_lags(const Ctx& c) {
  cudaError_t e = geo_ops(c).lags(c);
  if (e != cudaSuccess) return e;
  c.launches += 1;
  return launch_lag_spectra(c);
}

cudaError_t launch_lag_spectra(const Ctx& c) {
  const int La = 2 * c.fh - 1, Lb = 2 * c.fw - 1;
  LagSpecArgs a{c.K, c.fh, c.fw, La, Lb, La * c.fw, c.L.lags, c.L.chat};
  const size_t smem = (size_t)(La * c.fw + La + Lb) * sizeof(float2) + (size_t)La * Lb * sizeof(float);
  const int npairs = c.K * (c.K + 1) / 2;
  k_lag_spectra<<<npairs, kLagSpecNT, smem, c.stream>>>(a);
  c.launches += 1;
  return cudaGetLastError();
}

// one CTA per SM at most, and no more than the 2 NT slot words of an exchange hold (3 J per CTA)
int learn_cg_ctas(const Ctx& c) {
  const int La = 2 * c.fh - 1;
  const int nsm = c.nsm > 0 ? c.nsm : 1;
  return std::max(1, std::min(std::min(nsm, 2 * kNT / (3 * c.J)), std::max(c.K, La * c.fw)));
}

bool learn_cg_shape_ok(const Ctx& c) {
  const int G = learn_cg_ctas(c);
  const int NF = (2 * c.fh - 1) * c.fw;
  return (c.K + G - 1) / G <= 8 && 2 * c.J * NF <= 6 * kNT;
}

size_t learn_cg_smem_bytes(const Ctx& c, bool chat_smem) {
  const int La = 2 * c.fh - 1, Lb = 2 * c.fw - 1;
  const int G = learn_cg_ctas(c);
  return cg_smem_layout(c.K, c.J, c.S2, La * c.fw, c.fh, c.fw, La, Lb, kNT, G, chat_smem).total_floats *
         sizeof(float);
}

cudaError_t launch_learn_cg(const Ctx& c, float* d, int steps, int* dev_err) {
  constexpr int NT = kNT;
  CgArgs a;
  a.K = c.K; a.J = c.J; a.fh = c.fh; a.fw = c.fw; a.S2 = c.S2;
  a.La = 2 * c.fh - 1; a.Lb = 2 * c.fw - 1; a.NF = a.La * c.fw;
  a.G = 0; a.steps = steps; a.cg_max = c.p.cg_max;
  a.tol2 = c.p.cg_tol * c.p.cg_tol; a.mu_floor = kMuFloor;
  a.lags = c.L.lags; a.chat = c.L.chat; a.b = c.L.b; a.x = d;
  a.yv = reinterpret_cast<float2*>(c.L.yw);   // the words buffers hold the plain values
  a.zv = reinterpret_cast<float*>(c.L.zw);
  a.mu = c.L.mu; a.iters = c.L.iters; a.err = dev_err;
  a.spin = c.wait_limit > 0 ? c.wait_limit : kSpinLimit;
  // the grid: one CTA per SM at most (every CTA must be resident: the exchanges wait on all)
  a.G = learn_cg_ctas(c);
  // the exchange counter restarts at 0 every launch; the slots (floats, then the counter) live in
  // the slot buffer
  a.slots = reinterpret_cast<float*>(c.L.slots);
  a.arrivals = reinterpret_cast<unsigned*>(a.slots + (size_t)2 * a.G * kSlotWords);
  cudaError_t e = cudaMemsetAsync(a.arrivals, 0, sizeof(unsigned), c.stream);
  if (e != cudaSuccess) return e;
  auto kern = c.J == 1 ? k_learn_cg<NT, 1> : c.J == 2 ? k_learn_cg<NT, 2> : k_learn_cg<NT, 3>;
  // the CTA's bins of the lag spectra stay in shared memory when they fit
  a.chat_smem = learn_cg_smem_bytes(c, true) <= kSmemLimit ? 1 : 0;
  const size_t smem = learn_cg_smem_bytes(c, a.chat_smem != 0);
  if (smem > kSmemLimit) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if ((c.K + a.G - 1) / a.G > 8) return cudaErrorInvalidValue;   // filters per CTA
  if (a.G * 3 * c.J > 2 * NT) return cudaErrorInvalidValue;       // slot words per exchange
  if (2 * c.J * a.NF > 6 * NT) return cudaErrorInvalidValue;      // y_hat words per filter
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(a.G), dim3(NT), args, smem, c.stream);
}

}  // namespace csc
