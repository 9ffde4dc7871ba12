// The CG of the video learning (Sec. 3.2, Eqs. Learning_new .. mu_update, on the 3-D extension of
// Sec. 3.3) as one persistent cooperative launch over all learning steps.
//
// The system per channel j is (S Z^T Z S^T + 2 diag(mu)) d_j = b_j, its matrix applied in the Fourier
// domain of the Lt x La x Lb lag grid (half spectrum along the last axis, NF = Lt La fw bins):
//     y_kj = crop F^-1 ( sum_k' C_hat_kk' F(p_k'j) ),   C_hat = F(C) / (Lt La Lb).
// The search direction (K J ft fh fw floats: 464 KB for K = 64 colour 5 x 11 x 11 filters) does not
// fit in one SM, so it is never gathered: CTA b owns
//   * the items (k, j) in [i0, i1) (filter k, channel j: the taps of x, r, z, p, b stay in its shared
//     memory for the whole launch) and transforms them between taps and bins (separable DFT stages,
//     register-blocked against shared-memory DFT matrices), and
//   * the lag-grid bins [f0, f1), where it forms y_hat = C_hat p_hat for every item.
// A CG iteration has two grid-wide exchanges, each a counter that every CTA increments (release) once
// its partial sums (one slot per CTA) and data (plain stores) are out, and that the readers poll
// (acquire) before reading both through L2:
//   Y: the bins publish y_hat and the partial p . A p, by Parseval over the half spectrum,
//          p . A p = sum_f wt(f) Re(y_hat conj p_hat) + (2 mu_k / (Lt La Lb)) |p_hat|^2,
//      wt = 1 at w2 = 0, else 2 (Lb is odd: no Nyquist bin);
//   Z: the items take alpha, update x, r and z = M^-1 r (Jacobi: 1 / (C_kk(0) + 2 mu_k)), publish
//      z_hat = F(z) and the partial r . z, r . r; every CTA then forms beta, the convergence flags,
//      p_hat = z_hat + beta p_hat at its bins and p = z + beta p on its items (the transform is
//      linear, so p never has to be transformed itself).
// A learning step starts with F(x) -> C x (two exchanges) and ends with one exchange of the items'
// squared norms, from which every CTA forms the same mu_k <- max(mu_k ||d_k||, floor) (Eq. mu_update);
// after the last step d_k <- d_k / max(1, ||d_k||). The partial sums are summed in a fixed order, so
// every CTA forms the same scalars and the result does not depend on timing. Every wait is bounded
// (the context's wait limit) and sets the error word when it runs out.
#include <cuda_runtime.h>

#include <algorithm>

#include "csc_internal.cuh"
#include "cg_exchange.cuh"

namespace csc {
namespace vcg {

constexpr int NT = 512;
constexpr int kItemsMax = 4;   // items per CTA (the norm exchange carries one word per item)
constexpr int kMaxK = 128;
constexpr int kMaxSlotVals = 2048;   // G x (values per CTA) of one exchange

struct VcgArgs {
  int K, J, ft, fh, fw, Lt, La, Lb, S3, NF, G, steps, cg_max;
  double tol2, mu_floor;
  const float* lags;        // [K][K][Lt La Lb]: C_kk at the zero lag (activity, preconditioner)
  int zero_lag, LLL;
  const float2* chat;       // [NF][K][K]: [f][k'][k] = C_hat_kk'(f) / (Lt La Lb)
  const float* b;           // [K][J][S3]
  float* x;                 // [K][J][S3] the filters (warm start in, solution out)
  double* mu;               // [K]
  const int* active;        // [K]: any code of filter k nonzero
  float2* zh;               // [K J][NF] F(x) / z_hat of every item (written by the items' CTAs)
  float2* yh;               // [K J][NF] y_hat of every item (written by the bins' CTAs)
  float* slots;             // [2][G][kSlotWords] partial sums of the exchanges (bank = exchange parity)
  unsigned* arrivals;       // exchange counter: G arrivals per exchange, zeroed before the launch
  int* iters;               // [steps]
  int* err;
  long long spin;
};

// shared-memory layout, the same on host and device: the DFT matrices, p_hat at the CTA's bins (rows
// padded to an odd stride: conflict-free stores), the items' vectors, then the items' transforms (y_hat,
// the two intermediate stages, the operator output)
struct VcgSmem {
  size_t tw, ph, X, R, Z, P, B, U, Y, Q2, Q1, T, total_floats;
  int nb, ni, phs;
};
// the six DFT matrices of the transforms, [input][output] (float2 offsets from tw)
struct VcgTw {
  int bf, af, tf, ti, ai, bi, total;
};
CSC_HD VcgTw vcg_tw(int ft, int fh, int fw, int Lt, int La) {
  VcgTw t;
  int o = 0;
  t.bf = o; o += fw * fw;   // [qb][w2]  e^{-2 pi i w2 qb / Lb}
  t.af = o; o += fh * La;   // [qa][w1]  e^{-2 pi i w1 qa / La}
  t.tf = o; o += ft * Lt;   // [qt][w0]  e^{-2 pi i w0 qt / Lt}
  t.ti = o; o += Lt * ft;   // [w0][qt]  e^{+2 pi i w0 qt / Lt}
  t.ai = o; o += La * fh;   // [w1][qa]  e^{+2 pi i w1 qa / La}
  t.bi = o; o += fw * fw;   // [w2][qb]  wt(w2) e^{+2 pi i w2 qb / Lb}, wt = 1 at w2 = 0, else 2
  t.total = o;
  return t;
}
CSC_HD VcgSmem vcg_layout(int K, int J, int ft, int fh, int fw, int Lt, int La, int Lb, int NF, int G) {
  VcgSmem L;
  const int KJ = K * J, S3 = ft * fh * fw;
  L.nb = (NF + G - 1) / G;
  L.ni = (KJ + G - 1) / G;
  L.phs = KJ | 1;
  size_t o = 0;
  L.tw = o; o += 2 * (size_t)vcg_tw(ft, fh, fw, Lt, La).total;
  L.ph = o; o += 2 * (size_t)L.nb * L.phs;
  L.X = o;  o += (size_t)L.ni * S3;
  L.R = o;  o += (size_t)L.ni * S3;
  L.Z = o;  o += (size_t)L.ni * S3;
  L.P = o;  o += (size_t)L.ni * S3;
  L.B = o;  o += (size_t)L.ni * S3;
  o = (o + 3) & ~(size_t)3;
  L.U = o;
  L.Y = o;  o += 2 * (size_t)L.ni * NF;
  L.Q2 = o; o += 2 * (size_t)L.ni * ft * La * fw;
  L.Q1 = o; o += 2 * (size_t)L.ni * ft * fh * fw;
  L.T = o;  o += (size_t)L.ni * S3;
  L.total_floats = o;
  (void)Lb;
  return L;
}

__device__ __forceinline__ float2 unit_root(int m, int L, float sign) {   // exp(sign 2 pi i m / L)
  int r = m % L;
  if (r < 0) r += L;
  float s, c;
  sincospif(2.0f * (float)r / (float)L, &s, &c);
  return make_float2(c, sign * s);
}

__device__ __forceinline__ void fence_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// One separable DFT stage over a batch of columns: out[c][o] = sum_n in[c][n] W[n][o] (o < nout,
// n < nin), each thread a chunk of CH outputs of one column, accumulated in registers (the lanes of a
// warp take consecutive columns of the same chunk: the W loads are broadcasts). col(c, ib, ob) gives
// the column's input and output base offsets; inputs sit at ib + n is, outputs at ob + o os.
template <int CH, class COL, class LOAD, class STORE>
__device__ __forceinline__ void dft_stage(int ncol, int nin, int nout, const float2* __restrict__ W, int is, int os,
                                          COL col, LOAD load, STORE store) {
  const int nch = (nout + CH - 1) / CH;
  for (int t = threadIdx.x; t < ncol * nch; t += NT) {
    const int ch = t / ncol, c = t - ch * ncol, o0 = ch * CH;
    int ib, ob;
    col(c, ib, ob);
    float2 acc[CH];
#pragma unroll
    for (int o = 0; o < CH; ++o) acc[o] = make_float2(0.f, 0.f);
    const float2* w = W + o0;
    for (int n = 0; n < nin; ++n, w += nout) {
      const float2 x = load(ib + n * is);
#pragma unroll
      for (int o = 0; o < CH; ++o)
        if (o0 + o < nout) acc[o] = cfma(x, w[o], acc[o]);
    }
#pragma unroll
    for (int o = 0; o < CH; ++o)
      if (o0 + o < nout) store(ob + (o0 + o) * os, acc[o]);
  }
}

// F(src) of the CTA's items (src [ni][S3] taps in shared memory) to zh (the items' rows):
// p_hat(f) = sum_q p(q) e^{-2 pi i (w0 qt / Lt + w1 qa / La + w2 qb / Lb)}, along qb, then qa, then qt.
// Does not end synchronised.
__device__ void taps_to_bins(const VcgArgs& a, int i0, int nic, const float* src, float2* Q1, float2* Q2,
                             const float2* tw, const VcgTw& T) {
  const int ft = a.ft, fh = a.fh, fw = a.fw, La = a.La, Lt = a.Lt, LF = La * fw;
  // qb -> w2 (real input): columns (i, qt, qa)
  dft_stage<4>(nic * ft * fh, fw, fw, tw + T.bf, 1, 1, [&](int c, int& ib, int& ob) { ib = c * fw; ob = c * fw; },
               [&](int i) { return make_float2(src[i], 0.f); }, [&](int i, float2 v) { Q1[i] = v; });
  __syncthreads();
  // qa -> w1: columns (i, qt, w2)
  dft_stage<6>(nic * ft * fw, fh, La, tw + T.af, fw, fw,
               [&](int c, int& ib, int& ob) { const int w2 = c % fw, r = c / fw; ib = r * fh * fw + w2; ob = r * LF + w2; },
               [&](int i) { return Q1[i]; }, [&](int i, float2 v) { Q2[i] = v; });
  __syncthreads();
  // qt -> w0: columns (i, w1, w2), to the items' rows of zh
  float2* zrow = a.zh + (size_t)i0 * a.NF;
  dft_stage<10>(nic * LF, ft, Lt, tw + T.tf, LF, LF,
                [&](int c, int& ib, int& ob) { const int i = c / LF, s = c - i * LF; ib = i * ft * LF + s; ob = i * a.NF + s; },
                [&](int i) { return Q2[i]; }, [&](int i, float2 v) { zrow[i] = v; });
}

// y = crop F^-1(y_hat) on the taps of the CTA's items, y_hat [ni][NF] in shared memory, to out [ni][S3]:
// y(q) = sum_f wt(w2) Re(y_hat(f) e^{+2 pi i (w0 qt / Lt + w1 qa / La + w2 qb / Lb)}), along w0, then
// w1, then w2. Ends synchronised.
__device__ void bins_to_taps(const VcgArgs& a, int nic, const float2* Y, float2* Q1, float2* Q2, float* out,
                             const float2* tw, const VcgTw& T) {
  const int ft = a.ft, fh = a.fh, fw = a.fw, La = a.La, Lt = a.Lt, LF = La * fw;
  // w0 -> qt: columns (i, w1, w2)
  dft_stage<5>(nic * LF, Lt, ft, tw + T.ti, LF, LF,
               [&](int c, int& ib, int& ob) { const int i = c / LF, s = c - i * LF; ib = i * a.NF + s; ob = i * ft * LF + s; },
               [&](int i) { return Y[i]; }, [&](int i, float2 v) { Q2[i] = v; });
  __syncthreads();
  // w1 -> qa: columns (i, qt, w2)
  dft_stage<4>(nic * ft * fw, La, fh, tw + T.ai, fw, fw,
               [&](int c, int& ib, int& ob) { const int w2 = c % fw, r = c / fw; ib = r * LF + w2; ob = r * fh * fw + w2; },
               [&](int i) { return Q2[i]; }, [&](int i, float2 v) { Q1[i] = v; });
  __syncthreads();
  // w2 -> qb, the real part (weights folded into the matrix): columns (i, qt, qa)
  dft_stage<4>(nic * ft * fh, fw, fw, tw + T.bi, 1, 1, [&](int c, int& ib, int& ob) { ib = c * fw; ob = c * fw; },
               [&](int i) { return Q1[i]; }, [&](int i, float2 v) { out[i] = v.x; });
  __syncthreads();
}

// y_hat_kj(f) = sum_k' C_hat_kk'(f) p_hat_k'j(f) at the CTA's bins [f0, f0 + nbc) for every item, to yh.
// A thread takes the pair k, k + Kh (Kh = ceil(K / 2)) of one bin, so that each p_hat value it reads
// from shared memory serves six complex products (the loop is bound by the FP32 pipe, not by the
// shared-memory reads); the lanes of a warp take consecutive k (contiguous C_hat reads, broadcast
// p_hat reads). This thread's Parseval terms of p . A p per channel into pa (tmn[k] = 2 mu_k /
// (Lt La Lb)). Does not end synchronised.
template <int J>
__device__ void product_bins(const VcgArgs& a, int f0, int nbc, const float2* ph, int phs, const float* tmn,
                             float (&pa)[J]) {
  const int K = a.K, Kh = (K + 1) / 2;
  for (int e = threadIdx.x; e < nbc * Kh; e += NT) {
    const int bi = e / Kh, k = e - bi * Kh, k2 = k + Kh, f = f0 + bi;
    const bool two = k2 < K;
    const float2* __restrict__ cf = a.chat + (size_t)f * K * K + k;
    const float2* pf = ph + (size_t)bi * phs;
    float2 acc[J], acc2[J];
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = acc2[j] = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int kp = 0; kp < K; ++kp) {
      const float2 c = __ldg(cf + (size_t)kp * K);
      const float2 c2 = two ? __ldg(cf + (size_t)kp * K + Kh) : make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const float2 p = pf[kp * J + j];
        acc[j] = cfma(c, p, acc[j]);
        acc2[j] = cfma(c2, p, acc2[j]);
      }
    }
    const float wt = (f % a.fw == 0) ? 1.f : 2.f;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      a.yh[(size_t)(k * J + j) * a.NF + f] = acc[j];
      const float2 p = pf[k * J + j];
      pa[j] = fmaf(wt, fmaf(acc[j].x, p.x, fmaf(acc[j].y, p.y, tmn[k] * fmaf(p.x, p.x, p.y * p.y))), pa[j]);
      if (two) {
        a.yh[(size_t)(k2 * J + j) * a.NF + f] = acc2[j];
        const float2 q = pf[k2 * J + j];
        pa[j] = fmaf(wt, fmaf(acc2[j].x, q.x, fmaf(acc2[j].y, q.y, tmn[k2] * fmaf(q.x, q.x, q.y * q.y))), pa[j]);
      }
    }
  }
}

// An exchange: every CTA stores its partial sums (vals[0..n), the slot of bank ep & 1) and its data
// (plain stores), then arrives on the counter with release semantics (the barrier before the call
// orders every thread's stores before thread 0's fence); a reader waits until the counter holds all G
// arrivals of exchange ep (acquire), then reads slots and data through L2.
__device__ __forceinline__ void arrive(const VcgArgs& a, const float* vals, int n, unsigned ep) {
  if (threadIdx.x != 0) return;
  float* s = a.slots + ((size_t)(ep & 1) * a.G + blockIdx.x) * kSlotWords;
  for (int i = 0; i < n; ++i) s[i] = vals[i];
  fence_gpu();   // release
  atomicAdd(a.arrivals, 1u);
}

// Waits for the G arrivals of exchange ep (thread 0, bounded: the error word is set when the wait runs
// out or another CTA set it), then in one round trip the slot values ([G][nw] into gv, shared memory)
// and whatever issue() reads of the exchanged data (into the caller's registers); forms the totals of
// the slots in a fixed order (one warp per value), calls then() on thread 0 (the iteration's scalars),
// then consume() on every thread. The scalars stay in float32: the device's float64 rate is a few
// operations per clock per SM, and float64 on the path of every exchange cost microseconds. Ends
// synchronised; false on an error.
template <class ISSUE, class F, class CONSUME>
__device__ bool exchange_in(const VcgArgs& a, unsigned ep, int nw, float* gv, float* tot, int* fail, ISSUE issue,
                            F then, CONSUME consume) {
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
  issue();
  const float* sb = a.slots + (size_t)(ep & 1) * a.G * kSlotWords;
  for (int i = threadIdx.x; i < a.G * nw; i += NT) gv[i] = __ldcg(sb + (size_t)(i / nw) * kSlotWords + i % nw);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < nw; i += NT / 32) {
    float v = 0.f;
    for (int b = lane; b < a.G; b += 32) v += gv[b * nw + i];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) tot[i] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) then();
  __syncthreads();
  consume();
  __syncthreads();
  return true;
}

// z_hat of every item at the CTA's bins (issue: the first U NT values into registers; consume: into
// ph[bi][item], with combine ph = z_hat + beta_j ph)
template <int J, int U>
struct BinsIn {
  float2 v[U];
  __device__ __forceinline__ void load(const VcgArgs& a, int f0, int nbc, int c0) {
    const int n = nbc * a.K * J;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = c0 + threadIdx.x + u * NT;
      if (idx < n) {
        const int item = idx / nbc, bi = idx - item * nbc;
        v[u] = __ldcg(a.zh + (size_t)item * a.NF + f0 + bi);
      }
    }
  }
  __device__ __forceinline__ void store(const VcgArgs& a, int nbc, int c0, float2* ph, int phs, bool combine,
                                        const float* beta) {
    const int n = nbc * a.K * J;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = c0 + threadIdx.x + u * NT;
      if (idx < n) {
        const int item = idx / nbc, bi = idx - item * nbc;
        float2& d = ph[(size_t)bi * phs + item];
        if (combine) {
          const float bt = beta[item % J];
          d = make_float2(fmaf(bt, d.x, v[u].x), fmaf(bt, d.y, v[u].y));
        } else {
          d = v[u];
        }
      }
    }
  }
  __device__ __forceinline__ void consume(const VcgArgs& a, int f0, int nbc, float2* ph, int phs, bool combine,
                                          const float* beta) {
    const int n = nbc * a.K * J;
    store(a, nbc, 0, ph, phs, combine, beta);
    for (int c0 = U * NT; c0 < n; c0 += U * NT) {
      load(a, f0, nbc, c0);
      store(a, nbc, c0, ph, phs, combine, beta);
    }
  }
};

// y_hat of the CTA's items at every bin (issue: the first U NT values; consume: into Y[i][f])
template <int U>
struct ItemsIn {
  float2 v[U];
  __device__ __forceinline__ void load(const VcgArgs& a, int i0, int nic, int c0) {
    const int n = nic * a.NF;
    const float2* src = a.yh + (size_t)i0 * a.NF;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = c0 + threadIdx.x + u * NT;
      if (idx < n) v[u] = __ldcg(src + idx);
    }
  }
  __device__ __forceinline__ void store(const VcgArgs& a, int nic, int c0, float2* Y) {
    const int n = nic * a.NF;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = c0 + threadIdx.x + u * NT;
      if (idx < n) Y[idx] = v[u];
    }
  }
  __device__ __forceinline__ void consume(const VcgArgs& a, int i0, int nic, float2* Y) {
    const int n = nic * a.NF;
    store(a, nic, 0, Y);
    for (int c0 = U * NT; c0 < n; c0 += U * NT) {
      load(a, i0, nic, c0);
      store(a, nic, c0, Y);
    }
  }
};

template <int JT>
__global__ void __launch_bounds__(NT, 1) k_vl_cg(VcgArgs a) {
  extern __shared__ float smf[];
  __shared__ float scratch[(NT / 32) * kSlotWords];
  __shared__ float tot[kSlotWords];
  __shared__ float gvals[kMaxSlotVals];   // the slot values of an exchange, [G][nw]
  __shared__ int s_fail;
  __shared__ double s_mu[kMaxK], s_nrm[kMaxK];
  __shared__ float s_c0[kMaxK], s_tm[kMaxK], s_tmn[kMaxK], s_jac[kMaxK];   // C_kk(0), 2 mu_k, / (Lt La Lb), Jacobi
  __shared__ int s_act[kMaxK];
  __shared__ float s_rz[kMaxJ], s_rr[kMaxJ], s_bb[kMaxJ];
  __shared__ float s_alpha[kMaxJ], s_beta[kMaxJ];
  __shared__ int s_done[kMaxJ], s_all;
  constexpr int J = JT;
  const int K = a.K, KJ = K * J, S3 = a.S3, G = a.G, NF = a.NF;
  const VcgSmem Ls = vcg_layout(K, J, a.ft, a.fh, a.fw, a.Lt, a.La, a.Lb, NF, G);
  const VcgTw Tw = vcg_tw(a.ft, a.fh, a.fw, a.Lt, a.La);
  float2* tw = reinterpret_cast<float2*>(smf + Ls.tw);   // the DFT matrices of the transforms
  float2* ph = reinterpret_cast<float2*>(smf + Ls.ph);   // [nb][phs] p_hat at the CTA's bins
  float2* Y = reinterpret_cast<float2*>(smf + Ls.Y);     // [ni][NF] y_hat of the CTA's items
  float2* Q2 = reinterpret_cast<float2*>(smf + Ls.Q2);
  float2* Q1 = reinterpret_cast<float2*>(smf + Ls.Q1);
  float* X = smf + Ls.X;   // [ni][S3] each: x, r, z, p, b and the operator output of the items
  float* R = smf + Ls.R;
  float* Z = smf + Ls.Z;
  float* P = smf + Ls.P;
  float* B = smf + Ls.B;
  float* T = smf + Ls.T;
  const int f0 = (int)((long long)blockIdx.x * NF / G), nbc = (int)((long long)(blockIdx.x + 1) * NF / G) - f0;
  const int i0 = (int)((long long)blockIdx.x * KJ / G), nic = (int)((long long)(blockIdx.x + 1) * KJ / G) - i0;
  const double invN = 1.0 / ((double)a.Lt * a.La * a.Lb);
  unsigned ep = 0;
  if (threadIdx.x == 0) s_fail = 0;
  {
    const int ft = a.ft, fh = a.fh, fw = a.fw, Lt = a.Lt, La = a.La, Lb = a.Lb;
    for (int e = threadIdx.x; e < fw * fw; e += NT) {
      const int u = e / fw, v = e - u * fw;   // [qb][w2] and [w2][qb]: u v
      tw[Tw.bf + e] = unit_root(u * v, Lb, -1.f);
      const float2 r = unit_root(u * v, Lb, 1.f);
      const float wt = (u == 0) ? 1.f : 2.f;   // u = w2 in [w2][qb]
      tw[Tw.bi + e] = make_float2(wt * r.x, wt * r.y);
    }
    for (int e = threadIdx.x; e < fh * La; e += NT) {
      const int qa = e / La, w1 = e - qa * La;
      tw[Tw.af + e] = unit_root(w1 * qa, La, -1.f);
      tw[Tw.ai + w1 * fh + qa] = unit_root(w1 * qa, La, 1.f);
    }
    for (int e = threadIdx.x; e < ft * Lt; e += NT) {
      const int qt = e / Lt, w0 = e - qt * Lt;
      tw[Tw.tf + e] = unit_root(w0 * qt, Lt, -1.f);
      tw[Tw.ti + w0 * ft + qt] = unit_root(w0 * qt, Lt, 1.f);
    }
  }
  for (int k = threadIdx.x; k < K; k += NT) {
    s_mu[k] = a.mu[k];
    const float c0 = a.lags[((size_t)k * K + k) * a.LLL + a.zero_lag];   // sum of z_k^2 over the codes
    s_c0[k] = c0;
    s_act[k] = a.active[k];
    if (!isfinite(c0)) atomicCAS(a.err, 0, (int)CSC_ERR_NONFINITE);    // a code was not finite
  }
  for (int o = threadIdx.x; o < nic * S3; o += NT) {
    X[o] = a.x[(size_t)i0 * S3 + o];
    B[o] = a.b[(size_t)i0 * S3 + o];
  }
  __syncthreads();
  const float tol2 = (float)a.tol2;
  auto conv_check = [&](bool init) {   // thread 0, after the totals of an exchange Z
    int all = 1;
    bool nonfinite = false;
    for (int j = 0; j < J; ++j) {
      if (init) {
        s_rz[j] = tot[j];
        s_rr[j] = tot[J + j];
        s_bb[j] = tot[2 * J + j];
        s_beta[j] = 0.f;
        s_done[j] = !(s_rr[j] > tol2 * s_bb[j]) || !(s_rz[j] > 0.f);
        if (!isfinite(s_rr[j]) || !isfinite(s_rz[j]) || !isfinite(s_bb[j])) nonfinite = true;
      } else if (!s_done[j]) {
        s_beta[j] = s_rz[j] > 0.f ? tot[j] / s_rz[j] : 0.f;
        s_rz[j] = tot[j];
        s_rr[j] = tot[J + j];
        s_done[j] = !(s_rr[j] > tol2 * s_bb[j]) || !(s_rz[j] > 0.f);
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
  };
  auto nothing = [] {};
  BinsIn<J, 6> bin_in;
  ItemsIn<9> item_in;

  // squared norms of the items (one word each) -> ||d_k|| in every CTA, and with do_mu the multiplier
  // update; the same totals in every CTA
  auto norms_exchange = [&](bool do_mu) -> bool {
    float sq[kItemsMax];
#pragma unroll
    for (int i = 0; i < kItemsMax; ++i) sq[i] = 0.f;
    for (int o = threadIdx.x; o < nic * S3; o += NT) add_at(sq, o / S3, X[o] * X[o]);
    block_reduce_to0<NT>(sq, scratch);
    arrive(a, sq, kItemsMax, ++ep);
    if (!exchange_in(a, ep, kItemsMax, gvals, tot, &s_fail, [] {}, [] {}, [] {})) return false;
    for (int k = threadIdx.x; k < K; k += NT) {
      double n2 = 0.0;
      for (int j = 0; j < J; ++j) {   // item k J + j sits in CTA b at position pos
        const int itm = k * J + j;
        const int b = (int)(((long long)(itm + 1) * G + KJ - 1) / KJ) - 1;
        const int pos = itm - (int)((long long)b * KJ / G);
        n2 += (double)gvals[b * kItemsMax + pos];
      }
      s_nrm[k] = sqrt(n2);
      if (do_mu && s_act[k]) s_mu[k] = fmax(s_mu[k] * s_nrm[k], a.mu_floor);
    }
    __syncthreads();
    return true;
  };

  for (int step = 0; step < a.steps; ++step) {
    for (int k = threadIdx.x; k < K; k += NT) {
      const double m2 = 2.0 * s_mu[k];
      s_tm[k] = (float)m2;
      s_tmn[k] = (float)(m2 * invN);
      s_jac[k] = s_act[k] ? (float)(1.0 / ((double)s_c0[k] + m2)) : 0.f;
    }
    __syncthreads();
    // ---- F(x) on the items; C x at the bins (two exchanges without sums) --------------------
    taps_to_bins(a, i0, nic, X, Q1, Q2, tw, Tw);
    __syncthreads();
    arrive(a, nullptr, 0, ++ep);
    if (!exchange_in(a, ep, 0, gvals, tot, &s_fail, [&] { bin_in.load(a, f0, nbc, 0); }, nothing,
                     [&] { bin_in.consume(a, f0, nbc, ph, Ls.phs, false, s_beta); }))
      return;
    __syncthreads();
    {
      float pa[J];
#pragma unroll
      for (int j = 0; j < J; ++j) pa[j] = 0.f;
      product_bins<J>(a, f0, nbc, ph, Ls.phs, s_tmn, pa);
    }
    __syncthreads();
    arrive(a, nullptr, 0, ++ep);
    // ---- r = b - (C x + 2 mu x), z = M^-1 r, p = z on the items; F(z) with r . z, r . r, b . b ----
    if (!exchange_in(a, ep, 0, gvals, tot, &s_fail, [&] { item_in.load(a, i0, nic, 0); }, nothing,
                     [&] { item_in.consume(a, i0, nic, Y); }))
      return;
    __syncthreads();
    bins_to_taps(a, nic, Y, Q1, Q2, T, tw, Tw);
    {
      float w3[3 * J];
#pragma unroll
      for (int u = 0; u < 3 * J; ++u) w3[u] = 0.f;
      for (int o = threadIdx.x; o < nic * S3; o += NT) {
        const int it = i0 + o / S3, k = it / J, j = it - k * J;
        const bool act = s_act[k] != 0;
        const float bv = B[o];
        const float rv = act ? bv - fmaf(s_tm[k], X[o], T[o]) : 0.f;
        const float zv = rv * s_jac[k];
        R[o] = rv;
        Z[o] = zv;
        P[o] = zv;
        add_at(w3, j, rv * zv);
        add_at(w3, J + j, rv * rv);
        if (act) add_at(w3, 2 * J + j, bv * bv);
      }
      __syncthreads();
      taps_to_bins(a, i0, nic, Z, Q1, Q2, tw, Tw);
      block_reduce_to0<NT>(w3, scratch);
      arrive(a, w3, 3 * J, ++ep);
    }
    if (!exchange_in(a, ep, 3 * J, gvals, tot, &s_fail, [&] { bin_in.load(a, f0, nbc, 0); }, [&] { conv_check(true); },
                     [&] { bin_in.consume(a, f0, nbc, ph, Ls.phs, false, s_beta); }))
      return;
    __syncthreads();
    int it = 0;
    for (; it < a.cg_max; ++it) {
      if (s_all) break;   // the same totals in every CTA
      // ---- y_hat = C_hat p_hat at the bins, p . A p (exchange Y) ------------------------------
      {
        float pa[J];
#pragma unroll
        for (int j = 0; j < J; ++j) pa[j] = 0.f;
        product_bins<J>(a, f0, nbc, ph, Ls.phs, s_tmn, pa);
        block_reduce_to0<NT>(pa, scratch);
        arrive(a, pa, J, ++ep);
      }
      // ---- alpha; x += alpha p, r -= alpha A p, z = M^-1 r on the items; F(z) (exchange Z) -------
      if (!exchange_in(a, ep, J, gvals, tot, &s_fail, [&] { item_in.load(a, i0, nic, 0); },
                       [&] {
                         for (int j = 0; j < J; ++j)
                           s_alpha[j] = (!s_done[j] && tot[j] > 0.f) ? s_rz[j] / tot[j] : 0.f;
                       },
                       [&] { item_in.consume(a, i0, nic, Y); }))
        return;
      bins_to_taps(a, nic, Y, Q1, Q2, T, tw, Tw);
      {
        float w2[2 * J];
#pragma unroll
        for (int u = 0; u < 2 * J; ++u) w2[u] = 0.f;
        for (int o = threadIdx.x; o < nic * S3; o += NT) {
          const int itm = i0 + o / S3, k = itm / J, j = itm - k * J;
          if (!s_act[k]) continue;   // r, z, p stay 0
          const float al = s_alpha[j];
          const float pv = P[o];
          const float apv = fmaf(s_tm[k], pv, T[o]);
          X[o] = fmaf(al, pv, X[o]);
          const float rv = fmaf(-al, apv, R[o]);
          const float zv = rv * s_jac[k];
          R[o] = rv;
          Z[o] = zv;
          add_at(w2, j, rv * zv);
          add_at(w2, J + j, rv * rv);
        }
        __syncthreads();
        taps_to_bins(a, i0, nic, Z, Q1, Q2, tw, Tw);
        block_reduce_to0<NT>(w2, scratch);
        arrive(a, w2, 2 * J, ++ep);
      }
      // ---- beta and convergence; p_hat = z_hat + beta p_hat at the bins, p = z + beta p ----------
      if (!exchange_in(a, ep, 2 * J, gvals, tot, &s_fail, [&] { bin_in.load(a, f0, nbc, 0); }, [&] { conv_check(false); },
                       [&] {
                         bin_in.consume(a, f0, nbc, ph, Ls.phs, true, s_beta);
                         for (int o = threadIdx.x; o < nic * S3; o += NT) P[o] = fmaf(s_beta[(i0 + o / S3) % J], P[o], Z[o]);
                       }))
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.iters) a.iters[step] = it;
    // ---- mu_k <- max(mu_k ||d_k||, floor) for active filters (Eq. mu_update) -------------------
    if (!norms_exchange(true)) return;
  }
  if (a.steps == 0 && !norms_exchange(false)) return;
  // ---- d_k <- d_k / max(1, ||d_k||); x and mu to global ----------------------------------------
  for (int o = threadIdx.x; o < nic * S3; o += NT) {
    const int k = (i0 + o / S3) / J;
    a.x[(size_t)i0 * S3 + o] = X[o] * (float)(1.0 / fmax(1.0, s_nrm[k]));
  }
  if (blockIdx.x == 0)
    for (int k = threadIdx.x; k < K; k += NT) a.mu[k] = s_mu[k];
}

}  // namespace vcg

// ---------------------------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------------------------
using namespace vcg;

// one CTA per SM at most (every CTA must be resident: the exchanges wait on all of them)
static int vcg_ctas(const Ctx& c) { return std::max(1, c.nsm > 0 ? c.nsm : 1); }

static VcgSmem vcg_layout_of(const Ctx& c, int G) {
  const int Lt = 2 * c.ft - 1, La = 2 * c.fh - 1, Lb = 2 * c.fw - 1;
  return vcg_layout(c.K, c.J, c.ft, c.fh, c.fw, Lt, La, Lb, Lt * La * c.fw, G);
}

bool video_cg_applies(const Ctx& c) {
  const int G = vcg_ctas(c);
  return c.K <= kMaxK && c.J >= 1 && c.J <= kMaxJ && (c.K * c.J + G - 1) / G <= kItemsMax &&
         G * std::max(3 * c.J, kItemsMax) <= kMaxSlotVals && vcg_layout_of(c, G).total_floats * sizeof(float) <= kSmemLimit;
}

size_t video_cg_words(const Ctx& c) {   // 8-byte words: z_hat, y_hat (float2 each), the slots, the counter
  const size_t NF = (size_t)(2 * c.ft - 1) * (2 * c.fh - 1) * c.fw;
  return 2 * NF * c.K * c.J + (size_t)vcg_ctas(c) * kSlotWords + 1;
}

cudaError_t launch_video_cg(const Ctx& c, unsigned long long* words, const float* lags, const float2* chat,
                            const float* b, float* x, double* mu, const int* active, int* iters, int steps) {
  VcgArgs a;
  a.K = c.K; a.J = c.J; a.ft = c.ft; a.fh = c.fh; a.fw = c.fw;
  a.Lt = 2 * c.ft - 1; a.La = 2 * c.fh - 1; a.Lb = 2 * c.fw - 1;
  a.S3 = c.ft * c.fh * c.fw; a.NF = a.Lt * a.La * c.fw;
  a.G = vcg_ctas(c); a.steps = steps; a.cg_max = c.p.cg_max;
  a.tol2 = c.p.cg_tol * c.p.cg_tol; a.mu_floor = kMuFloor;
  a.lags = lags; a.LLL = a.Lt * a.La * a.Lb;
  a.zero_lag = ((c.ft - 1) * a.La + (c.fh - 1)) * a.Lb + (c.fw - 1);
  a.chat = chat; a.b = b; a.x = x; a.mu = mu; a.active = active;
  const size_t nw = (size_t)a.NF * c.K * c.J;
  a.zh = reinterpret_cast<float2*>(words);
  a.yh = reinterpret_cast<float2*>(words + nw);
  a.slots = reinterpret_cast<float*>(words + 2 * nw);
  a.arrivals = reinterpret_cast<unsigned*>(words + 2 * nw + (size_t)a.G * kSlotWords);
  a.iters = iters; a.err = c.err;
  a.spin = c.wait_limit > 0 ? c.wait_limit : kSpinLimit;
  if (!video_cg_applies(c)) return cudaErrorInvalidValue;
  // the exchange count restarts at 0 every launch
  cudaError_t e = cudaMemsetAsync(a.arrivals, 0, sizeof(unsigned), c.stream);
  if (e != cudaSuccess) return e;
  auto kern = c.J == 1 ? k_vl_cg<1> : c.J == 2 ? k_vl_cg<2> : k_vl_cg<3>;
  const size_t smem = vcg_layout_of(c, a.G).total_floats * sizeof(float);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(a.G), dim3(NT), args, smem, c.stream);
}

}  // namespace csc
