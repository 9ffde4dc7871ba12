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

__global__ void __launch_bounds__(kGramNT) k_learn_gram(GramArgs a) {
  __shared__ float2 As[kGramT][kGramF];
  __shared__ float2 Bs[kGramT][kGramF];
  // tile pair (ti <= tj) from blockIdx.x
  int ti = 0, rem = blockIdx.x;
  while (rem >= a.ntile - ti) { rem -= a.ntile - ti; ++ti; }
  const int tj = ti + rem;
  const int o0 = blockIdx.y * kGramF;
  const int f = threadIdx.x % kGramF;
  const int grp = threadIdx.x / kGramF;   // 0..7
  const int kq = grp % 4, kpq = grp / 4;  // k rows 4kq..4kq+3, k' rows 8kpq..8kpq+7
  float2 acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) acc[i][jj] = make_float2(0.f, 0.f);
  const int o = o0 + f;
  for (int n = 0; n < a.N; ++n) {
    for (int e = threadIdx.x; e < kGramT * kGramF; e += kGramNT) {
      const int r = e / kGramF, ff = e % kGramF;
      const int oo = o0 + ff;
      const int ka = ti * kGramT + r, kb = tj * kGramT + r;
      As[r][ff] = (ka < a.K && oo < a.Omega) ? a.zhat[((size_t)n * a.K + ka) * a.Omega + oo]
                                              : make_float2(0.f, 0.f);
      Bs[r][ff] = (kb < a.K && oo < a.Omega) ? a.zhat[((size_t)n * a.K + kb) * a.Omega + oo]
                                              : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 av[4], bv[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) av[i] = As[4 * kq + i][f];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) bv[jj] = Bs[8 * kpq + jj][f];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) acc[i][jj] = cfmac(av[i], bv[jj], acc[i][jj]);
    __syncthreads();
  }
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
// bounded grid barrier for the cooperative CG launch
// ---------------------------------------------------------------------------------------------
constexpr long long kSpinLimit = 2000000000LL;   // ~1 s of SM clocks

__device__ bool grid_sync(unsigned* bar, unsigned nblocks, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    int ok = 1;
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      // one polling thread per CTA, no sleep between polls: sleeping added ~20 us per barrier
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (*(volatile int*)err) { ok = 0; break; }
        if (clock64() - t0 > kSpinLimit) { atomicExch(err, (int)CSC_ERR_TIMEOUT); ok = 0; break; }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------------------------
// persistent CG over all learning steps
// ---------------------------------------------------------------------------------------------
struct CgArgs {
  int K, J, fh, fw, S2, La, Lb, G, steps, cg_max;
  double tol2, mu_floor;
  const float* lags;  // [K][K][La*Lb]
  const float* b;     // [K][J][S2]
  float* x;           // [K][J][S2]  d (in/out)
  float* r;           // [K][J][S2]
  float* zv;          // [K][J][S2]  preconditioned residual
  float* Ap;          // [K][J][S2]
  double* mu;         // [K]
  float* minv;        // [K][S2][S2] block-Jacobi inverses (null: scalar Jacobi)
  float* dots;        // [G][4][kMaxJ] per-CTA partial dot products
  unsigned* bar;
  int* iters;         // [steps]
  int* err;
};

__device__ __forceinline__ uint32_t cg_smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// copy n floats of read-only global data into shared memory with asynchronous copies
template <int NT>
__device__ __forceinline__ void stage_async(float* dst, const float* src, int n) {
  for (int i = threadIdx.x; i < n; i += NT)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(cg_smem_addr(dst + i)), "l"(src + i) : "memory");
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
}

// dst[i] = src[i] + beta(i) * dst[i] over the whole vector, src written by other CTAs (read
// through L2), loads batched 8 per thread
template <int NT>
__device__ __forceinline__ void axpy_from_l2(float* dst, const float* src, int n, int JS, int S2,
                                             const float* beta, bool overwrite) {
  for (int i0 = threadIdx.x; i0 < n; i0 += 8 * NT) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = (i0 + u * NT < n) ? __ldcg(src + i0 + u * NT) : 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * NT;
      if (i < n) dst[i] = overwrite ? v[u] : fmaf(beta[(i % JS) / S2], dst[i], v[u]);
    }
  }
  __syncthreads();
}

// y_k = (S Z^T Z S^T) p for filter k (+ 2 mu_k p_k), p in shared memory for all filters. The lag
// blocks C_{k,k'} (La x LB each, contiguous in k') are staged through shared memory in chunks of
// ngroups filters; thread (qa, grp) accumulates output row qa against filter k' = chunk + grp.
template <int SI, int NT>
__device__ void matvec_k(const CgArgs& a, int k, const float* pp, float* red, float* cbuf, float two_mu,
                         float* out) {
  const int fh = a.fh, J = a.J, K = a.K, La = a.La, S2 = a.S2;
  constexpr int LB = 2 * SI - 1;
  const int LL = La * LB;
  const int ngroups = NT / fh;
  const int t = threadIdx.x;
  const bool worker = t < ngroups * fh;
  const int qa = worker ? t % fh : 0, grp = worker ? t / fh : 0;
  float acc[kMaxJ][SI];
#pragma unroll
  for (int j = 0; j < kMaxJ; ++j)
#pragma unroll
    for (int q = 0; q < SI; ++q) acc[j][q] = 0.f;
  for (int kp0 = 0; kp0 < K; kp0 += ngroups) {
    const int nk = min(ngroups, K - kp0);
    stage_async<NT>(cbuf, a.lags + ((size_t)k * K + kp0) * LL, nk * LL);
    if (worker && grp < nk) {
      const int kp = kp0 + grp;
      const float* C = cbuf + (size_t)grp * LL;
      for (int qa2 = 0; qa2 < fh; ++qa2) {
        const float* crow = C + (qa - qa2 + fh - 1) * LB;
        float c[LB];
#pragma unroll
        for (int i = 0; i < LB; ++i) c[i] = crow[i];
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j) {
          if (j < J) {
            const float* prow = pp + ((size_t)kp * J + j) * S2 + qa2 * SI;
            float pv[SI];
#pragma unroll
            for (int i = 0; i < SI; ++i) pv[i] = prow[i];
#pragma unroll
            for (int qb = 0; qb < SI; ++qb)
#pragma unroll
              for (int qb2 = 0; qb2 < SI; ++qb2) acc[j][qb] = fmaf(c[qb - qb2 + SI - 1], pv[qb2], acc[j][qb]);
          }
        }
      }
    }
    __syncthreads();
  }
  if (worker) {
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j)
      if (j < J)
#pragma unroll
        for (int qb = 0; qb < SI; ++qb) red[((grp * fh + qa) * J + j) * SI + qb] = acc[j][qb];
  }
  __syncthreads();
  for (int o = t; o < J * S2; o += NT) {
    const int j = o / S2, q = o - j * S2, qa_ = q / SI, qb = q - qa_ * SI;
    float sum = 0.f;
    for (int gidx = 0; gidx < ngroups; ++gidx) sum += red[((gidx * fh + qa_) * J + j) * SI + qb];
    out[((size_t)k * J + j) * S2 + q] = sum + two_mu * pp[((size_t)k * J + j) * S2 + q];
  }
  __syncthreads();
}

// Sums vals[0..n) over the block in float32 (the device's float64 rate is a few operations per
// clock per SM, so per-thread float64 work is kept out of the CG loop); warp partials go to
// scratch [NT/32][4 kMaxJ], warp 0 finishes, every thread gets the sums back in vals.
template <int NT>
__device__ void block_sum(float* vals, int n, float* scratch) {
  for (int i = 0; i < n; ++i) {
    float v = vals[i];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) scratch[(threadIdx.x >> 5) * 4 * kMaxJ + i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int i = 0; i < n; ++i) {
      float v = (threadIdx.x < NT / 32) ? scratch[threadIdx.x * 4 * kMaxJ + i] : 0.f;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (threadIdx.x == 0) scratch[i] = v;
    }
  }
  __syncthreads();
  for (int i = 0; i < n; ++i) vals[i] = scratch[i];
  __syncthreads();
}

// sum over the G CTAs of slot entries dots[gb][base + j], j < n (written by other CTAs: read
// through L2), in a fixed order by warp 0 in float64, into bcast (shared memory)
template <int NT>
__device__ void grid_dots(const float* dots, int G, int base, int n, double* bcast) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int gb = lane; gb < G; gb += 32) s += (double)__ldcg(dots + (size_t)gb * 4 * kMaxJ + base + j);
      for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
      if (lane == 0) bcast[j] = s;
    }
  }
  __syncthreads();
}

// z_k = M_k^{-1} r_k for one filter, and the partial dot r_k . z_k. M_k is the filter's own block
// of the normal-equation matrix (C_kk Toeplitz + 2 mu_k I, inverted at the start of the call), held
// in shared memory (mloc) when the CTA owns this one filter, else read from a.minv; without
// block inverses, the diagonal. rk is shared-memory scratch of J * S2 floats.
template <int NT>
__device__ void precondition_k(const CgArgs& a, int k, bool act, float sjac, const float* mloc, float* rk,
                               float* part) {
  const int S2 = a.S2, JS = a.J * S2;
  __syncthreads();   // r_k complete
  for (int o = threadIdx.x; o < JS; o += NT) rk[o] = a.r[(size_t)k * JS + o];
  __syncthreads();
  const float* m = mloc ? mloc : (a.minv ? a.minv + (size_t)k * S2 * S2 : nullptr);
  for (int o = threadIdx.x; o < JS; o += NT) {
    const int j = o / S2, q = o - j * S2;
    float zv = 0.f;
    if (act) {
      if (m) {
        // M_k^{-1} is symmetric: column q, consecutive threads on consecutive addresses
        const float* r = rk + (size_t)j * S2;
        float sacc = 0.f;
#pragma unroll 4
        for (int q2 = 0; q2 < S2; ++q2) sacc = fmaf(m[(size_t)q2 * S2 + q], r[q2], sacc);
        zv = sacc;
      } else {
        zv = rk[o] * sjac;
      }
    }
    a.zv[(size_t)k * JS + o] = zv;
    part[1 * kMaxJ + j] = fmaf(rk[o], zv, part[1 * kMaxJ + j]);
  }
}

template <int SI, int NT>
__global__ void __launch_bounds__(NT, 1) k_learn_cg(CgArgs a) {
  extern __shared__ float smf[];
  __shared__ double scratch[(NT / 32) * 4 * kMaxJ];
  __shared__ double bc[4 * kMaxJ];
  // scalars of the iteration, kept by thread 0 (float64) and broadcast through shared memory
  __shared__ double s_rz[kMaxJ], s_rr[kMaxJ], s_bb[kMaxJ];
  __shared__ float s_alpha[kMaxJ], s_beta[kMaxJ], s_twomu, s_jac;
  __shared__ int s_done[kMaxJ], s_all;
  const int K = a.K, J = a.J, S2 = a.S2, G = a.G;
  const int JS = J * S2;
  const int ngroups = NT / a.fh;
  float* pp = smf;                                            // [K][J][S2]
  float* red = pp + (size_t)K * JS;                           // [ngroups][fh][J][SI]
  float* cbuf = red + (size_t)ngroups * a.fh * J * SI;        // [ngroups][La][Lb]
  float* rk = cbuf + (size_t)ngroups * a.La * a.Lb;           // [J][S2]
  float* mloc = rk + JS;                                      // [S2][S2] (+ [S2] during the inversion)
  const bool own_one = (G == K) && a.minv;                    // one filter per CTA: keep its inverse
  const int La = a.La, ctr = (a.fh - 1) * a.Lb + (a.fw - 1);   // lag tau = 0

  auto active = [&](int k) { return a.lags[((size_t)k * K + k) * La * a.Lb + ctr] > 0.f; };
  auto precond = [&](int k) {   // called by one thread
    const double m = (double)a.lags[((size_t)k * K + k) * La * a.Lb + ctr] + 2.0 * a.mu[k];
    return (float)(1.0 / m);
  };

  // ---- block-Jacobi preconditioner for this call: inverse of (C_kk Toeplitz + 2 mu_k I) -------
  // (the mu at entry; the preconditioner need not track the later mu updates exactly)
  if (a.minv) {
    float* A = mloc;                    // [S2][S2]
    float* colv = A + (size_t)S2 * S2;  // [S2]
    const int fh = a.fh, fw = a.fw, Lb = a.Lb;
    for (int k = blockIdx.x; k < K; k += G) {
      const bool act = active(k);
      if (threadIdx.x == 0) s_twomu = (float)(2.0 * a.mu[k]);
      __syncthreads();
      const float tm = s_twomu;
      const float* C = a.lags + ((size_t)k * K + k) * La * Lb;
      for (int e = threadIdx.x; e < S2 * S2; e += NT) {
        const int q = e / S2, q2 = e - q * S2;
        const int qa = q / fw, qb = q - qa * fw, qa2 = q2 / fw, qb2 = q2 - qa2 * fw;
        const float diag = (q == q2) ? 1.f : 0.f;
        A[e] = act ? C[(qa - qa2 + fh - 1) * Lb + (qb - qb2 + fw - 1)] + tm * diag : diag;
      }
      __syncthreads();
      // in-place Gauss-Jordan inversion (symmetric positive definite: no pivoting)
      for (int pv = 0; pv < S2; ++pv) {
        for (int i = threadIdx.x; i < S2; i += NT) colv[i] = A[(size_t)i * S2 + pv];
        __syncthreads();
        const float inv = 1.f / colv[pv];
        for (int j = threadIdx.x; j < S2; j += NT)
          if (j != pv) A[(size_t)pv * S2 + j] *= inv;
        __syncthreads();
        for (int i = threadIdx.x >> 5; i < S2; i += NT / 32) {
          if (i == pv) continue;
          const float ci = colv[i];
          float* row = A + (size_t)i * S2;
          const float* prow = A + (size_t)pv * S2;
          for (int j = threadIdx.x & 31; j < S2; j += 32) row[j] = (j != pv) ? fmaf(-ci, prow[j], row[j]) : -ci * inv;
        }
        if (threadIdx.x == 0) A[(size_t)pv * S2 + pv] = inv;
        __syncthreads();
      }
      if (!own_one) {
        float* dst = a.minv + (size_t)k * S2 * S2;
        for (int e = threadIdx.x; e < S2 * S2; e += NT) dst[e] = A[e];
      }
      __syncthreads();
    }
  }
  const float* mk = own_one ? mloc : nullptr;
  float* fscratch = reinterpret_cast<float*>(scratch);

  for (int step = 0; step < a.steps; ++step) {
    // ---- r = b - A x, z = M^{-1} r, p = z -----------------------------------------------
    axpy_from_l2<NT>(pp, a.x, K * JS, JS, S2, nullptr, true);
    float part[4 * kMaxJ];
    for (int i = 0; i < 4 * kMaxJ; ++i) part[i] = 0.f;
    for (int k = blockIdx.x; k < K; k += G) {
      const bool act = active(k);
      if (threadIdx.x == 0) {
        s_twomu = (float)(2.0 * a.mu[k]);
        s_jac = act ? precond(k) : 0.f;
      }
      __syncthreads();
      matvec_k<SI, NT>(a, k, pp, red, cbuf, s_twomu, a.Ap);
      for (int o = threadIdx.x; o < JS; o += NT) {
        const size_t idx = (size_t)k * JS + o;
        const int j = o / S2;
        const float bv = a.b[idx];
        const float rv = act ? bv - a.Ap[idx] : 0.f;
        a.r[idx] = rv;
        part[2 * kMaxJ + j] = fmaf(rv, rv, part[2 * kMaxJ + j]);
        if (act) part[3 * kMaxJ + j] = fmaf(bv, bv, part[3 * kMaxJ + j]);
      }
      precondition_k<NT>(a, k, act, s_jac, mk, rk, part);
    }
    block_sum<NT>(part, 4 * kMaxJ, fscratch);
    if (threadIdx.x == 0)
      for (int i = 0; i < 4 * kMaxJ; ++i) a.dots[(size_t)blockIdx.x * 4 * kMaxJ + i] = part[i];
    if (!grid_sync(a.bar, G, a.err)) return;
    grid_dots<NT>(a.dots, G, kMaxJ, 3 * kMaxJ, bc);
    if (threadIdx.x == 0)
      for (int j = 0; j < kMaxJ; ++j) {
        s_rz[j] = bc[j];
        s_rr[j] = bc[kMaxJ + j];
        s_bb[j] = bc[2 * kMaxJ + j];
        s_done[j] = (j >= J);
      }
    axpy_from_l2<NT>(pp, a.zv, K * JS, JS, S2, nullptr, true);
    int it = 0;
    for (; it < a.cg_max; ++it) {
      if (threadIdx.x == 0) {
        int all = 1;
        for (int j = 0; j < J; ++j) {
          s_done[j] = s_done[j] || !(s_rr[j] > a.tol2 * s_bb[j]) || !(s_rz[j] > 0.0);
          all = all && s_done[j];
        }
        s_all = all;
      }
      __syncthreads();
      if (s_all) break;
      // ---- Ap, p.Ap --------------------------------------------------------------------
      for (int i = 0; i < 4 * kMaxJ; ++i) part[i] = 0.f;
      for (int k = blockIdx.x; k < K; k += G) {
        const bool act = active(k);
        if (threadIdx.x == 0) s_twomu = (float)(2.0 * a.mu[k]);
        __syncthreads();
        matvec_k<SI, NT>(a, k, pp, red, cbuf, s_twomu, a.Ap);
        for (int o = threadIdx.x; o < JS; o += NT) {
          const size_t idx = (size_t)k * JS + o;
          const int j = o / S2;
          if (act) part[j] = fmaf(pp[idx], a.Ap[idx], part[j]);
        }
      }
      block_sum<NT>(part, kMaxJ, fscratch);
      if (threadIdx.x == 0)
        for (int j = 0; j < kMaxJ; ++j) a.dots[(size_t)blockIdx.x * 4 * kMaxJ + j] = part[j];
      if (!grid_sync(a.bar, G, a.err)) return;
      grid_dots<NT>(a.dots, G, 0, kMaxJ, bc);
      if (threadIdx.x == 0)
        for (int j = 0; j < kMaxJ; ++j) {
          const double pap = bc[j];
          s_alpha[j] = (j < J && !s_done[j] && pap > 0.0) ? (float)(s_rz[j] / pap) : 0.f;
        }
      __syncthreads();
      // ---- x += alpha p, r -= alpha Ap, z = M^{-1} r ---------------------------------------
      for (int i = 0; i < 4 * kMaxJ; ++i) part[i] = 0.f;
      for (int k = blockIdx.x; k < K; k += G) {
        if (!active(k)) continue;
        if (threadIdx.x == 0) s_jac = precond(k);
        __syncthreads();
        for (int o = threadIdx.x; o < JS; o += NT) {
          const size_t idx = (size_t)k * JS + o;
          const int j = o / S2;
          const float al = s_alpha[j];
          a.x[idx] = fmaf(al, pp[idx], a.x[idx]);
          const float rv = fmaf(-al, a.Ap[idx], a.r[idx]);
          a.r[idx] = rv;
          part[2 * kMaxJ + j] = fmaf(rv, rv, part[2 * kMaxJ + j]);
        }
        precondition_k<NT>(a, k, true, s_jac, mk, rk, part);
      }
      block_sum<NT>(part, 4 * kMaxJ, fscratch);
      if (threadIdx.x == 0)
        for (int i = kMaxJ; i < 3 * kMaxJ; ++i) a.dots[(size_t)blockIdx.x * 4 * kMaxJ + i] = part[i];
      if (!grid_sync(a.bar, G, a.err)) return;
      grid_dots<NT>(a.dots, G, kMaxJ, 2 * kMaxJ, bc);
      if (threadIdx.x == 0) {
        for (int j = 0; j < kMaxJ; ++j) {
          if (j < J && !s_done[j]) {
            s_beta[j] = s_rz[j] > 0.0 ? (float)(bc[j] / s_rz[j]) : 0.f;
            s_rz[j] = bc[j];
            s_rr[j] = bc[kMaxJ + j];
          } else {
            s_beta[j] = 0.f;
          }
        }
      }
      __syncthreads();
      // every CTA keeps the whole search direction: p = z + beta p
      axpy_from_l2<NT>(pp, a.zv, K * JS, JS, S2, s_beta, false);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.iters) a.iters[step] = it;
    // ---- mu_k <- max(mu_k ||d_k||, floor) for active filters (Eq. mu_update) ------------------
    for (int k = blockIdx.x; k < K; k += G) {
      float sq[4 * kMaxJ];
      for (int i = 0; i < 4 * kMaxJ; ++i) sq[i] = 0.f;
      for (int o = threadIdx.x; o < JS; o += NT) {
        const float xv = a.x[(size_t)k * JS + o];
        sq[0] = fmaf(xv, xv, sq[0]);
      }
      block_sum<NT>(sq, 1, fscratch);
      if (threadIdx.x == 0 && active(k)) a.mu[k] = fmax(a.mu[k] * sqrt((double)sq[0]), a.mu_floor);
    }
    if (!grid_sync(a.bar, G, a.err)) return;
  }
  // ---- d_k <- d_k / max(1, ||d_k||) ---------------------------------------------------------
  for (int k = blockIdx.x; k < K; k += G) {
    float sq[4 * kMaxJ];
    for (int i = 0; i < 4 * kMaxJ; ++i) sq[i] = 0.f;
    for (int o = threadIdx.x; o < JS; o += NT) {
      const float xv = a.x[(size_t)k * JS + o];
      sq[0] = fmaf(xv, xv, sq[0]);
    }
    block_sum<NT>(sq, 1, fscratch);
    const float sc = 1.0f / fmaxf(1.0f, sqrtf(sq[0]));
    for (int o = threadIdx.x; o < JS; o += NT) a.x[(size_t)k * JS + o] *= sc;
  }
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
cudaError_t launch_learn_rhs(const Ctx& c) { return geo_ops(c).rhs(c); }

cudaError_t launch_learn_gram(const Ctx& c) {
  const int ntile = (c.K + kGramT - 1) / kGramT;
  GramArgs a{c.N, c.K, c.g.Omega, ntile, c.L.zhat, c.L.gram};
  dim3 grid(ntile * (ntile + 1) / 2, (c.g.Omega + kGramF - 1) / kGramF);
  k_learn_gram<<<grid, kGramNT, 0, c.stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_learn_lags(const Ctx& c) { return geo_ops(c).lags(c); }

template <int SI>
static cudaError_t launch_cg_si(const Ctx& c, CgArgs a) {
  constexpr int NT = kNT;
  auto kern = k_learn_cg<SI, NT>;
  const int ngroups = NT / c.fh;
  size_t smem = ((size_t)c.K * c.J * c.S2 + (size_t)ngroups * c.fh * c.J * SI +
                 (size_t)ngroups * (2 * c.fh - 1) * (2 * SI - 1) + (size_t)c.J * c.S2 +
                 (a.minv ? (size_t)c.S2 * c.S2 + c.S2 : 0)) * sizeof(float);
  if (smem > kSmemLimit) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  a.G = std::min(c.K, per_sm * c.nsm);
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(a.G), dim3(NT), args, smem, c.stream);
}

cudaError_t launch_learn_cg(const Ctx& c, float* d, int steps, int* dev_err) {
  CgArgs a;
  a.K = c.K; a.J = c.J; a.fh = c.fh; a.fw = c.fw; a.S2 = c.S2;
  a.La = 2 * c.fh - 1; a.Lb = 2 * c.fw - 1; a.G = 0; a.steps = steps; a.cg_max = c.p.cg_max;
  a.tol2 = c.p.cg_tol * c.p.cg_tol; a.mu_floor = kMuFloor;
  const size_t nvec = (size_t)c.K * c.J * c.S2;
  a.lags = c.L.lags; a.b = c.L.b; a.x = d;
  a.r = c.L.vec; a.zv = c.L.vec + nvec; a.Ap = c.L.vec + 2 * nvec;
  a.mu = c.L.mu; a.minv = c.L.minv; a.dots = c.L.dots; a.bar = c.L.bar; a.iters = c.L.iters; a.err = dev_err;
  cudaError_t e = cudaMemsetAsync(c.L.bar, 0, 2 * sizeof(unsigned), c.stream);
  if (e != cudaSuccess) return e;
  switch (c.fw) {
    case 1: return launch_cg_si<1>(c, a);
    case 3: return launch_cg_si<3>(c, a);
    case 5: return launch_cg_si<5>(c, a);
    case 7: return launch_cg_si<7>(c, a);
    case 9: return launch_cg_si<9>(c, a);
    case 11: return launch_cg_si<11>(c, a);
    case 13: return launch_cg_si<13>(c, a);
    case 15: return launch_cg_si<15>(c, a);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace csc
