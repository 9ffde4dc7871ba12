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
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (*(volatile int*)err) { ok = 0; break; }
        if (clock64() - t0 > kSpinLimit) { atomicExch(err, (int)CSC_ERR_TIMEOUT); ok = 0; break; }
        __nanosleep(100);
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
  double* dots;       // [G][4][kMaxJ]
  unsigned* bar;
  int* iters;         // [steps]
  int* err;
};

// y_k = (S Z^T Z S^T) p for filter k (+ 2 mu_k p_k), p in shared memory for all filters
template <int SI, int NT>
__device__ void matvec_k(const CgArgs& a, int k, const float* pp, float* red, float two_mu, float* out) {
  const int fh = a.fh, J = a.J, K = a.K, La = a.La, S2 = a.S2;
  constexpr int LB = 2 * SI - 1;
  const int ngroups = NT / fh;
  const int t = threadIdx.x;
  if (t < ngroups * fh) {
    const int qa = t % fh, grp = t / fh;
    float acc[kMaxJ][SI];
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j)
#pragma unroll
      for (int q = 0; q < SI; ++q) acc[j][q] = 0.f;
    for (int kp = grp; kp < K; kp += ngroups) {
      const float* C = a.lags + ((size_t)k * K + kp) * La * LB;
      for (int qa2 = 0; qa2 < fh; ++qa2) {
        const float* crow = C + (qa - qa2 + fh - 1) * LB;
        float c[LB];
#pragma unroll
        for (int i = 0; i < LB; ++i) c[i] = __ldg(crow + i);
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
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j)
      if (j < J)
#pragma unroll
        for (int qb = 0; qb < SI; ++qb) red[((grp * fh + qa) * J + j) * SI + qb] = acc[j][qb];
  }
  __syncthreads();
  for (int o = t; o < J * S2; o += NT) {
    const int j = o / S2, q = o - j * S2, qa = q / SI, qb = q - qa * SI;
    float s = 0.f;
    for (int gidx = 0; gidx < ngroups; ++gidx) s += red[((gidx * fh + qa) * J + j) * SI + qb];
    out[((size_t)k * J + j) * S2 + q] = s + two_mu * pp[((size_t)k * J + j) * S2 + q];
  }
  __syncthreads();
}

template <int NT>
__device__ void block_sum(double* vals, int n, double* scratch) {
  // sums vals[0..n) across the block; result in vals (thread-local in, block-uniform out)
  for (int i = 0; i < n; ++i) {
    double v = vals[i];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) scratch[(threadIdx.x >> 5) * 4 * kMaxJ + i] = v;
  }
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += scratch[w * 4 * kMaxJ + i];
    vals[i] = s;
  }
  __syncthreads();
}

template <int SI, int NT>
__global__ void __launch_bounds__(NT, 1) k_learn_cg(CgArgs a) {
  extern __shared__ float smf[];
  __shared__ double scratch[(NT / 32) * 4 * kMaxJ];
  const int K = a.K, J = a.J, S2 = a.S2, G = a.G;
  const int JS = J * S2;
  float* pp = smf;                              // [K][J][S2]
  float* red = pp + (size_t)K * JS;             // [ngroups][fh][J][SI]
  const int La = a.La, ctr = (a.fh - 1) * a.Lb + (a.fw - 1);   // lag tau = 0

  auto active = [&](int k) { return a.lags[((size_t)k * K + k) * La * a.Lb + ctr] > 0.f; };
  auto precond = [&](int k) {
    const double m = (double)a.lags[((size_t)k * K + k) * La * a.Lb + ctr] + 2.0 * a.mu[k];
    return (float)(1.0 / m);
  };

  for (int step = 0; step < a.steps; ++step) {
    // ---- r = b - A x, z = M^{-1} r, p = z -----------------------------------------------
    for (int i = threadIdx.x; i < K * JS; i += NT) pp[i] = a.x[i];
    __syncthreads();
    double part[4 * kMaxJ];
    for (int i = 0; i < 4 * kMaxJ; ++i) part[i] = 0.0;
    for (int k = blockIdx.x; k < K; k += G) {
      const bool act = active(k);
      const float two_mu = (float)(2.0 * a.mu[k]);
      matvec_k<SI, NT>(a, k, pp, red, two_mu, a.Ap);
      const float minv = act ? precond(k) : 0.f;
      for (int o = threadIdx.x; o < JS; o += NT) {
        const size_t idx = (size_t)k * JS + o;
        const int j = o / S2;
        const float bv = a.b[idx];
        const float rv = act ? bv - a.Ap[idx] : 0.f;
        const float zv = rv * minv;
        a.r[idx] = rv;
        a.zv[idx] = zv;
        part[1 * kMaxJ + j] += (double)rv * zv;
        part[2 * kMaxJ + j] += (double)rv * rv;
        part[3 * kMaxJ + j] += act ? (double)bv * bv : 0.0;
      }
    }
    block_sum<NT>(part, 4 * kMaxJ, scratch);
    if (threadIdx.x == 0)
      for (int i = 0; i < 4 * kMaxJ; ++i) a.dots[(size_t)blockIdx.x * 4 * kMaxJ + i] = part[i];
    if (!grid_sync(a.bar, G, a.err)) return;
    double rz[kMaxJ], rr[kMaxJ], bb[kMaxJ];
    for (int j = 0; j < J; ++j) {
      rz[j] = rr[j] = bb[j] = 0.0;
      for (int gb = 0; gb < G; ++gb) {
        rz[j] += a.dots[(size_t)gb * 4 * kMaxJ + 1 * kMaxJ + j];
        rr[j] += a.dots[(size_t)gb * 4 * kMaxJ + 2 * kMaxJ + j];
        bb[j] += a.dots[(size_t)gb * 4 * kMaxJ + 3 * kMaxJ + j];
      }
    }
    for (int i = threadIdx.x; i < K * JS; i += NT) pp[i] = a.zv[i];
    __syncthreads();
    int it = 0;
    bool done[kMaxJ];
    for (int j = 0; j < kMaxJ; ++j) done[j] = (j >= J);
    for (; it < a.cg_max; ++it) {
      bool all = true;
      for (int j = 0; j < J; ++j) {
        done[j] = done[j] || !(rr[j] > a.tol2 * bb[j]) || !(rz[j] > 0.0);
        all = all && done[j];
      }
      if (all) break;
      // ---- Ap, p.Ap --------------------------------------------------------------------
      for (int i = 0; i < 4 * kMaxJ; ++i) part[i] = 0.0;
      for (int k = blockIdx.x; k < K; k += G) {
        const bool act = active(k);
        matvec_k<SI, NT>(a, k, pp, red, (float)(2.0 * a.mu[k]), a.Ap);
        for (int o = threadIdx.x; o < JS; o += NT) {
          const size_t idx = (size_t)k * JS + o;
          const int j = o / S2;
          if (act) part[j] += (double)pp[idx] * a.Ap[idx];
        }
      }
      block_sum<NT>(part, kMaxJ, scratch);
      if (threadIdx.x == 0)
        for (int j = 0; j < kMaxJ; ++j) a.dots[(size_t)blockIdx.x * 4 * kMaxJ + j] = part[j];
      if (!grid_sync(a.bar, G, a.err)) return;
      float alpha[kMaxJ];
      for (int j = 0; j < kMaxJ; ++j) {
        double pap = 0.0;
        if (j < J)
          for (int gb = 0; gb < G; ++gb) pap += a.dots[(size_t)gb * 4 * kMaxJ + j];
        alpha[j] = (j < J && !done[j] && pap > 0.0) ? (float)(rz[j] / pap) : 0.f;
      }
      // ---- x += alpha p, r -= alpha Ap, z = M^{-1} r ---------------------------------------
      for (int i = 0; i < 4 * kMaxJ; ++i) part[i] = 0.0;
      for (int k = blockIdx.x; k < K; k += G) {
        if (!active(k)) continue;
        const float minv = precond(k);
        for (int o = threadIdx.x; o < JS; o += NT) {
          const size_t idx = (size_t)k * JS + o;
          const int j = o / S2;
          const float al = alpha[j];
          a.x[idx] = fmaf(al, pp[idx], a.x[idx]);
          const float rv = fmaf(-al, a.Ap[idx], a.r[idx]);
          const float zv = rv * minv;
          a.r[idx] = rv;
          a.zv[idx] = zv;
          part[1 * kMaxJ + j] += (double)rv * zv;
          part[2 * kMaxJ + j] += (double)rv * rv;
        }
      }
      block_sum<NT>(part, 4 * kMaxJ, scratch);
      if (threadIdx.x == 0)
        for (int i = kMaxJ; i < 3 * kMaxJ; ++i) a.dots[(size_t)blockIdx.x * 4 * kMaxJ + i] = part[i];
      if (!grid_sync(a.bar, G, a.err)) return;
      float betav[kMaxJ];
      for (int j = 0; j < kMaxJ; ++j) {
        double rzn = 0.0, rrn = 0.0;
        if (j < J)
          for (int gb = 0; gb < G; ++gb) {
            rzn += a.dots[(size_t)gb * 4 * kMaxJ + 1 * kMaxJ + j];
            rrn += a.dots[(size_t)gb * 4 * kMaxJ + 2 * kMaxJ + j];
          }
        if (j < J && !done[j]) {
          betav[j] = rz[j] > 0.0 ? (float)(rzn / rz[j]) : 0.f;
          rz[j] = rzn;
          rr[j] = rrn;
        } else {
          betav[j] = 0.f;
        }
      }
      // every CTA keeps the whole search direction: p = z + beta p
      for (int i = threadIdx.x; i < K * JS; i += NT) {
        const int j = (i % JS) / S2;
        pp[i] = fmaf(betav[j], pp[i], a.zv[i]);
      }
      __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.iters) a.iters[step] = it;
    // ---- mu_k <- max(mu_k ||d_k||, floor) for active filters (Eq. mu_update) ------------------
    for (int k = blockIdx.x; k < K; k += G) {
      double s[4 * kMaxJ];
      for (int i = 0; i < 4 * kMaxJ; ++i) s[i] = 0.0;
      for (int o = threadIdx.x; o < JS; o += NT) {
        const float xv = a.x[(size_t)k * JS + o];
        s[0] += (double)xv * xv;
      }
      block_sum<NT>(s, 1, scratch);
      if (threadIdx.x == 0 && active(k)) a.mu[k] = fmax(a.mu[k] * sqrt(s[0]), a.mu_floor);
    }
    if (!grid_sync(a.bar, G, a.err)) return;
  }
  // ---- d_k <- d_k / max(1, ||d_k||) ---------------------------------------------------------
  for (int k = blockIdx.x; k < K; k += G) {
    double s[4 * kMaxJ];
    for (int i = 0; i < 4 * kMaxJ; ++i) s[i] = 0.0;
    for (int o = threadIdx.x; o < JS; o += NT) {
      const float xv = a.x[(size_t)k * JS + o];
      s[0] += (double)xv * xv;
    }
    block_sum<NT>(s, 1, scratch);
    const double nrm = sqrt(s[0]);
    const float sc = (float)(1.0 / fmax(1.0, nrm));
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
  const size_t smem = ((size_t)c.K * c.J * c.S2 + (size_t)ngroups * c.fh * c.J * SI) * sizeof(float);
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
  a.mu = c.L.mu; a.dots = c.L.dots; a.bar = c.L.bar; a.iters = c.L.iters; a.err = dev_err;
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
