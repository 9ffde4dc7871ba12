// Coding subproblem of Sec. 3.2: the dual ADMM of Eq. Inference_solution in the Fourier domain.
//
// With v = D^T lambda^{i+1} - z^i / rho the three updates collapse onto one real state per map:
//     theta = clamp(v), z = rho (clamp(v) - v) (the l1 soft threshold), and the next lambda
//     right-hand side D theta + D z/rho - x/rho = D u - x/rho with u = 2 clamp(v) - v.
// One iteration is therefore, per image n:
//     r_hat  = sum_k d_hat_k F(u_k) - x_hat / rho                 (contraction over the K maps)
//     lam    = (A(w) + I/rho)^{-1} r_hat, A(w) = sum_k d_hat_k d_hat_k^H     (J x J per frequency)
//     w_k    = F^{-1}( sum_j conj(d_hat_jk) lam_j )                (= D_k^T lambda)
//     v_k   <- w_k - (clamp(v_k) - v_k)
// The sweep kernel visits each map once per iteration: it builds w_hat_k from the lambda of the
// previous sweep, inverts it, updates v_k in HBM, forms u_k of the new state, transforms it and
// accumulates d_hat_k F(u_k) into the partial sums that the next sweep turns into lambda.
// A CTA owns a contiguous range of the N*K maps; its partial sums per image go to slot (cta + n),
// and an image's lambda sums the slots of the CTAs covering it in ascending order (deterministic).
#include <cuda_runtime.h>

#include <algorithm>

#include "csc_internal.cuh"

namespace csc {

// ---------------------------------------------------------------------------------------------
// per-frequency system (A(w) + I/rho)^{-1} / D, built in float64 (Sec. 3.2; J x J blocks, Sec. 3.3)
// ---------------------------------------------------------------------------------------------
__device__ void solve_prep_at(const PrepArgs& a, int o) {
  if (a.J == 1) {
    // |d_hat_k|^2 summed in float32 over groups of four filters (relative error below 3e-7 per
    // group), the groups and the reciprocal in float64: the device's float64 rate is a small
    // fraction of its float32 rate, and one float64 add per four filters keeps this pass near its
    // memory time on batches of many size classes
    double s = 1.0 / a.rho;
    int k = 0;
    for (; k + 4 <= a.K; k += 4) {
      float t = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 d = a.dhat[(size_t)(k + q) * a.Omega + o];
        t = fmaf(d.x, d.x, t);
        t = fmaf(d.y, d.y, t);
      }
      s += (double)t;
    }
    for (; k < a.K; ++k) {
      const float2 d = a.dhat[(size_t)k * a.Omega + o];
      s += (double)fmaf(d.x, d.x, d.y * d.y);
    }
    a.pdiag[o] = (float)(a.invD / s);
    return;
  }
  // Hermitian J x J: A_{ij} = sum_k d_ik conj(d_jk) + delta_ij / rho, inverted by Gauss-Jordan
  const int J = a.J;
  double re[kMaxJ][2 * kMaxJ], im[kMaxJ][2 * kMaxJ];
  for (int i = 0; i < J; ++i)
    for (int j = 0; j < 2 * J; ++j) { re[i][j] = 0.0; im[i][j] = 0.0; }
  for (int k = 0; k < a.K; ++k) {
    for (int i = 0; i < J; ++i) {
      const float2 di = a.dhat[((size_t)k * J + i) * a.Omega + o];
      for (int j = 0; j < J; ++j) {
        const float2 dj = a.dhat[((size_t)k * J + j) * a.Omega + o];
        re[i][j] += (double)di.x * dj.x + (double)di.y * dj.y;
        im[i][j] += (double)di.y * dj.x - (double)di.x * dj.y;
      }
    }
  }
  for (int i = 0; i < J; ++i) { re[i][i] += 1.0 / a.rho; re[i][J + i] = 1.0; }
  for (int c = 0; c < J; ++c) {
    // Hermitian positive definite: pivot on the diagonal
    const double pr = re[c][c], pi = im[c][c];
    const double den = pr * pr + pi * pi;
    const double ir = pr / den, ii = -pi / den;
    for (int j = 0; j < 2 * J; ++j) {
      const double xr = re[c][j], xi = im[c][j];
      re[c][j] = xr * ir - xi * ii;
      im[c][j] = xr * ii + xi * ir;
    }
    for (int i = 0; i < J; ++i) {
      if (i == c) continue;
      const double fr = re[i][c], fi = im[i][c];
      for (int j = 0; j < 2 * J; ++j) {
        re[i][j] -= fr * re[c][j] - fi * im[c][j];
        im[i][j] -= fr * im[c][j] + fi * re[c][j];
      }
    }
  }
  float2* out = a.pmat + (size_t)o * J * J;
  for (int i = 0; i < J; ++i)
    for (int j = 0; j < J; ++j)
      out[i * J + j] = make_float2((float)(re[i][J + j] * a.invD), (float)(im[i][J + j] * a.invD));
}

__global__ void k_solve_prep(PrepArgs a) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < a.Omega) solve_prep_at(a, o);
}

// several systems in one launch (the size classes of an uneven batch): system blockIdx.y
__global__ void k_solve_prep_batch(const PrepArgs* list) {
  const PrepArgs a = list[blockIdx.y];
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < a.Omega; o += gridDim.x * blockDim.x) solve_prep_at(a, o);
}

// z = rho (clamp(v) - v) for every element (zero coding iterations)
__global__ void k_codes_from_state(const float* __restrict__ v, float* __restrict__ z, size_t n,
                                   float beta, float rho) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float x = v[i];
    z[i] = rho * (fminf(fmaxf(x, -beta), beta) - x);
  }
}

// per image: sum_j (1/D) sum_w weight(w) |sum_slots partial - x_hat|^2  (Parseval on the half spectrum)
struct ObjFinalArgs {
  int N, K, J, G, H, W, Wc, Omega;
  const float2* part;
  const float2* xhat;
  double* out;
};

__global__ void k_objective_final(ObjFinalArgs a) {
  const int n = blockIdx.x;
  const long long NK = (long long)a.N * a.K;
  const int c0 = (int)((((long long)n * a.K + 1) * a.G - 1) / NK);
  const int c1 = (int)((((long long)(n + 1) * a.K) * a.G - 1) / NK);
  double s = 0.0;
  for (int j = 0; j < a.J; ++j) {
    const float2* xh = a.xhat + ((size_t)n * a.J + j) * a.Omega;
    for (int o = threadIdx.x; o < a.Omega; o += blockDim.x) {
      float2 r = make_float2(-xh[o].x, -xh[o].y);
      for (int c = c0; c <= c1; ++c) r = cadd(r, a.part[((size_t)(c + n) * a.J + j) * a.Omega + o]);
      const int col = o % a.Wc;
      const double wgt = (col == 0 || (2 * col == a.W)) ? 1.0 : 2.0;
      s += wgt * ((double)r.x * r.x + (double)r.y * r.y);
    }
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    a.out[n] = t / ((double)a.H * a.W);
  }
}

// per image: out_n = sum of the partial-sum slots of the CTAs covering image n (ascending order)
struct SumSlotsArgs {
  int N, K, J, G, Omega;
  const float2* part;
  float2* out;   // [N][J][Omega]
};

__global__ void k_sum_slots(SumSlotsArgs a) {
  const int n = blockIdx.y;
  const long long NK = (long long)a.N * a.K;
  const int c0 = (int)((((long long)n * a.K + 1) * a.G - 1) / NK);
  const int c1 = (int)((((long long)(n + 1) * a.K) * a.G - 1) / NK);
  const int JO = a.J * a.Omega;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < JO; i += gridDim.x * blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int c = c0; c <= c1; ++c) s = cadd(s, a.part[(size_t)(c + n) * JO + i]);
    a.out[(size_t)n * JO + i] = s;
  }
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
size_t sweep_smem_bytes(const Geometry& g, int J, int mode) {
  const bool lam = (mode == kIter || mode == kLast);
  const bool acc = (mode != kLast);
  size_t c = (size_t)g.H * g.P + (lam ? (size_t)J * g.Omega : 0) + (acc ? (size_t)J * g.Omega : 0) +
             (size_t)(g.Wh + g.H + g.Wc);
  return c * sizeof(float2);
}

cudaError_t launch_fft_maps(const Ctx& c, const float* in, int nmaps, int filter_mode, float2* out) {
  cudaError_t e = geo_ops(c).fft_maps(c, in, nmaps, filter_mode, out);
  // the fused 128 x 128 sweep reads the filter spectra in its own thread order
  if (e == cudaSuccess && filter_mode == 1 && out == c.dhat && c.dhatp) e = launch_permute_dhat128(c);
  return e;
}

cudaError_t launch_code_spectra(const Ctx& c, const float* in, int nmaps, float2* out) {
  if (c.g.ct_id == 1) return launch_spectra_f128(c, in, nmaps, out);
  return geo_ops(c).fft_maps(c, in, nmaps, 0, out);
}

cudaError_t launch_solve_prep(const Ctx& c) {
  PrepArgs a{c.K, c.J, c.g.Omega, c.p.rho, 1.0 / ((double)c.g.D), c.dhat, c.pdiag, c.pmat};
  k_solve_prep<<<(c.g.Omega + 255) / 256, 256, 0, c.stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_solve_prep_batch(const PrepArgs* list, int n, int max_omega, int nsm, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  // about four resident blocks per SM over all systems
  const int gx = std::max(1, std::min((max_omega + 255) / 256, (4 * nsm + n - 1) / n));
  for (int c0 = 0; c0 < n; c0 += 65535)   // grid y limit
    k_solve_prep_batch<<<dim3(gx, std::min(65535, n - c0)), 256, 0, st>>>(list + c0);
  return cudaGetLastError();
}

cudaError_t launch_sweep(const Ctx& c, int mode, const float2* part_in, float2* part_out, float* v,
                         float* z) {
  return launch_sweep_ex(c, mode, part_in, part_out, v, z, nullptr, nullptr);
}

cudaError_t launch_sweep_ex(const Ctx& c, int mode, const float2* part_in, float2* part_out, float* v,
                            float* z, float* v_out, float2* lam_store) {
  SweepArgs a;
  a.N = c.N; a.K = c.K; a.J = c.J; a.G = c.G;
  a.beta = (float)c.p.beta; a.rho = (float)c.p.rho;
  a.dhat = c.dhat; a.xhat = c.xhat; a.pdiag = c.pdiag; a.pmat = c.pmat;
  a.part_in = part_in; a.part_out = part_out; a.v = v; a.z = z; a.l1 = c.l1; a.tw = c.tw;
  a.v_out = v_out;
  a.lam_store = lam_store;
  a.err = c.cerr;
  a.tf32 = (c.p.precision == CSC_MIXED_TF32 && mode != kObjective) ? 1 : 0;
  // the bf16 copy of d_hat is refreshed by csc_code only; the objective stays float32
  a.dhat16 = (c.p.precision == CSC_MIXED_BF16 && mode != kObjective) ? c.dhat16 : nullptr;
  const bool al = ((uintptr_t)v % 16 == 0) && ((uintptr_t)z % 16 == 0) && ((uintptr_t)v_out % 16 == 0);
  a.vec4 = (al && c.g.D % 16 == 0 && c.g.W % 4 == 0) ? 1 : 0;
  if (fused128_applies(c, a)) return launch_sweep_fused128(c, mode, a);
  return geo_ops(c).sweep(c, mode, a);
}

__global__ void k_to_bf16(const float2* __restrict__ in, __nv_bfloat162* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = __floats2bfloat162_rn(in[i].x, in[i].y);
}

cudaError_t launch_to_bf16(const Ctx& c, const float2* in, __nv_bfloat162* out, size_t n) {
  const int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)c.nsm * 8);
  k_to_bf16<<<grid, 256, 0, c.stream>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_sum_slots(const Ctx& c, const float2* part, float2* out) {
  SumSlotsArgs a{c.N, c.K, c.J, c.G, c.g.Omega, part, out};
  dim3 grid((c.J * c.g.Omega + 255) / 256, c.N);
  k_sum_slots<<<grid, 256, 0, c.stream>>>(a);
  return cudaGetLastError();
}

// the half-sample symmetric extension of each H0 x W0 plane: pixel (h, w) of the 2 H0 x 2 W0 plane
// reads (m(h, H0), m(w, W0)) with m(i, n) = i for i < n and 2 n - 1 - i otherwise
__global__ void k_symmetric_extend(const float* __restrict__ in, float* __restrict__ out, long long planes, int H0,
                                   int W0) {
  const int W = 2 * W0;
  const long long per = 4LL * H0 * W0, n = planes * per;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long pl = i / per;
    const int r = (int)(i - pl * per);
    const int h = r / W, w = r - h * W;
    const int hs = h < H0 ? h : 2 * H0 - 1 - h, ws = w < W0 ? w : 2 * W0 - 1 - w;
    out[i] = in[pl * H0 * W0 + (long long)hs * W0 + ws];
  }
}

cudaError_t launch_symmetric_extend(const Ctx& c, const float* in, float* out) {
  const long long planes = (long long)c.N * c.J;
  const long long n = planes * 4LL * c.H0 * c.W0;
  const int grid = (int)std::min<long long>((n + 255) / 256, (long long)c.nsm * 8);
  k_symmetric_extend<<<grid, 256, 0, c.stream>>>(in, out, planes, c.H0, c.W0);
  return cudaGetLastError();
}

cudaError_t launch_codes_from_state_n(const Ctx& c, const float* v, float* z, size_t n) {
  const int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)c.nsm * 8);
  k_codes_from_state<<<grid, 256, 0, c.stream>>>(v, z, n, (float)c.p.beta, (float)c.p.rho);
  return cudaGetLastError();
}

cudaError_t launch_codes_from_state(const Ctx& c, const float* v, float* z) {
  const size_t n = (size_t)c.N * c.K * c.g.D;
  const int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)c.nsm * 8);
  k_codes_from_state<<<grid, 256, 0, c.stream>>>(v, z, n, (float)c.p.beta, (float)c.p.rho);
  return cudaGetLastError();
}

cudaError_t launch_objective_final(const Ctx& c, const float2* part, double* out_img) {
  ObjFinalArgs a{c.N, c.K, c.J, c.G, c.g.H, c.g.W, c.g.Wc, c.g.Omega, part, c.xhat, out_img};
  k_objective_final<<<c.N, 512, 0, c.stream>>>(a);
  return cudaGetLastError();
}

}  // namespace csc
