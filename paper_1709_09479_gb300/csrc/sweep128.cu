// The coding sweep for grey 128 x 128 images, with the 2-D FFTs fused into the ADMM steps.
//
// Same arithmetic as k_sweep (Eq. Inference_solution: per map, w_k = F^-1(conj(d_hat_k) lambda_hat),
// the state update, u_k = 2 clamp(v_k) - v_k and the accumulation of d_hat_k F(u_k)), with one
// map's spectrum in shared memory. The transforms are laid out so that every thread keeps the same
// few rows, columns and frequencies through the whole map visit and most hand-offs between steps
// stay in registers:
//
//   * the spatial side is the column transform. A real map is read as 64 complex columns
//     z[h][m] = x[h][2m] + i x[h][2m+1]; thread (m, g) holds the 16 rows h = g + 8 j of column m.
//     The last inverse column pass produces exactly these rows, so the state update, u, and the
//     first forward column pass run on registers, with coalesced 8-byte loads and stores of v;
//   * the frequency side is the row transform (64-point complex FFT of each row of Z) followed by
//     the real split. The split pairs bin (kh, kw) with (-kh, 64-kw), so each thread owns two
//     residue classes of kw in two mirrored rows; the accumulation into sum_k d_hat_k u_hat_k, the
//     next map's conj(d_hat_k) lambda_hat and the inverse split all run on that thread's registers;
//   * 128 = 16 x 8 (columns) and 64 = 8 x 8 (rows) Cooley-Tukey passes; every pass writes its
//     outputs over the shared-memory cells it read, so a map visit takes six block barriers.
//
// Per-thread frequency data (d_hat, lambda_hat, the accumulator) use a thread-major order:
// slot s of thread t at s*512 + t (s < 16), the two Nyquist bins of threads t < 64 at
// 8192 + e*64 + t. d_hat is copied into that order once per set of filter spectra (k_permute_dhat).
#include <cuda_runtime.h>

#include <algorithm>

#include "csc_internal.cuh"

namespace csc {
namespace f128 {

constexpr int H = 128, W = 128, D = H * W, P = 65, NT = 512;
constexpr int OM = H * (W / 2 + 1);   // 8320 half-spectrum bins
constexpr int NQ = 64;                 // threads holding Nyquist bins
static_assert(16 * NT + 2 * NQ == OM, "slot layout covers the half spectrum");

// The two (row, residue class of kw mod 8) items of thread t in the row/split phase. Item B is
// the split partner of item A (row -kh, class -k mod 8), except for the four classes that are
// their own partners ((0|64, 0|4)), which threads r = 0 and r = 64 of c = 0 hold two of each.
struct Items {
  int rowA, rowB, kA, kB;
  bool self;
};
CSC_HD Items items_of(int t) {
  const int r = t & 127, c = t >> 7;
  Items it;
  if (c == 0) {
    const bool sp = (r & 63) == 0;
    it.kA = it.kB = (r < 64) ? 0 : 4;
    it.rowA = sp ? 0 : r;
    it.rowB = sp ? 64 : 128 - r;
    it.self = sp;
  } else {
    it.kA = c;
    it.kB = 8 - c;
    it.rowA = r;
    it.rowB = (128 - r) & 127;
    it.self = false;
  }
  return it;
}

// canonical half-spectrum index (kh * 65 + kw) of thread-major position p
CSC_HD int canonical_of(int p) {
  if (p < 16 * NT) {
    const int s = p / NT, t = p % NT;
    const Items it = items_of(t);
    const int j = s & 7;
    return (s < 8) ? it.rowA * 65 + it.kA + 8 * j : it.rowB * 65 + it.kB + 8 * j;
  }
  const int e = (p - 16 * NT) / NQ, t = (p - 16 * NT) % NQ;
  const Items it = items_of(t);
  return (e == 0 ? it.rowA : it.rowB) * 65 + 64;
}

__device__ __forceinline__ float clampb(float v, float b) { return fminf(fmaxf(v, -b), b); }

// pull `bytes` of the next map into L2 while this one is transformed
__device__ __forceinline__ void prefetch_l2_f128(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// forward split of one bin: X = (Za + conj Zb)/2 - i w (Za - conj Zb)/2
__device__ __forceinline__ float2 split_fwd(float2 ya, float2 yb, float2 w) {
  const float2 s = make_float2(ya.x + yb.x, ya.y - yb.y);
  const float2 d = make_float2(ya.x - yb.x, ya.y + yb.y);
  const float2 wd = cmul(w, d);
  return make_float2(0.5f * (s.x + wd.y), 0.5f * (s.y - wd.x));
}
// inverse split (unnormalised): Z = (Xa + conj Xb) + i conj(w) (Xa - conj Xb)
__device__ __forceinline__ float2 split_inv(float2 xa, float2 xb, float2 w) {
  const float2 s = make_float2(xa.x + xb.x, xa.y - xb.y);
  const float2 d = make_float2(xa.x - xb.x, xa.y + xb.y);
  const float2 e = cmulc(d, w);
  return make_float2(s.x - e.y, s.y + e.x);
}

// partner value of value j of an item of class k: the bin (-kh, 64 - kw) in the partner item
// (class 0: j = 0 pairs with the partner's Nyquist bin, j > 0 with value 8 - j; other classes
// with value 7 - j)
template <int J>
__device__ __forceinline__ float2 partner(const float2 (&p)[8], float2 pnyq, bool cls0) {
  return cls0 ? (J == 0 ? pnyq : p[(8 - J) & 7]) : p[7 - J];
}
// the partner's Y value for the forward split (Y is periodic in kw with period 64)
template <int J>
__device__ __forceinline__ float2 partner_y(const float2 (&p)[8], bool cls0) {
  return cls0 ? p[(8 - J) & 7] : p[7 - J];
}

template <int MODE>
__global__ void __launch_bounds__(NT, 1) k_sweep_f128(SweepArgs a, const float2* __restrict__ dhatp) {
  extern __shared__ float2 sm[];
  constexpr bool kLam = (MODE == kIter || MODE == kLast);
  constexpr bool kAcc = (MODE != kLast);
  float2* buf = sm;                                   // [128][P]
  float2* lam = buf + H * P;                          // [OM] thread-major
  float2* acc = lam + (kLam ? OM : 0);                // [OM] thread-major
  float2* T = acc + (kAcc ? OM : 0);                  // [128] exp(-2 pi i m / 128)
  const int t = threadIdx.x;
  for (int i = t; i < H; i += NT) T[i] = a.tw[W / 2 + i];

  // thread roles
  const int wc = t & 63, g = t >> 6;                  // column phase: column m = wc, row block g
  const int r = t & 127, c = t >> 7;                  // row phase
  const Items it = items_of(t);
  const bool nyq = t < NQ;                            // holds the Nyquist bins of both items
  const bool cls0 = (it.kA == 0);

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
#pragma unroll 2
      for (int s = 0; s < 18; ++s) {
        if (s >= 16 && !nyq) break;
        const int p = s < 16 ? s * NT + t : 16 * NT + (s - 16) * NQ + t;
        const int o = canonical_of(p);
        const float2 x = xh[o];
        float2 acc2 = make_float2(-x.x * irho, -x.y * irho);
        for (int cc = c0; cc <= c1; ++cc) acc2 = cadd(acc2, a.part_in[(size_t)(cc + n) * OM + o]);
        const float2 l = cscale(acc2, a.pdiag[o]);
        lam[p] = l;
        if (ls) ls[o] = l;
      }
    }
    if (kAcc) {
#pragma unroll
      for (int s = 0; s < 16; ++s) acc[s * NT + t] = make_float2(0.f, 0.f);
      if (nyq) {
        acc[16 * NT + t] = make_float2(0.f, 0.f);
        acc[16 * NT + NQ + t] = make_float2(0.f, 0.f);
      }
    }

    for (int k = kb; k < ke; ++k) {
      const size_t map = (size_t)n * a.K + k;
      const float2* dk = dhatp + (size_t)k * OM;
      if (threadIdx.x < 4 && (long long)map + 1 < m1) {
        const float* nxt = (MODE == kObjective) ? a.z + (map + 1) * D : a.v + (map + 1) * D;
        prefetch_l2_f128(nxt + threadIdx.x * (D / 4), (unsigned)D);
      }
      float2 zc[16];   // column phase registers: rows h = g + 8 j of column wc
      if (kLam) {
        if (!kAcc) __syncthreads();   // the previous map's column reads precede these writes
        // ---- w_hat = conj(d_hat_k) lambda_hat at this thread's bins; inverse split; first
        //      inverse row pass (8-point, over kw = class + 8 n1) ----
        {
          float2 xa[8], xb[8], na = make_float2(0.f, 0.f), nb = make_float2(0.f, 0.f);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            xa[j] = cmulc(lam[j * NT + t], dk[j * NT + t]);
            xb[j] = cmulc(lam[(8 + j) * NT + t], dk[(8 + j) * NT + t]);
          }
          if (nyq) {
            na = cmulc(lam[16 * NT + t], dk[16 * NT + t]);
            nb = cmulc(lam[16 * NT + NQ + t], dk[16 * NT + NQ + t]);
          }
          float2 za[8], zb[8];
          const bool sf = it.self;
#define CSC_F128_UNSPLIT(J)                                                                       \
  {                                                                                               \
    const float2 pa = sf ? partner<J>(xa, na, cls0) : partner<J>(xb, nb, cls0);                   \
    const float2 pb = sf ? partner<J>(xb, nb, cls0) : partner<J>(xa, na, cls0);                   \
    za[J] = split_inv(xa[J], pa, T[it.kA + 8 * J]);                                               \
    zb[J] = split_inv(xb[J], pb, T[it.kB + 8 * J]);                                               \
  }
          CSC_F128_UNSPLIT(0) CSC_F128_UNSPLIT(1) CSC_F128_UNSPLIT(2) CSC_F128_UNSPLIT(3)
          CSC_F128_UNSPLIT(4) CSC_F128_UNSPLIT(5) CSC_F128_UNSPLIT(6) CSC_F128_UNSPLIT(7)
#undef CSC_F128_UNSPLIT
          dft8<true>(za);
          dft8<true>(zb);
          float2* ra = buf + it.rowA * P + 8 * it.kA;
          float2* rb = buf + it.rowB * P + 8 * it.kB;
          ra[0] = za[0];
          rb[0] = zb[0];
#pragma unroll
          for (int q = 1; q < 8; ++q) {
            ra[q] = cmulc(za[q], T[(2 * it.kA * q) & 127]);
            rb[q] = cmulc(zb[q], T[(2 * it.kB * q) & 127]);
          }
        }
        __syncthreads();
        // ---- second inverse row pass: row r, classes c and c + 4 -> canonical columns m ----
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int k1 = c + 4 * h2;
          float2* row = buf + r * P;
          float2 y[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) y[q] = row[8 * q + k1];
          dft8<true>(y);
#pragma unroll
          for (int q = 0; q < 8; ++q) row[k1 + 8 * q] = y[q];
        }
        __syncthreads();
        // ---- first inverse column pass: column wc, kh = 16 n1 + n2 for n2 = g, g + 8 ----
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int n2 = g + 8 * h2;
          float2 y[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) y[q] = buf[(16 * q + n2) * P + wc];
          dft8<true>(y);
          buf[n2 * P + wc] = y[0];
#pragma unroll
          for (int q = 1; q < 8; ++q) buf[(16 * q + n2) * P + wc] = cmulc(y[q], T[(n2 * q) & 127]);
        }
        __syncthreads();
        // ---- second inverse column pass: rows h = g + 8 j of column wc ----
        float2 vv[16];
        const float* vk = a.v + map * D;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          vv[j] = __ldcs(reinterpret_cast<const float2*>(vk + (g + 8 * j) * W + 2 * wc));
#pragma unroll
        for (int q = 0; q < 16; ++q) zc[q] = buf[(16 * g + q) * P + wc];
        dft16<true>(zc);
        // zc[out_slot<16>(j)] is w at rows h = g + 8 j: state update (and codes on the last sweep)
        float* vw = (a.v_out ? a.v_out : a.v) + map * D;
        float* zk = (MODE == kLast && a.z) ? a.z + map * D : nullptr;
        float2 u[16];
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
            u[j] = make_float2(2.f * clampb(vn.x, beta) - vn.x, 2.f * clampb(vn.y, beta) - vn.y);
          }
        }
        if (kAcc) {
#pragma unroll
          for (int j = 0; j < 16; ++j) zc[j] = u[j];
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
            zc[j] = make_float2(2.f * clampb(x.x, beta) - x.x, 2.f * clampb(x.y, beta) - x.y);
          } else {
            l1f += fabsf(x.x) + fabsf(x.y);
          }
        }
        l1 += (double)l1f;
      }

      if (kAcc) {
        // ---- first forward column pass: 16-point over rows 8 n1 + g, twiddle w128^(g k1) ----
        dft16<false>(zc);
        buf[(16 * g) * P + wc] = zc[out_slot<16>(0)];
#pragma unroll
        for (int k1 = 1; k1 < 16; ++k1) buf[(16 * g + k1) * P + wc] = cmul(zc[out_slot<16>(k1)], T[(g * k1) & 127]);
        __syncthreads();
        // ---- second forward column pass: k1 = g, g + 8 -> canonical rows kh = k1 + 16 k2 ----
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int k1 = g + 8 * h2;
          float2 y[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) y[q] = buf[(16 * q + k1) * P + wc];
          dft8<false>(y);
#pragma unroll
          for (int q = 0; q < 8; ++q) buf[(k1 + 16 * q) * P + wc] = y[q];
        }
        __syncthreads();
        // ---- first forward row pass: row r, n2 = c, c + 4; twiddle w64^(n2 k1) ----
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int n2 = c + 4 * h2;
          float2* row = buf + r * P;
          float2 y[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) y[q] = row[8 * q + n2];
          dft8<false>(y);
          row[n2] = y[0];
#pragma unroll
          for (int q = 1; q < 8; ++q) row[8 * q + n2] = cmul(y[q], T[(2 * n2 * q) & 127]);
        }
        __syncthreads();
        // ---- second forward row pass of items A and B, split, accumulate d_hat_k u_hat ----
        {
          float2 da[8], db[8], dna = make_float2(0.f, 0.f), dnb = make_float2(0.f, 0.f);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            da[j] = __ldg(dk + j * NT + t);
            db[j] = __ldg(dk + (8 + j) * NT + t);
          }
          if (nyq) {
            dna = __ldg(dk + 16 * NT + t);
            dnb = __ldg(dk + 16 * NT + NQ + t);
          }
          float2 ya[8], yb[8];
          const float2* ra = buf + it.rowA * P + 8 * it.kA;
          const float2* rb = buf + it.rowB * P + 8 * it.kB;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            ya[q] = ra[q];
            yb[q] = rb[q];
          }
          dft8<false>(ya);
          dft8<false>(yb);
          const bool sf = it.self;
#define CSC_F128_SPLIT(J)                                                                         \
  {                                                                                               \
    const float2 pa = sf ? partner_y<J>(ya, cls0) : partner_y<J>(yb, cls0);                       \
    const float2 pb = sf ? partner_y<J>(yb, cls0) : partner_y<J>(ya, cls0);                       \
    const float2 xa = split_fwd(ya[J], pa, T[it.kA + 8 * J]);                                     \
    const float2 xb = split_fwd(yb[J], pb, T[it.kB + 8 * J]);                                     \
    acc[J * NT + t] = cfma(da[J], xa, acc[J * NT + t]);                                           \
    acc[(8 + J) * NT + t] = cfma(db[J], xb, acc[(8 + J) * NT + t]);                               \
  }
          CSC_F128_SPLIT(0) CSC_F128_SPLIT(1) CSC_F128_SPLIT(2) CSC_F128_SPLIT(3)
          CSC_F128_SPLIT(4) CSC_F128_SPLIT(5) CSC_F128_SPLIT(6) CSC_F128_SPLIT(7)
#undef CSC_F128_SPLIT
          if (nyq) {
            // kw = 64 (w^64 = -1) of both rows, from their kw = 0 values
            const float2 pa = sf ? ya[0] : yb[0];
            const float2 pb = sf ? yb[0] : ya[0];
            const float2 m1w = make_float2(-1.f, 0.f);
            acc[16 * NT + t] = cfma(dna, split_fwd(ya[0], pa, m1w), acc[16 * NT + t]);
            acc[16 * NT + NQ + t] = cfma(dnb, split_fwd(yb[0], pb, m1w), acc[16 * NT + NQ + t]);
          }
        }
      }
    }
    if (kAcc) {
      float2* dst = a.part_out + (size_t)(cta + n) * OM;
#pragma unroll 2
      for (int s = 0; s < 18; ++s) {
        if (s >= 16 && !nyq) break;
        const int p = s < 16 ? s * NT + t : 16 * NT + (s - 16) * NQ + t;
        dst[canonical_of(p)] = acc[p];
      }
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

__global__ void k_permute_dhat(const float2* __restrict__ in, float2* __restrict__ out, int K) {
  const size_t n = (size_t)K * OM;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t k = i / OM;
    const int p = (int)(i - k * OM);
    out[i] = in[k * OM + canonical_of(p)];
  }
}

size_t smem_bytes(int mode) {
  const bool lam = (mode == kIter || mode == kLast);
  const bool acc = (mode != kLast);
  return ((size_t)H * P + (lam ? OM : 0) + (acc ? OM : 0) + H) * sizeof(float2);
}

template <int MODE>
cudaError_t launch_mode(const Ctx& c, const SweepArgs& a) {
  auto kern = k_sweep_f128<MODE>;
  const size_t smem = smem_bytes(MODE);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<c.G, NT, smem, c.stream>>>(a, c.dhatp);
  return cudaGetLastError();
}

}  // namespace f128

bool fused128_applies(const Ctx& c, const SweepArgs& a) {
  return c.dhatp && c.g.ct_id == 1 && c.J == 1 && a.dhat16 == nullptr && a.vec4;
}

cudaError_t launch_sweep_fused128(const Ctx& c, int mode, const SweepArgs& a) {
  switch (mode) {
    case kPrologue: return f128::launch_mode<kPrologue>(c, a);
    case kIter: return f128::launch_mode<kIter>(c, a);
    case kLast: return f128::launch_mode<kLast>(c, a);
    default: return f128::launch_mode<kObjective>(c, a);
  }
}

cudaError_t launch_permute_dhat128(const Ctx& c) {
  const size_t n = (size_t)c.K * f128::OM;
  const int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)c.nsm * 8);
  f128::k_permute_dhat<<<grid, 256, 0, c.stream>>>(c.dhat, c.dhatp, c.K);
  c.launches += 1;
  return cudaGetLastError();
}

}  // namespace csc
