// Per-frequency code Gram on the 5th-generation tensor cores (mixed-precision learning).
//
// The learning step needs, for every frequency w, the K x K Hermitian matrix
//     G(w) = Z(w)^H Z(w),   Z(w) in C^{N x K} (the code spectra of N images),
// which is the only dense contraction on the path (a K x N by N x K product per frequency).
// With C1 = [Re Z ; Im Z] (2N x K) and C2 = [Im Z ; -Re Z]:
//     Re G = C1^T C1,   Im G = C1^T C2.
// One CTA per frequency (persistent over frequencies) stages C1^T (K rows of 2N bfloat16, K-major)
// in shared memory in the canonical no-swizzle core-matrix layout, and one thread issues
// tcgen05.mma kind::f16 (M = 128 rows = filters, N = K rounded up to 16, K-step 16 = images):
// the Re G accumulator pairs K-step s with itself; the Im G accumulator pairs the Re half of C1^T
// with its Im half and the Im half with the Re half under the descriptor's negate-B bit, so C2 is
// never materialised. Both accumulators sit in the same TMEM lanes (row k), so the epilogue thread
// of row k reads its Re and Im rows with tcgen05.ld and writes G_kk'(w) for k' >= k.
// Waits on the MMA-completion mbarrier are bounded; on timeout the CTA records an error flag, frees
// its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "csc_internal.cuh"

namespace csc {

constexpr int kTcThreads = 128;
constexpr long long kTcSpinLimit = 2000000000LL;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor (tcgen05): start, leading (K-direction core-matrix) byte offset,
// stride (8-row-group) byte offset, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_bf16(int n, bool negate_b) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (negate_b ? (1u << 14) : 0u) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcGramArgs {
  int N, K, Omega;
  int npad;              // N rounded up to 16: each C1^T row holds 2 * npad bf16
  int ntile;             // K rounded up to 16 (MMA N)
  const __nv_bfloat16* zt;  // [Omega][K][2 * npad]  (Re over images, then Im), zero padded
  float2* gram;          // [npairs][Omega]
  int* err;
};

__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(TcGramArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row_bytes = 4 * a.npad;               // 2 * npad bf16
  const int chunks = row_bytes / 16;              // 16-byte chunks per row (core-matrix columns)
  const uint32_t lbo = 128u;                      // next core matrix along K
  const uint32_t sbo = (uint32_t)chunks * 128u;   // next group of 8 rows
  const uint32_t tile = smem_addr(smem);
  constexpr uint32_t kCols = 256;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_base)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t acc_re = tmem, acc_im = tmem + (uint32_t)a.ntile;
  const int ksteps = a.npad / 8;                  // 16 bf16 (two core matrices) per K-step
  const int half = ksteps / 2;
  const uint32_t id_pos = idesc_bf16(a.ntile, false), id_neg = idesc_bf16(a.ntile, true);
  uint32_t phase = 0;
  bool ok = true;

  for (int o = blockIdx.x; o < a.Omega && ok; o += gridDim.x) {
    // stage C1^T rows (filters) of frequency o; rows >= K are zero
    const uint4* src = reinterpret_cast<const uint4*>(a.zt + (size_t)o * a.K * 2 * a.npad);
    for (int i = threadIdx.x; i < 128 * chunks; i += kTcThreads) {
      const int m = i / chunks, c = i - m * chunks;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (m < a.K) val = src[(size_t)m * chunks + c];
      const uint32_t off = (uint32_t)(m >> 3) * sbo + (uint32_t)c * lbo + (uint32_t)(m & 7) * 16u;
      *reinterpret_cast<uint4*>(smem + off) = val;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      for (int s = 0; s < ksteps; ++s) {
        const uint64_t ad = smem_desc(tile + (uint32_t)s * 2u * lbo, lbo, sbo);
        mma_bf16(acc_re, ad, ad, id_pos, s > 0 ? 1u : 0u);
        const int sb = s < half ? s + half : s - half;
        const uint64_t bd = smem_desc(tile + (uint32_t)sb * 2u * lbo, lbo, sbo);
        mma_bf16(acc_im, ad, bd, s < half ? id_pos : id_neg, s > 0 ? 1u : 0u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_addr(&mbar))
                   : "memory");
    }
    // bounded wait for the MMAs of this frequency
    {
      const long long t0 = clock64();
      uint32_t done = 0;
      while (!done) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_addr(&mbar)), "r"(phase)
            : "memory");
        if (!done && clock64() - t0 > kTcSpinLimit) {
          atomicExch(a.err, (int)CSC_ERR_TIMEOUT);
          ok = false;
          break;
        }
      }
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (__syncthreads_and(ok ? 1 : 0) == 0) { ok = false; break; }
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (filter k), 16 columns at a time
    const int k = 32 * warp + lane;
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    for (int c0 = 0; c0 < a.ntile; c0 += 16) {
      float gr[16], gi[16];
      tmem_ld16(acc_re + lane_off + (uint32_t)c0, gr);
      tmem_ld16(acc_im + lane_off + (uint32_t)c0, gi);
      if (k < a.K) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int kp = c0 + i;
          if (kp >= k && kp < a.K) {
            const long long p = (long long)k * a.K - (long long)k * (k - 1) / 2 + (kp - k);
            a.gram[p * a.Omega + o] = make_float2(gr[i], gi[i]);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols));
}

// z_hat [N][K][Omega] float32 -> zt [Omega][K][2*npad] bf16 (Re over images, then Im, zero padded):
// a CTA transposes one filter's 32-frequency slab through shared memory
struct ZtArgs {
  int N, K, Omega, npad;
  const float2* zhat;
  __nv_bfloat16* zt;
};

__global__ void __launch_bounds__(256) k_zt_transpose(ZtArgs a) {
  extern __shared__ float2 slab[];   // [N][32]
  const int k = blockIdx.y;
  const int o0 = blockIdx.x * 32;
  for (int i = threadIdx.x; i < a.N * 32; i += blockDim.x) {
    const int n = i / 32, f = i % 32;
    const int o = o0 + f;
    slab[i] = (o < a.Omega) ? a.zhat[((size_t)n * a.K + k) * a.Omega + o] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int row = 2 * a.npad;
  for (int i = threadIdx.x; i < 32 * row; i += blockDim.x) {
    const int f = i / row, e = i - f * row;
    const int o = o0 + f;
    if (o >= a.Omega) continue;
    const int n = e < a.npad ? e : e - a.npad;
    float v = 0.f;
    if (n < a.N) v = e < a.npad ? slab[n * 32 + f].x : slab[n * 32 + f].y;
    a.zt[((size_t)o * a.K + k) * row + e] = __float2bfloat16_rn(v);
  }
}

size_t tc_gram_smem_bytes(int N) {
  const int npad = (N + 15) / 16 * 16;
  return (size_t)128 * 4 * npad;
}

cudaError_t launch_learn_gram_tc(const Ctx& c, void* zt_buf, int* dev_err) {
  const int npad = (c.N + 15) / 16 * 16;
  const int ntile = (c.K + 15) / 16 * 16;
  __nv_bfloat16* zt = static_cast<__nv_bfloat16*>(zt_buf);
  ZtArgs za{c.N, c.K, c.g.Omega, npad, c.L.zhat, zt};
  dim3 tg((c.g.Omega + 31) / 32, c.K);
  const size_t tsm = (size_t)c.N * 32 * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_zt_transpose, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm);
  if (e != cudaSuccess) return e;
  k_zt_transpose<<<tg, 256, tsm, c.stream>>>(za);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  TcGramArgs a{c.N, c.K, c.g.Omega, npad, ntile, zt, c.L.gram, dev_err};
  // at least 80 KB per CTA keeps two CTAs (2 x 256 TMEM columns) per SM
  size_t smem = tc_gram_smem_bytes(c.N);
  if (smem < 80 * 1024) smem = 80 * 1024;
  if ((e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  const int grid = std::min(c.g.Omega, 2 * c.nsm);
  k_gram_tc<<<grid, kTcThreads, smem, c.stream>>>(a);
  return cudaGetLastError();
}

}  // namespace csc
