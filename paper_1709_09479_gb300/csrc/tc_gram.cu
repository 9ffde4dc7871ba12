// Per-frequency code Gram on the 5th-generation tensor cores.
//
// The learning step needs, for every frequency w, the K x K Hermitian matrix
//     G(w) = Z(w)^H Z(w),   Z(w) in C^{N x K} (the code spectra of N images),
// which is the only dense contraction on the path (a K x N by N x K product per frequency), and the
// right-hand-side spectra R_kj(w) = sum_n conj(z_hat_nk(w)) x_hat_nj(w), which are the same product
// with the J image spectra appended to Z as extra columns.
// With C1 = [Re Z ; Im Z] (2N x K) and C2 = [Im Z ; -Re Z]:
//     Re G = C1^T C1,   Im G = C1^T C2.
//
// The code spectra come frequency-major, zt[w][n K + k], so the N x K values of one frequency are
// one contiguous run. One CTA owns one frequency at a time (persistent over frequencies, two CTAs
// per SM so that one's epilogue overlaps the other's MMAs). The images are taken in chunks of NC:
// all 128 threads load z_hat_nk(w) for the chunk (rows K..K+J-1 from the image spectra x_hat_nj(w);
// rows k >= K + J and images n >= N are zero), split them into tensor-core operands and store them as
// C1^T rows (filters) of [Re over the chunk's images | Im over them] in the canonical no-swizzle
// K-major core-matrix layout.
// One thread then issues tcgen05.mma (M = 128 rows = filters, N = K + J rounded up to 16): the Re G
// accumulator pairs each K-step with itself, the Im G accumulator pairs the Re half of a chunk row
// with its Im half and the Im half with the Re half under the descriptor's negate-B bit, so C2 is
// never materialised. A ring of STAGES chunk buffers lets the loads of chunk i + 1 and the stores of
// later chunks run while the MMAs of chunk i execute; each buffer is released by a tcgen05.commit.
//
// Two operand precisions:
//   X3 = true   float32-accurate 3xTF32 (a.passes = 3), or one TF32 product (a.passes = 1: the
//               CSC_MIXED_TF32 mode): v = hi + lo with hi, lo rounded to TF32 (10 explicit mantissa
//               bits); G accumulates hi.hi + hi.lo + lo.hi in FP32 (kind::tf32). The dropped lo.lo term
//               and the rounding of lo are below 2^-21 relative per product.
//   X3 = false  BF16 operands, FP32 accumulation (kind::f16), the mixed-precision mode.
//
// The epilogue thread of TMEM lane k reads its Re and Im rows with tcgen05.ld and writes G_kk'(w)
// for k <= k' < K, frequency-major with the pairs in column order (gram[w][k'(k'+1)/2 + k], so the
// lanes of a warp store one contiguous run per column k'), and R_kj(w) for the appended columns.
// Every wait on an mbarrier is bounded; on timeout the CTA records CSC_ERR_TIMEOUT, waits (bounded)
// for its own MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "csc_internal.cuh"

namespace csc {

constexpr int kTcThreads = 256;   // warps w and w + 4 share TMEM lane quarter w & 3
constexpr long long kTcSpinLimit = 2000000000LL;
constexpr int kTcRowBytes = 128;                       // one chunk row: [Re | Im] of the chunk's images
constexpr int kTcPieceBytes = 128 * kTcRowBytes;       // 128 rows
constexpr int kTcKSteps = kTcRowBytes / 32;            // 32 bytes (2 core matrices) per MMA K-step
constexpr uint32_t kTcLbo = 128;                       // next core matrix along K
constexpr uint32_t kTcSbo = kTcRowBytes / 16 * 128;    // next group of 8 rows
constexpr int kTcCols = 256;                           // TMEM columns: Re G at 0, Im G at 128

template <bool X3>
struct TcCfg {
  static constexpr int NC = X3 ? 16 : 32;              // images per chunk (element 4 or 2 bytes)
  static constexpr int PIECES = X3 ? 2 : 1;            // hi, lo
  static constexpr int STAGES = 2;                     // operand stages
  static constexpr int RAW = X3 ? 3 : 2;               // raw (float2) chunk stages in flight
  static constexpr int STAGE_BYTES = PIECES * kTcPieceBytes;
};

// raw chunk row stride (float2) for R = K + J rows: >= R and = 8 (mod 16), so that the two
// images of a half-warp's conversion reads fall in opposite halves of the banks
__host__ __device__ constexpr int raw_pitch(int R) { return (R + 7) / 16 * 16 + 8; }

template <bool X3>
size_t gram_tc_smem(int R) {
  using C = TcCfg<X3>;
  return (size_t)C::STAGES * C::STAGE_BYTES + (size_t)C::RAW * C::NC * raw_pitch(R) * sizeof(float2);
}

__device__ __forceinline__ void cp_async8z(void* dst, const void* src, bool valid) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor (tcgen05): start, leading (K-direction core-matrix) byte offset,
// stride (8-row-group) byte offset, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((kTcLbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((kTcSbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D f32 (bits 4-5 = 1), A and B of format fmt (bits 7-9, 10-12; BF16 = 1,
// TF32 = 2), negate-B bit 14, both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28 (M = 128)
__host__ __device__ constexpr uint32_t idesc_mma(uint32_t fmt, int n, bool negate_b) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (negate_b ? (1u << 14) : 0u) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

template <bool X3>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    uint32_t accumulate) {
  if constexpr (X3) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// bounded wait for the completion of phase `parity` of an mbarrier; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kTcSpinLimit) return false;
  }
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

// round to the nearest TF32 value (10 explicit mantissa bits; ties away from zero), kept in a
// float32 container with the 13 low bits clear
// v rounded to the nearest TF32 value (10-bit mantissa, ties away from zero), as a float32 bit
// pattern with the low 13 bits clear; NaN and Inf pass through unchanged
__device__ __forceinline__ float round_tf32(float v) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r & 0xFFFFE000u);
}

struct TcGramArgs {
  int N, K, J, Omega;
  int ntile;                // B rows (MMA N): K + J rounded up to 16, <= 128
  int rows;                 // loaded rows: K + J
  const float2* zt;         // [Omega][N K] frequency-major code spectra
  const float2* xhat;       // [N][J][Omega]
  float2* gram;             // [Omega][np], pair (k <= k') at k'(k'+1)/2 + k
  int np;                   // K (K + 1) / 2
  float2* rspec;            // [K][J][Omega]
  int* err;
  int passes;               // TF32 kernel: 3 (hi.hi + hi.lo + lo.hi, float32-accurate) or 1 (hi.hi: TF32 operands)
};

template <bool X3>
__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(TcGramArgs a) {
  using C = TcCfg<X3>;
  constexpr int NC = C::NC;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t empty_bar[C::STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wq = warp & 3, wh = warp >> 2;
  const int r8 = lane & 7, q4 = lane >> 3;
  const uint32_t tile = smem_addr(smem);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_base)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&empty_bar[s])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&acc_bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&drain_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t acc_re = tmem, acc_im = tmem + 128u;
  constexpr uint32_t fmt = X3 ? 2u : 1u;
  const uint32_t id_pos = idesc_mma(fmt, a.ntile, false), id_neg = idesc_mma(fmt, a.ntile, true);
  const int nchunks = (a.N + NC - 1) / NC;

  // raw chunks: [NC images][RP rows] float2, rows 0..K-1 the codes' spectra, K..K+J-1 the images'
  const int R = a.rows, RP = raw_pitch(R);
  float2* raw = reinterpret_cast<float2*>(smem + C::STAGES * C::STAGE_BYTES);
  const size_t NK = (size_t)a.N * a.K;
  // copies of chunk ch of frequency o into raw stage rs: thread t < R copies row t of every image
  // (one contiguous run of K values per image for the codes); images n >= N are zero-filled
  auto issue_chunk = [&](int o, int ch, int rs) {
    const int k = threadIdx.x & 127;
    if (k < R) {
      float2* dst = raw + (size_t)rs * NC * RP + k;
      const float2* zo = a.zt + (size_t)o * NK + k;
#pragma unroll 4
      for (int nl = threadIdx.x >> 7; nl < NC; nl += 2) {
        const int n = ch * NC + nl;
        const bool v = n < a.N;
        const float2* src = k < a.K ? zo + (size_t)(v ? n : 0) * a.K
                                    : a.xhat + ((size_t)(v ? n : 0) * a.J + (k - a.K)) * a.Omega + o;
        cp_async8z(dst + nl * RP, src, v);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  // element u = 2 uu + wh of this thread's share of a chunk: image 4 (u % (NC/4)) + q4, row
  // 8 kg + r8 with kg = 4 (u / (NC/4)) + wq; a warp's 32 lanes write 32 distinct banks of one
  // core-matrix column
  auto convert_chunk = [&](int rs, int s) {
    const float2* rw = raw + (size_t)rs * NC * RP;
    uint8_t* st = smem + s * C::STAGE_BYTES;
#pragma unroll
    for (int uu = 0; uu < NC / 2; ++uu) {
      const int u = 2 * uu + wh;
      const int nl = 4 * (u % (NC / 4)) + q4;
      const int k = 8 * (4 * (u / (NC / 4)) + wq) + r8;
      const float2 v = k < R ? rw[nl * RP + k] : make_float2(0.f, 0.f);
      const int row = (k >> 3) * (int)kTcSbo + (k & 7) * 16;
      if constexpr (X3) {
        const int cre = nl * 4, cim = (NC + nl) * 4;   // byte columns
        const float hr = round_tf32(v.x), hi = round_tf32(v.y);
        const float lr = round_tf32(v.x - hr), li = round_tf32(v.y - hi);
        uint8_t* p0 = st + row;
        uint8_t* p1 = st + kTcPieceBytes + row;
        *reinterpret_cast<float*>(p0 + (cre >> 4) * kTcLbo + (cre & 15)) = hr;
        *reinterpret_cast<float*>(p0 + (cim >> 4) * kTcLbo + (cim & 15)) = hi;
        *reinterpret_cast<float*>(p1 + (cre >> 4) * kTcLbo + (cre & 15)) = lr;
        *reinterpret_cast<float*>(p1 + (cim >> 4) * kTcLbo + (cim & 15)) = li;
      } else {
        const int cre = nl * 2, cim = (NC + nl) * 2;
        uint8_t* p0 = st + row;
        *reinterpret_cast<__nv_bfloat16*>(p0 + (cre >> 4) * kTcLbo + (cre & 15)) = __float2bfloat16_rn(v.x);
        *reinterpret_cast<__nv_bfloat16*>(p0 + (cim >> 4) * kTcLbo + (cim & 15)) = __float2bfloat16_rn(v.y);
      }
    }
  };

  bool ok = true;
  int nfreq = 0;        // frequencies finished by this CTA
  // this CTA's chunk sequence: (o, ch) for o = blockIdx.x, blockIdx.x + gridDim.x, ..., ch < nchunks
  const int nmine = blockIdx.x < a.Omega ? ((a.Omega - 1 - (int)blockIdx.x) / (int)gridDim.x + 1) : 0;
  const int total = nmine * nchunks;
  auto chunk_o = [&](int i) { return (int)blockIdx.x + (i / nchunks) * (int)gridDim.x; };
  for (int i = 0; i < C::RAW - 1; ++i) {
    if (i < total) issue_chunk(chunk_o(i), i % nchunks, i % C::RAW);
    else asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int it = 0; it < total && ok; ++it) {
    const int o = chunk_o(it), ch = it % nchunks;
    // copies of chunk it + RAW - 1 go into the raw stage that chunk it - 1 used (converted before
    // the last block barrier)
    const int ahead = it + C::RAW - 1;
    if (ahead < total) issue_chunk(chunk_o(ahead), ahead % nchunks, ahead % C::RAW);
    else asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group %0;\n" ::"n"(C::RAW - 1) : "memory");   // chunk it has landed
    __syncthreads();
    const int s = it % C::STAGES;
    if (it >= C::STAGES && !mbar_wait(&empty_bar[s], (uint32_t)((it / C::STAGES - 1) & 1))) ok = false;
    if (ok) convert_chunk(it % C::RAW, s);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    if (__syncthreads_and(ok ? 1 : 0) == 0) { ok = false; break; }
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t base = tile + (uint32_t)(s * C::STAGE_BYTES);
#pragma unroll
      for (int ks = 0; ks < kTcKSteps; ++ks) {
        const int kb = ks < kTcKSteps / 2 ? ks + kTcKSteps / 2 : ks - kTcKSteps / 2;
        const uint32_t idi = ks < kTcKSteps / 2 ? id_pos : id_neg;
#pragma unroll
        for (int c = 0; c < (X3 ? a.passes : 1); ++c) {
          const uint32_t pa = (c == 2) ? kTcPieceBytes : 0u;   // hi.hi, hi.lo, lo.hi
          const uint32_t pb = (c == 1) ? kTcPieceBytes : 0u;
          const uint64_t ad = smem_desc(base + pa + (uint32_t)ks * 2u * kTcLbo);
          const uint64_t bre = smem_desc(base + pb + (uint32_t)ks * 2u * kTcLbo);
          const uint64_t bim = smem_desc(base + pb + (uint32_t)kb * 2u * kTcLbo);
          const uint32_t accum = (ch > 0 || ks > 0 || c > 0) ? 1u : 0u;
          mma<X3>(acc_re, ad, bre, id_pos, accum);
          mma<X3>(acc_im, ad, bim, idi, accum);
        }
      }
      mma_commit(&empty_bar[s]);
      if (ch + 1 == nchunks) mma_commit(&acc_bar);
    }
    if (ch + 1 < nchunks) continue;
    if (!ok) break;
    // epilogue: the frequency's accumulators are complete
    if (!mbar_wait(&acc_bar, (uint32_t)(nfreq & 1))) ok = false;
    ++nfreq;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (__syncthreads_and(ok ? 1 : 0) == 0) { ok = false; break; }
    // warp w reads TMEM lanes 32 (w & 3) .. + 31 (filter k); warps w < 4 take the first half of the
    // 16-column groups, warps w >= 4 the rest
    const int k = 32 * wq + lane;
    const uint32_t lane_off = (uint32_t)(32 * wq) << 16;
    const int ngroups = a.ntile / 16, gsplit = (ngroups + 1) / 2;
    // G_kk'(w) at gram[w][k'(k'+1)/2 + k]: for one column k' the lanes' k are consecutive, so a
    // warp's store is one contiguous run
    float2* gcol = a.gram + (size_t)o * a.np + k;
    float2* rrow = a.rspec + ((long long)k * a.J - a.K) * a.Omega + o;
    for (int gi0 = wh ? gsplit : 0; gi0 < (wh ? ngroups : gsplit); ++gi0) {
      const int c0 = 16 * gi0;
      float gr[16], gim[16];
      tmem_ld16(acc_re + lane_off + (uint32_t)c0, gr);
      tmem_ld16(acc_im + lane_off + (uint32_t)c0, gim);
      if (k < a.K) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int kp = c0 + i;
          if (kp >= k && kp < a.K) gcol[kp * (kp + 1) / 2] = make_float2(gr[i], gim[i]);
          else if (kp >= a.K && kp < a.rows) rrow[(long long)kp * a.Omega] = make_float2(gr[i], gim[i]);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  }
  if (!ok && threadIdx.x == 0) atomicExch(a.err, (int)CSC_ERR_TIMEOUT);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  // drain: every MMA this CTA issued has completed before its TMEM is released
  if (threadIdx.x == 0) mma_commit(&drain_bar);
  if (!mbar_wait(&drain_bar, 0u)) {
    if (threadIdx.x == 0) atomicExch(a.err, (int)CSC_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcCols));
}

// out[o][m] = in[m][o]: 32 x 32 tiles through shared memory (both sides in 256-byte coalesced rows)
constexpr int kTrTile = 32;

__global__ void __launch_bounds__(256) k_spectra_transpose(const float2* __restrict__ in, int nmaps, int Omega,
                                                           float2* __restrict__ out) {
  __shared__ float2 tile[kTrTile][kTrTile + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  const int tiles_o = (Omega + kTrTile - 1) / kTrTile;
  const long long ntiles = (long long)tiles_o * ((nmaps + kTrTile - 1) / kTrTile);
  for (long long tid = blockIdx.x; tid < ntiles; tid += gridDim.x) {
    const int to = (int)(tid % tiles_o), tm = (int)(tid / tiles_o);
    const int o0 = to * kTrTile, m0 = tm * kTrTile;
    __syncthreads();   // the previous tile's reads precede these writes
#pragma unroll
    for (int r = ty; r < kTrTile; r += 8) {
      const int m = m0 + r, o = o0 + tx;
      if (m < nmaps && o < Omega) tile[r][tx] = __ldcs(in + (size_t)m * Omega + o);
    }
    __syncthreads();
#pragma unroll
    for (int r = ty; r < kTrTile; r += 8) {
      const int o = o0 + r, m = m0 + tx;
      if (m < nmaps && o < Omega) out[(size_t)o * nmaps + m] = tile[tx][r];
    }
  }
}

cudaError_t launch_spectra_transpose(const Ctx& c, const float2* in, int nmaps, float2* out) {
  if (nmaps <= 0) return cudaSuccess;
  const long long ntiles = (long long)((c.g.Omega + kTrTile - 1) / kTrTile) * ((nmaps + kTrTile - 1) / kTrTile);
  const int grid = (int)std::min<long long>(ntiles, (long long)c.nsm * 8);
  k_spectra_transpose<<<grid, 256, 0, c.stream>>>(in, nmaps, c.g.Omega, out);
  return cudaGetLastError();
}

bool gram_tc_applies(const Ctx& c) { return c.K + c.J <= 128; }

template <bool X3>
static cudaError_t launch_gram_tc_t(const Ctx& c, float2* rspec, int* dev_err, int passes) {
  const int rows = c.K + c.J;
  const int ntile = (rows + 15) / 16 * 16;
  TcGramArgs a{c.N, c.K, c.J, c.g.Omega, ntile, rows, c.L.zt, c.xhat, c.L.gram, c.K * (c.K + 1) / 2, rspec, dev_err,
               passes};
  // at least 80 KB per CTA keeps at most two CTAs (2 x 256 TMEM columns) per SM
  const int smem = (int)std::max<size_t>(gram_tc_smem<X3>(rows), 80 * 1024);
  cudaError_t e = cudaFuncSetAttribute(k_gram_tc<X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(c.g.Omega, 2 * c.nsm);
  k_gram_tc<X3><<<grid, kTcThreads, smem, c.stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_learn_gram_tc(const Ctx& c, int prec, float2* rspec, int* dev_err) {
  if (!gram_tc_applies(c) || !rspec) return cudaErrorInvalidValue;
  if (prec == CSC_MIXED_BF16) return launch_gram_tc_t<false>(c, rspec, dev_err, 1);
  return launch_gram_tc_t<true>(c, rspec, dev_err, prec == CSC_MIXED_TF32 ? 1 : 3);
}

}  // namespace csc
