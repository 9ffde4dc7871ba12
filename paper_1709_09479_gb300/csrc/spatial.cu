// Direct spatial D and D^T on the 5th-generation tensor cores: the coding iteration of
// Eq. Inference_solution with the two filter products taken as convolutions on the pixel grid, and
// the Fourier domain kept only for the per-frequency solve of the dual variable (one channel per
// image instead of K maps per image).
//
// With the state v of the dual ADMM and u = 2 clamp(v) - v, one iteration is
//   r      = sum_k d_k * u_k                       convolution, K maps -> one channel      (k_sp_conv)
//   lambda = F^-1( P(w) F(r - x / rho) )           P = (sum_k |d_hat_k|^2 + 1/rho)^-1      (k_sp_lambda)
//   w_k    = d_k (x) lambda                        correlation (D^T), one channel -> K maps
//   v     <- w - (clamp(v) - v)                                                            (k_sp_corr)
// which is the Fourier-domain sweep's iteration (its products sum_k d_hat_k u_hat_k and
// conj(d_hat_k) lambda_hat are these convolutions by the convolution theorem), so the two routes
// agree up to rounding. Filter tap (ta, tb) acts at offset (ta - ch, tb - cw), ch = (fh-1)/2,
// cw = (fw-1)/2, circularly on the 128 x 128 grid.
//
// Both filter products are dense contractions over one image row of 128 pixels (the MMA's M = 128
// rows = TMEM lanes):
//   D^T   Wr[p][k] = sum_t A[p][t] d_k[t],   A[p][t] = lambda(h + ta - ch, p + tb - cw):
//         the taps t = ta fw + tb of the row's pixels, gathered from fh rows of lambda;
//   D     Yr[p][t] = sum_k u_k(h, p) d_k[t], then r(h + ta - ch, p + tb - cw) += Yr[p][t]:
//         every input row scatters its products over fh output rows (a shift-add over the taps,
//         done by the thread of each output column in a fixed order).
// Operands are float32 values split as hi + lo (hi rounded to TF32, lo = v - hi read by the MMA as
// TF32) and multiplied as hi.hi + hi.lo + lo.hi (kind::tf32, FP32 accumulation in TMEM):
// float32-accurate, the dropped lo.lo term and the truncation of lo below 2^-20 relative per product.
// The TF32 mode takes hi.hi alone.
//
// Kernel shape (both products): one CTA per SM, persistent over its range of rows, four roles:
//   warps 4-11  producers, two groups of four warps: stage the row's operand chunks (32 contraction
//               elements for D, 64 taps for D^T: every chunk is one hand-off to the MMA warp, the
//               cost that bounds these kernels), split into TF32 hi and lo, in TMEM (the MMA's A
//               operand: lane p = pixel p, one column per element; group g fills the stage of parity
//               g, thread p of a group writes lane p with tcgen05.st), so that shared memory carries
//               only the filter operand (the MMA's B), the state ring and the exchanges;
//   warp 14     lane 0 issues the MMAs of each filled stage (an issuing thread waits for the tensor
//               pipe, so it must not be a producer: the next chunk is built meanwhile);
//   warps 0-3   epilogue: TMEM lane p = pixel p (two accumulators, so the epilogue of row i runs
//               under the MMAs of row i + 1);
//   warp 12     loader of the state v: one TMA tile load of 1 row x 128 pixels per stage (D^T: 16
//               maps, five stages; D: 32 maps, two rings of two, one per producer group), with
//               full/empty mbarriers; boxes further ahead are prefetched into L2;
//   warp 13     loader of the lambda rows of D^T's tiles (double-buffered).
// The filter operand (up to 128 x 128 hi + lo, 128 KB) stays in shared memory for the whole launch.
// Every mbarrier wait is bounded: on timeout the CTA records CSC_ERR_TIMEOUT, stops issuing work,
// waits (under the default bound) for its MMAs and copies in flight and frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "csc_internal.cuh"

namespace csc {
namespace sp {

constexpr int kThreads = 480;                  // epilogue 0-3, producers 4-11, loaders 12-13, MMA 14
constexpr int kProd = 256;                     // producer threads: two per pixel row of a chunk
constexpr int kWarpV = 12, kWarpL = 13;        // loader warps (state, lambda rows)
constexpr int kWarpMma = 14;                   // lane 0 issues every MMA of the CTA
constexpr int kMmaThread = 32 * kWarpMma;
constexpr int kPix = 128;                        // pixels of a row: MMA M, TMEM lanes
constexpr int kAK = 32;                          // contraction elements of D's A chunks (one hand-off, 4 K-steps)
constexpr int kAKDt = 64;                        // ... of D^T's A chunks (its producers read no state: 8 K-steps)
constexpr int kCh = 16;                          // contraction elements of an operand chunk (2 K-steps)
constexpr uint32_t kLbo = 128;                   // next core matrix (8 rows x 16 bytes) along the contraction
constexpr uint32_t kSbo = 512;                   // next group of 8 rows: a chunk row is 64 bytes
constexpr int kAStages = 2;                      // A operand stages (16 KB each)
constexpr int kVStages = 5;                      // state stages in flight (D^T; D has 2 rings of 2)
constexpr int kPrefetch = 24;                    // state boxes fetched into L2 ahead of the ring
constexpr int kVStage = kCh * kPix * 4;          // D^T's state box: 16 maps x 128 pixels
constexpr int kVStageD = kAK * kPix * 4;         // D's state box: 32 maps x 128 pixels (one A chunk)
constexpr int kYsPitch = kCh + 1;                // epilogue exchange of the conv: [2][128 pixels][17]
constexpr int kTmemCols = 512;                   // two accumulators of up to 128 columns, then the A stages
constexpr uint32_t kAColBase = 256;              // A stage s at columns kAColBase + 2 AK s: hi 0..AK-1, lo AK..
constexpr long long kDefaultSpin = 2000000000LL; // ~1 s of SM clocks
constexpr uint32_t kSuspendHintNs = 100000;      // longest suspension of one mbarrier try_wait

// byte offset of (row, contraction element kk < 16) in a chunk block: core matrices of 8 rows x 4
// elements, kLbo apart along the contraction, kSbo apart along the rows
__host__ __device__ __forceinline__ uint32_t cm_off(int row, int kk) {
  return (uint32_t)((row >> 3) * kSbo + (kk >> 2) * kLbo + (row & 7) * 16 + (kk & 3) * 4);
}

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// shared-memory matrix descriptor: start, leading (contraction) and stride (8-row) byte offsets,
// descriptor version 1 (bit 46), no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t a) {
  return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)(kLbo >> 4) << 16) | ((uint64_t)(kSbo >> 4) << 32) |
         ((uint64_t)1 << 46);
}
// instruction descriptor: D f32, A and B TF32, both K-major, N >> 3 at bits 17-22, M = 128
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
// A from TMEM (lane = row, one column per TF32 element), B from shared memory
__device__ __forceinline__ void mma_tf32_ta(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void bar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(bar)), "r"(count));
}
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(saddr(bar)) : "memory");
}
// one arrival per warp once all its lanes are past this point (the consumer barriers count warps:
// 32 arrivals of one warp on one mbarrier would be serialised in the shared-memory unit)
__device__ __forceinline__ void warp_arrive(uint64_t* bar) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) bar_arrive(bar);
}
// bounded wait for the completion of phase `parity`; false on timeout. The waiting thread is
// suspended by the hardware until the phase completes (or the hint expires) rather than spinning, so
// that the warps that wait do not take issue slots from the ones that work
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(saddr(bar)), "r"(parity), "r"(kSuspendHintNs)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}
__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
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
// 16 consecutive TMEM columns of the warp's 32 lanes from registers (no wait)
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
// The producer thread of TMEM lane threadIdx.x % 128 writes its row of an A stage: stage_begin after
// the stage is free (the MMAs that read it have completed), 16 elements at a time with stage_put
// (hi at columns e0.., lo at AK + e0..), stage_end before the mbarrier arrival that hands the stage
// to the MMA issuer
template <int AK>
__device__ __forceinline__ uint32_t stage_begin(uint32_t tmem, int st) {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  return tmem + ((uint32_t)(threadIdx.x & 96) << 16) + kAColBase + (uint32_t)(2 * AK) * (uint32_t)st;
}
template <int AK>
__device__ __forceinline__ void stage_put(uint32_t ta, int e0, const uint32_t* hv, const uint32_t* lv) {
  tmem_st16(ta + (uint32_t)e0, hv);
  tmem_st16(ta + (uint32_t)(AK + e0), lv);
}
__device__ __forceinline__ void stage_end() {
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ float clampb(float v, float b) { return fminf(fmaxf(v, -b), b); }
// the TF32 hi part of the streamed operands: v rounded to 10 explicit mantissa bits, half-way cases
// away from zero, by integer arithmetic on the bit pattern (add half of the lowest kept bit, clear
// the 13 dropped bits; a carry moves into the exponent as it should, Inf and NaN keep their class).
// The lo part v - hi is exact in float32 and is passed as is: the MMA reads its TF32 bits, i.e.
// truncates it, an error below 2^-10 of lo, itself below 2^-11 of v.
__device__ __forceinline__ float tf32_hi(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

// the taps of a filter support known at compile time (FW > 0): tap t = ta fw + tb, padding taps
// t >= fh fw up to the next multiple of 16
template <int FH, int FW>
struct Taps {
  static constexpr int T = FH * FW, TP = (T + 15) / 16 * 16, NCH = TP / 16, NCHA = (TP + kAKDt - 1) / kAKDt,
                       CH = (FH - 1) / 2, CW = (FW - 1) / 2;
  // D^T gather: lambda row offset (row fh is the zero row) and column shift of tap t
  __host__ __device__ static constexpr int row(int t) { return t < T ? (t / FW) * kPix : FH * kPix; }
  __host__ __device__ static constexpr int shift(int t) { return t < T ? t % FW - CW : 0; }
  // D scatter: source pixel shift, whether t closes its filter row, its filter row
  __host__ __device__ static constexpr int src(int t) { return t < T ? CW - t % FW : 0; }
  __host__ __device__ static constexpr bool closes(int t) { return t < T && t % FW == FW - 1; }
  __host__ __device__ static constexpr int ta(int t) { return t / FW; }
};

struct SpArgs {
  int N, K, T, fh, fw;    // images, filters, taps (fh fw), filter support
  int Kp, Tp;             // K and T rounded up to 16
  int passes;             // 3: hi.hi + hi.lo + lo.hi; 1: hi.hi (TF32 operands)
  float beta, rho;
  const uint8_t* bop;     // the launch's filter operand, hi then lo (chunk-major, see k_sp_operands)
  float* v;               // [N][K][128][128] ADMM state
  float* z;               // corr, last iteration: codes (may be null)
  const float* lam;       // corr: [N][128][128] dual variable
  float* r;               // conv: [N][128][128] sum_k d_k * u_k
  int* err;
  long long spin;
};

// the two filter operands from d [K][fh fw]: bt for D^T (rows = filters k < Kp, contraction over
// taps: chunk t / 16 is a [Kp][16] block) and bc for D (rows = taps t < Tp, contraction over
// filters: chunk k / 16 is a [Tp][16] block); each as the hi split followed by the lo split
__global__ void k_sp_operands(const float* __restrict__ d, int K, int T, int Kp, int Tp, uint8_t* bt, uint8_t* bc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Kp * Tp) return;
  const int k = i / Tp, t = i - k * Tp;
  const float x = (k < K && t < T) ? d[(size_t)k * T + t] : 0.f;
  const float hi = tf32r(x), lo = tf32r(x - hi);
  const size_t split = (size_t)Kp * Tp * 4;
  const size_t ot = (size_t)(t >> 4) * Kp * 64 + cm_off(k, t & 15);
  const size_t oc = (size_t)(k >> 4) * Tp * 64 + cm_off(t, k & 15);
  *reinterpret_cast<float*>(bt + ot) = hi;
  *reinterpret_cast<float*>(bt + split + ot) = lo;
  *reinterpret_cast<float*>(bc + oc) = hi;
  *reinterpret_cast<float*>(bc + split + oc) = lo;
}

// TMA bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) into shared memory,
// counted on the mbarrier's transaction count
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(bar))
               : "memory");
}
// TMA tile load of one box of the 3-D tensor map at coordinates (x, y, z) into shared memory
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(saddr(bar))
      : "memory");
}
// the same box fetched into L2 only (no shared memory, no completion to wait for)
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* map, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];\n" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z)
               : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

struct Sync {
  uint64_t a_full[kAStages];    // A stage built by the producer warps
  uint64_t a_empty[kAStages];   // A stage free again (MMA commit)
  uint64_t acc_full[2];         // accumulator complete (MMA commit)
  uint64_t acc_empty[2];        // accumulator read by the 4 epilogue warps
  uint64_t v_full[kVStages];    // state stage landed (the loader's expected bytes)
  uint64_t v_empty[kVStages];   // state stage read by its consumers (epilogue of D^T, producers of D)
  uint64_t l_full[2];           // lambda rows of a tile landed (D^T)
  uint64_t l_empty[2];          // lambda rows read by the producers
  uint64_t drain;
  uint32_t tmem;
};

// start of both product kernels: the filter operand into shared memory (the caller has written
// its own tables before), the mbarriers, TMEM
__device__ __forceinline__ void kernel_begin(const SpArgs& a, uint8_t* sb, size_t bbytes, Sync& s, unsigned v_consumers) {
  const int4* src = reinterpret_cast<const int4*>(a.bop);
  int4* dst = reinterpret_cast<int4*>(sb);
  for (size_t i = threadIdx.x; i < bbytes / 16; i += kThreads) dst[i] = __ldg(src + i);
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(&s.tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 32) {
    for (int i = 0; i < 2; ++i) {
      bar_init(&s.acc_full[i], 1);
      bar_init(&s.acc_empty[i], 4);        // epilogue warps
      bar_init(&s.l_full[i], 1);
      bar_init(&s.l_empty[i], kProd / 32);  // producer warps
    }
    for (int i = 0; i < kAStages; ++i) {
      bar_init(&s.a_full[i], kProd / 64);   // the warps of one producer group
      bar_init(&s.a_empty[i], 1);
    }
    for (int i = 0; i < kVStages; ++i) {
      bar_init(&s.v_full[i], 1);
      bar_init(&s.v_empty[i], v_consumers);   // consumer warps
    }
    bar_init(&s.drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// every MMA of the CTA has completed before its TMEM is released (the drain keeps the default bound
// whatever the context's wait limit); a timeout anywhere is recorded
__device__ __forceinline__ void kernel_end(const SpArgs& a, Sync& s, bool ok) {
  if (threadIdx.x == kMmaThread) {
    commit(&s.drain);
    if (!bar_wait(&s.drain, 0u, kDefaultSpin)) ok = false;
  }
  if (!ok) atomicExch(a.err, (int)CSC_ERR_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(s.tmem), "r"(kTmemCols));
}

// the MMAs of one A chunk (nks K-steps of 8 elements x passes) into accumulator acc; B's K-step ks of
// the chunk lies in its 16-element block bblk0 + ks / 2 (blocks blk bytes apart). The commit frees
// the A stage, and after the row's last chunk marks the accumulator complete
template <int AK>
__device__ __forceinline__ void issue_chunk(const SpArgs& a, Sync& s, bool ok, uint32_t acc, uint32_t astage,
                                            uint32_t bblk0, uint32_t blk, int nks, uint32_t bsplit, uint32_t id,
                                            bool first, int st, bool last, int accb) {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok) {
#pragma unroll
    for (int ks = 0; ks < AK / 8; ++ks) {
      if (ks >= nks) break;
      const uint32_t b = bblk0 + (uint32_t)(ks >> 1) * blk + (uint32_t)(ks & 1) * 2u * kLbo;
      for (int ps = 0; ps < a.passes; ++ps) {
        const uint32_t pa = (ps == 2) ? (uint32_t)AK : 0u;   // hi.hi, hi.lo, lo.hi
        const uint32_t pb = (ps == 1) ? bsplit : 0u;
        mma_tf32_ta(acc, astage + pa + (uint32_t)ks * 8u, sdesc(b + pb), id, (first && ks == 0 && ps == 0) ? 0u : 1u);
      }
    }
  }
  commit(&s.a_empty[st]);
  if (last) commit(&s.acc_full[accb]);
}

// lane 0 of the MMA warp: every A chunk of every row tile once the producers have filled its stage
// (and, for a row's first chunk, once the epilogue has emptied the accumulator it reuses). The
// contraction has kdim elements (a multiple of 16): chunk c covers AK of them from AK c; the filter
// operand's 16-element blocks are blk bytes apart from sb0
template <int AK>
__device__ __forceinline__ void mma_loop(const SpArgs& a, Sync& s, bool& ok, uint32_t tmem, uint32_t sb0,
                                         uint32_t blk, int kdim, uint32_t id, int ntiles, int nch) {
  const uint32_t bsplit = (uint32_t)(a.Kp * a.Tp * 4);
  for (int i = 0; i < ntiles; ++i) {
    for (int c = 0; c < nch; ++c) {
      const int q = i * nch + c, st = q % kAStages;
      if (ok) ok = bar_wait(&s.a_full[st], (uint32_t)((q / kAStages) & 1), a.spin);
      if (c == 0 && i >= 2 && ok) ok = bar_wait(&s.acc_empty[i & 1], (uint32_t)(((i >> 1) - 1) & 1), a.spin);
      const int nks = min(AK, kdim - AK * c) / 8;
      issue_chunk<AK>(a, s, ok, tmem + (uint32_t)((i & 1) * 128), tmem + kAColBase + (uint32_t)(2 * AK) * (uint32_t)st,
                      sb0 + (uint32_t)(c * (AK / kCh)) * blk, blk, nks, bsplit, id, c == 0, st, c == nch - 1, i & 1);
    }
  }
}

// The state ring as RINGS rings of PER stages: item q goes to ring q % RINGS, which one consumer group
// reads in item order. A consumer must never wait for a stage's next phase before it has waited for
// the current one (an mbarrier parity wait cannot tell the two apart, and the loads of different
// items may land out of order), so consumer groups that take alternate items get a ring each.
template <int RINGS, int PER>
struct Ring {
  static constexpr int STAGES = RINGS * PER;
  __device__ static int stage(int q) { return (q % RINGS) * PER + (q / RINGS) % PER; }
  __device__ static int phase(int q) { return (q / RINGS) / PER; }
};
using RingDt = Ring<1, kVStages>;   // D^T: the four epilogue warps read every item
using RingD = Ring<2, 2>;           // D: producer group g reads the items of parity g

// lane 0 of the state loader warp: the state rows of every item, in item order, into the ring (item
// q = row tile q / groups, maps MAPS (q % groups) ..; tile_row(i) gives the tile's image n and row
// h): one TMA box of MAPS maps x 1 row x 128 pixels of the tensor map vmap over v viewed as
// [N K][128][128] (maps past the image's K belong to the next image, or lie past the end and read as
// zeros; their values are never used). A stage is refilled only after its consumers released it, so
// every copy lands in a free stage and completes the phase it was counted in; when a wait gives up
// the loader issues nothing more. The boxes kPrefetch items ahead are fetched into L2 meanwhile (the
// ring alone holds too few bytes to cover the latency of HBM). Before returning it waits (under the
// default bound) for the copies of the last stages it filled, so that none is in flight when the CTA
// ends.
template <class R, int MAPS, class TileRow>
__device__ __forceinline__ void load_states(const SpArgs& a, Sync& s, const CUtensorMap* vmap, float* vring,
                                            int nitems, int groups, TileRow tile_row, bool& ok) {
  auto box = [&](int q, int& h, int& z) {
    const int i = q / groups, k0 = (q - i * groups) * MAPS;
    int n;
    tile_row(i, n, h);
    z = n * a.K + k0;
  };
  for (int q = 0; q < min(kPrefetch, nitems); ++q) {
    int h, z;
    box(q, h, z);
    tma_prefetch_3d(vmap, 0, h, z);
  }
  int issued = 0;
  for (int q = 0; q < nitems; ++q) {
    const int st = R::stage(q), ph = R::phase(q);
    if (ph >= 1) ok = ok && bar_wait(&s.v_empty[st], (uint32_t)((ph - 1) & 1), a.spin);
    if (!ok) break;
    int h, z;
    box(q, h, z);
    bar_expect(&s.v_full[st], (uint32_t)(MAPS * kPix * 4));
    tma_load_3d(vring + (size_t)st * MAPS * kPix, vmap, 0, h, z, &s.v_full[st]);
    issued = q + 1;
    if (q + kPrefetch < nitems) {
      box(q + kPrefetch, h, z);
      tma_prefetch_3d(vmap, 0, h, z);
    }
  }
  for (int q = max(issued - R::STAGES, 0); q < issued; ++q)
    bar_wait(&s.v_full[R::stage(q)], (uint32_t)(R::phase(q) & 1), kDefaultSpin);
}

// ---- D^T and the state update: one tile = one image row (n, h) -----------------------------------
// shared memory: filter operand bt | A stages [2][hi | lo] | state ring | lambda rows [2][fh + 1][128]
// (row fh stays zero: the padding taps read it) | tap table (row offset, column shift)
template <bool LAST, int FH, int FW>
__global__ void __launch_bounds__(kThreads, 1) k_sp_corr(SpArgs a, const __grid_constant__ CUtensorMap vmap) {
  using CT = Taps<FH, FW>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ Sync s;
  const int warp = threadIdx.x >> 5;
  const int nch = (a.Tp + kAKDt - 1) / kAKDt, NG = a.Kp / kCh, TA = nch * kAKDt;
  const size_t bbytes = (size_t)2 * a.Kp * a.Tp * 4;
  uint8_t* sb = smem;
  float* vring = reinterpret_cast<float*>(sb + bbytes);
  float* lbuf = vring + kVStages * kCh * kPix;
  const int lrows = a.fh + 1;
  int* tap_a = reinterpret_cast<int*>(lbuf + 2 * lrows * kPix);
  int* tap_b = tap_a + TA;
  const int ch = (a.fh - 1) / 2, cw = (a.fw - 1) / 2;
  for (int t = threadIdx.x; t < TA; t += kThreads) {
    const int ta = t / a.fw, tb = t - ta * a.fw;
    tap_a[t] = t < a.T ? ta * kPix : a.fh * kPix;
    tap_b[t] = t < a.T ? tb - cw : 0;
  }
  for (int i = threadIdx.x; i < 2 * kPix; i += kThreads) lbuf[((i >> 7) * lrows + a.fh) * kPix + (i & 127)] = 0.f;
  kernel_begin(a, sb, bbytes, s, 4);
  const uint32_t tmem = s.tmem;
  const int NH = a.N * kPix;
  const int t0 = (int)((long long)blockIdx.x * NH / gridDim.x);
  const int t1 = (int)((long long)(blockIdx.x + 1) * NH / gridDim.x);
  const int ntiles = t1 - t0;
  const size_t plane = (size_t)kPix * kPix;
  auto tile_row = [&](int i, int& n, int& h) {
    const int tile = t0 + i;
    n = tile / kPix;
    h = tile - n * kPix;
  };
  bool ok = true;

  if (warp >= 4 && warp < kWarpV) {
    // producers: group g (warps 4-7: g = 0, warps 8-11: g = 1) builds the chunks of A stage g (every
    // other chunk); thread p of a group builds row p (pixel p) of its chunks from the tile's lambda rows
    const int pp = threadIdx.x - 128, p = pp & (kPix - 1), grp = pp >> 7;
    for (int i = 0; i < ntiles; ++i) {
      const int b = i & 1;
      if (ok) ok = bar_wait(&s.l_full[b], (uint32_t)((i >> 1) & 1), a.spin);
      const float* lb = lbuf + b * lrows * kPix;
      auto chunk = [&](int c, auto tap) {
        const int q = i * nch + c, st = q % kAStages;
        if (st != grp) return;
        if (q >= kAStages && ok) ok = bar_wait(&s.a_empty[st], (uint32_t)(((q / kAStages) - 1) & 1), a.spin);
        const uint32_t ta = stage_begin<kAKDt>(tmem, st);
#pragma unroll
        for (int e0 = 0; e0 < kAKDt; e0 += 16) {
          uint32_t hv[16], lv[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float x = tap(c * kAKDt + e0 + e);
            const float h = tf32_hi(x);
            hv[e] = __float_as_uint(h);
            lv[e] = __float_as_uint(x - h);
          }
          stage_put<kAKDt>(ta, e0, hv, lv);
        }
        stage_end();
        warp_arrive(&s.a_full[st]);
      };
      if constexpr (FW > 0) {
        // compile-time taps: every gather address is p plus constants
#pragma unroll
        for (int c = 0; c < CT::NCHA; ++c)
          chunk(c, [&](int t) { return lb[CT::row(t) + ((p + CT::shift(t)) & (kPix - 1))]; });
      } else {
        for (int c = 0; c < nch; ++c) chunk(c, [&](int t) { return lb[tap_a[t] + ((p + tap_b[t]) & (kPix - 1))]; });
      }
      warp_arrive(&s.l_empty[b]);   // this group's reads of the tile's lambda rows are done
    }
  } else if (warp == kWarpMma) {
    if ((threadIdx.x & 31) == 0)
      mma_loop<kAKDt>(a, s, ok, tmem, saddr(sb), (uint32_t)(a.Kp * 64), a.Tp, idesc_tf32(a.Kp), ntiles, nch);
    __syncwarp();
  } else if (warp == kWarpV) {
    if ((threadIdx.x & 31) == 0) load_states<RingDt, kCh>(a, s, &vmap, vring, ntiles * NG, NG, tile_row, ok);
    __syncwarp();
  } else if (warp == kWarpL) {
    // lane 0: the fh lambda rows of every tile (rows h + ta - ch, circularly)
    if ((threadIdx.x & 31) == 0) {
      int issued = 0;   // as for the state loader: nothing more after a wait gave up
      for (int i = 0; i < ntiles; ++i) {
        const int b = i & 1;
        if (i >= 2) ok = ok && bar_wait(&s.l_empty[b], (uint32_t)(((i >> 1) - 1) & 1), a.spin);
        if (!ok) break;
        int n, h;
        tile_row(i, n, h);
        float* dst = lbuf + b * lrows * kPix;
        const float* src = a.lam + (size_t)n * plane;
        bar_expect(&s.l_full[b], (uint32_t)(a.fh * kPix * 4));
        for (int ta = 0; ta < a.fh; ++ta)
          bulk_g2s(dst + ta * kPix, src + (size_t)((h + ta - ch) & (kPix - 1)) * kPix, kPix * 4, &s.l_full[b]);
        issued = i + 1;
      }
      for (int i = max(issued - 2, 0); i < issued; ++i) bar_wait(&s.l_full[i & 1], (uint32_t)((i >> 1) & 1), kDefaultSpin);
    }
    __syncwarp();
  } else if (warp < 4) {
    // epilogue: thread p = TMEM lane p = pixel p
    const int p = threadIdx.x;
    const int warp_lane0 = 32 * warp;
    const uint32_t lane_off = (uint32_t)warp_lane0 << 16;
    const float beta = a.beta, rho = a.rho;
    for (int i = 0; i < ntiles; ++i) {
      int n, h;
      tile_row(i, n, h);
      if (ok) ok = bar_wait(&s.acc_full[i & 1], (uint32_t)((i >> 1) & 1), a.spin);
      ok = __all_sync(0xFFFFFFFFu, ok);   // tcgen05.ld below is warp-collective: one decision per warp
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t acc = tmem + (uint32_t)((i & 1) * 128) + lane_off;
      const size_t base = ((size_t)n * a.K * kPix + h) * kPix + p;
      for (int g = 0; g < NG; ++g) {
        const int q = i * NG + g, st = RingDt::stage(q);
        if (ok) ok = bar_wait(&s.v_full[st], (uint32_t)(RingDt::phase(q) & 1), a.spin);
        ok = __all_sync(0xFFFFFFFFu, ok);
        float w[16] = {};
        if (ok) tmem_ld16(acc + (uint32_t)(g * 16), w);   // after a timeout: no TMEM read, results void
        const float* vs = vring + (size_t)st * kCh * kPix + p;
        float old[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) old[e] = vs[e * kPix];
        warp_arrive(&s.v_empty[st]);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int k = g * kCh + e;
          if (k < a.K) {
            const float nv = w[e] - (clampb(old[e], beta) - old[e]);
            a.v[base + (size_t)k * plane] = nv;
            if (LAST && a.z) a.z[base + (size_t)k * plane] = rho * (clampb(nv, beta) - nv);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      warp_arrive(&s.acc_empty[i & 1]);
    }
  }
  kernel_end(a, s, ok);
}

// ---- D: r = sum_k d_k * u_k ------------------------------------------------------------------------
// The CTA owns the output rows [o0, o1) of the N x 128 rows, split into one segment [h0, h1) per
// image it meets. A segment's input rows run from h0 - (fh - 1 - ch) to h1 - 1 + ch (unwrapped,
// taken mod 128), each a tile whose Yr is scattered to the output rows h + ta - ch. Output row o
// receives its fh contributions from consecutive input rows (tap row ta = fh - 1 first, ta = 0 last);
// the thread of column p keeps the partial sums of the fh rows in flight in a ring (slot o mod fh, a
// column of its own), stores the first contribution, adds the others in that order, and writes the
// row of r when its last contribution is in: every r value is formed by one thread in a fixed order.
struct ConvTile {
  int n, hu, h0, h1;
};
__device__ __forceinline__ ConvTile conv_tile(int i, int o0, int o1, int fh) {
  int n = o0 / kPix;
  while (true) {
    const int h0 = max(o0 - n * kPix, 0), h1 = min(o1 - n * kPix, kPix);
    const int cnt = h1 - h0 + fh - 1;
    if (i < cnt) return ConvTile{n, h0 - (fh - 1 - (fh - 1) / 2) + i, h0, h1};
    i -= cnt;
    ++n;
  }
}
__device__ __forceinline__ int conv_tiles(int o0, int o1, int fh) {
  if (o1 <= o0) return 0;
  const int nseg = (o1 - 1) / kPix - o0 / kPix + 1;
  return (o1 - o0) + nseg * (fh - 1);
}

// shared memory: filter operand bc | A stages [2][hi | lo] | state ring | epilogue exchange
// [2][128][17] (alternating, one barrier per chunk) | output ring [fh][128] | tap table
template <int FH, int FW>
__global__ void __launch_bounds__(kThreads, 1) k_sp_conv(SpArgs a, const __grid_constant__ CUtensorMap vmap) {
  using CT = Taps<FH, FW>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ Sync s;
  const int warp = threadIdx.x >> 5;
  const int nch = (a.Kp + kAK - 1) / kAK, ntc = a.Tp / kCh;
  const size_t bbytes = (size_t)2 * a.Kp * a.Tp * 4;
  uint8_t* sb = smem;
  float* vring = reinterpret_cast<float*>(sb + bbytes);
  float* ys = vring + RingD::STAGES * kAK * kPix;
  float* oring = ys + 2 * kPix * kYsPitch;
  int* tap_i = reinterpret_cast<int*>(oring + a.fh * kPix);
  const int ch = (a.fh - 1) / 2, cw = (a.fw - 1) / 2;
  // tap t of the scatter: source row shift cw - tb (low byte, signed), last tap of its filter row
  // (bit 8), filter row ta (bits 16..); the padding taps t >= T carry zero products and no flag
  for (int t = threadIdx.x; t < a.Tp; t += kThreads) {
    const int ta = t / a.fw, tb = t - ta * a.fw;
    tap_i[t] = t < a.T ? (((cw - tb) & 0xFF) | ((tb == a.fw - 1) ? 0x100 : 0) | (ta << 16)) : 0;
  }
  kernel_begin(a, sb, bbytes, s, kProd / 64);
  const uint32_t tmem = s.tmem;
  const int NH = a.N * kPix;
  const int o0 = (int)((long long)blockIdx.x * NH / gridDim.x);
  const int o1 = (int)((long long)(blockIdx.x + 1) * NH / gridDim.x);
  const int ntiles = conv_tiles(o0, o1, a.fh);
  const size_t plane = (size_t)kPix * kPix;
  bool ok = true;

  if (warp >= 4 && warp < kWarpV) {
    // producers: group g builds the chunks of A stage g (every other chunk); thread p of a group
    // stages u_k(h, p) of the chunk's 16 filters as row p
    const int pp = threadIdx.x - 128, p = pp & (kPix - 1), grp = pp >> 7;
    const float beta = a.beta;
    for (int i = 0; i < ntiles; ++i) {
      for (int c = 0; c < nch; ++c) {
        const int q = i * nch + c, st = q % kAStages, vst = RingD::stage(q);
        if (st != grp) continue;   // with two A stages, also the state ring of this group
        if (ok) ok = bar_wait(&s.v_full[vst], (uint32_t)(RingD::phase(q) & 1), a.spin);
        if (q >= kAStages && ok) ok = bar_wait(&s.a_empty[st], (uint32_t)(((q / kAStages) - 1) & 1), a.spin);
        const float* vs = vring + (size_t)vst * kAK * kPix + p;
        float x[kAK];
#pragma unroll
        for (int e = 0; e < kAK; ++e) x[e] = vs[e * kPix];
        warp_arrive(&s.v_empty[vst]);
        const uint32_t ta = stage_begin<kAK>(tmem, st);
#pragma unroll
        for (int e0 = 0; e0 < kAK; e0 += 16) {
          uint32_t hv[16], lv[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int k = c * kAK + e0 + e;
            const float u = k < a.K ? 2.f * clampb(x[e0 + e], beta) - x[e0 + e] : 0.f;
            const float h = tf32_hi(u);
            hv[e] = __float_as_uint(h);
            lv[e] = __float_as_uint(u - h);
          }
          stage_put<kAK>(ta, e0, hv, lv);
        }
        stage_end();
        warp_arrive(&s.a_full[st]);
      }
    }
  } else if (warp == kWarpMma) {
    if ((threadIdx.x & 31) == 0)
      mma_loop<kAK>(a, s, ok, tmem, saddr(sb), (uint32_t)(a.Tp * 64), a.Kp, idesc_tf32(a.Tp), ntiles, nch);
    __syncwarp();
  } else if (warp == kWarpV) {
    if ((threadIdx.x & 31) == 0) {
      auto tile_row = [&](int i, int& n, int& h) {
        const ConvTile tl = conv_tile(i, o0, o1, a.fh);
        n = tl.n;
        h = tl.hu & (kPix - 1);
      };
      load_states<RingD, kAK>(a, s, &vmap, vring, ntiles * nch, nch, tile_row, ok);
    }
    __syncwarp();
  } else if (warp < 4) {
    // epilogue: thread p reads TMEM lane p (input pixel p), then acts for output column p
    const int p = threadIdx.x;
    const int fh = FH > 0 ? FH : a.fh;
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    int gc = 0;   // chunks exchanged so far: the exchange buffer alternates with it
    for (int i = 0; i < ntiles; ++i) {
      const ConvTile tl = conv_tile(i, o0, o1, a.fh);
      if (ok) ok = bar_wait(&s.acc_full[i & 1], (uint32_t)((i >> 1) & 1), a.spin);
      ok = __all_sync(0xFFFFFFFFu, ok);
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t acc = tmem + (uint32_t)((i & 1) * 128) + lane_off;
      float* rn = a.r + (size_t)tl.n * plane + p;
      // ring slot of output row hu - ch (tap row 0); tap row ta uses the next slots, circularly
      const int s0 = (((tl.hu - ch) % fh) + fh) % fh;
      float cur = 0.f;
      // the taps of chunk tc: scatter source shift, whether the tap closes its filter row, the row
      auto chunk = [&](int tc, auto src, auto closes, auto row) {
        float y[16] = {};
        if (ok) tmem_ld16(acc + (uint32_t)(tc * 16), y);
        // a buffer is rewritten two chunks later, after every thread has passed the barrier of the
        // chunk between, i.e. finished its reads of it
        float* yb = ys + (gc & 1) * kPix * kYsPitch;
        ++gc;
#pragma unroll
        for (int e = 0; e < 16; ++e) yb[p * kYsPitch + e] = y[e];
        named_sync(2, 128);
        float yv[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) yv[e] = yb[((p + src(tc * kCh + e)) & (kPix - 1)) * kYsPitch + e];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int t = tc * kCh + e;
          cur += yv[e];
          if (closes(t)) {
            // taps (ta, 0 .. fw-1) of this input row are in: output row hu + ta - ch
            const int ta = row(t);
            const int sl = s0 + ta < fh ? s0 + ta : s0 + ta - fh;
            float* slot = oring + sl * kPix + p;
            const float val = (ta == fh - 1) ? cur : *slot + cur;
            *slot = val;
            const int ho = tl.hu + ta - ch;
            if (ta == 0 && ho >= tl.h0 && ho < tl.h1) rn[(size_t)ho * kPix] = val;   // row complete
            cur = 0.f;
          }
        }
      };
      if constexpr (FW > 0) {
#pragma unroll
        for (int tc = 0; tc < CT::NCH; ++tc)
          chunk(tc, [](int t) { return CT::src(t); }, [](int t) { return CT::closes(t); }, [](int t) { return CT::ta(t); });
      } else {
        for (int tc = 0; tc < ntc; ++tc)
          chunk(tc, [&](int t) { return (int)(signed char)(tap_i[t] & 0xFF); }, [&](int t) { return (tap_i[t] & 0x100) != 0; },
                [&](int t) { return tap_i[t] >> 16; });
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      warp_arrive(&s.acc_empty[i & 1]);
    }
  }
  kernel_end(a, s, ok);
}

// ---- lambda = F^-1( P F(r - x / rho) ): one CTA per image, the 2-D real FFTs in shared memory ------
template <int NT>
__global__ void __launch_bounds__(NT) k_sp_lambda(const float* __restrict__ r, const float* __restrict__ x,
                                                  const float* __restrict__ pdiag, const float2* __restrict__ tw_g,
                                                  float irho, float* __restrict__ lam, int* err) {
  using G = GeoCT<128, 128>;
  extern __shared__ float2 sm[];
  const G g;
  float2* buf = sm;
  const Twiddles tw = stage_twiddles<G, NT>(g, buf + G::H * G::P, tw_g);
  float* bf = reinterpret_cast<float*>(buf);
  const size_t off = (size_t)blockIdx.x * G::D;
  for (int q = threadIdx.x; q < G::D; q += NT) {
    const int h = q >> 7, w = q & 127;
    bf[2 * G::P * h + w] = r[off + q] - x[off + q] * irho;
  }
  __syncthreads();
  rfft2<G, NT>(g, buf, tw);
  // P / D: the inverse below is unnormalised
  for (int o = threadIdx.x; o < G::Omega; o += NT) {
    const int h = o / G::Wc, c = o - h * G::Wc;
    const float s = pdiag[o];
    float2 b = buf[h * G::P + c];
    buf[h * G::P + c] = make_float2(b.x * s, b.y * s);
  }
  __syncthreads();
  irfft2<G, NT>(g, buf, tw);
  __syncthreads();
  bool bad = false;
  for (int q = threadIdx.x; q < G::D; q += NT) {
    const int h = q >> 7, w = q & 127;
    const float v = bf[2 * G::P * h + w];
    lam[off + q] = v;
    bad |= !isfinite(v);
  }
  if (bad) atomicExch(err, (int)CSC_ERR_NONFINITE);
}

}  // namespace sp

// ---- host side ---------------------------------------------------------------------------------------
static int round16(int v) { return (v + 15) / 16 * 16; }

bool spatial_applies(const Ctx& c, std::string* why) {
  auto no = [&](const char* m) {
    if (why) *why = m;
    return false;
  };
  if (c.video || c.uneven || c.sym) return no("direct spatial coding is for uniform 2-D batches");
  if (c.J != 1) return no("direct spatial coding needs J = 1");
  if (c.g.H != 128 || c.g.W != 128) return no("direct spatial coding needs 128 x 128 images");
  if (c.K > 128) return no("direct spatial coding needs K <= 128");
  if (c.fh * c.fw > 128 || c.fh > 15) return no("direct spatial coding needs fh * fw <= 128 and fh <= 15");
  if (c.p.precision != CSC_FP32 && c.p.precision != CSC_MIXED_TF32)
    return no("direct spatial coding runs in CSC_FP32 (3xTF32) or CSC_MIXED_TF32");
  return true;
}

size_t spatial_operand_bytes(const Ctx& c) { return (size_t)2 * round16(c.K) * round16(c.fh * c.fw) * 4; }

static size_t corr_smem(const Ctx& c) {
  return spatial_operand_bytes(c) + sp::kVStages * sp::kVStage +
         (size_t)2 * (c.fh + 1) * sp::kPix * 4 + (size_t)2 * ((round16(c.fh * c.fw) + sp::kAKDt - 1) / sp::kAKDt * sp::kAKDt) * 4;
}
static size_t conv_smem(const Ctx& c) {
  return spatial_operand_bytes(c) + sp::RingD::STAGES * sp::kVStageD +
         (size_t)2 * sp::kPix * sp::kYsPitch * 4 + (size_t)c.fh * sp::kPix * 4 + (size_t)round16(c.fh * c.fw) * 4;
}
static constexpr int kLamThreads = 512;
static size_t lambda_smem() { return ((size_t)128 * odd_pitch(65) + 64 + 128 + 65) * sizeof(float2); }

static sp::SpArgs sp_args(const Ctx& c, const uint8_t* bop, float* v, float* z) {
  sp::SpArgs a{};
  a.N = c.N; a.K = c.K; a.T = c.fh * c.fw; a.fh = c.fh; a.fw = c.fw;
  a.Kp = round16(c.K); a.Tp = round16(a.T);
  a.passes = (c.p.precision == CSC_MIXED_TF32) ? 1 : 3;
  a.beta = (float)c.p.beta; a.rho = (float)c.p.rho;
  a.bop = bop; a.v = v; a.z = z; a.lam = c.sp_lam; a.r = c.sp_r;
  a.err = c.cerr;   // read at the end of csc_code like the sweeps' flag
  a.spin = c.wait_limit > 0 ? c.wait_limit : sp::kDefaultSpin;
  return a;
}

cudaError_t launch_spatial_operands(const Ctx& c, const float* d) {
  const int Kp = round16(c.K), Tp = round16(c.fh * c.fw);
  const int n = Kp * Tp;
  sp::k_sp_operands<<<(n + 255) / 256, 256, 0, c.stream>>>(d, c.K, c.fh * c.fw, Kp, Tp, c.sp_bt, c.sp_bc);
  return cudaGetLastError();
}

static int sp_grid(const Ctx& c) { return std::min(c.nsm, c.N * sp::kPix); }

// the tensor map of the state v as [N K][128][128] float32 with boxes of `maps` maps x 1 row x 128
// pixels (the loader's stage); the encoder comes from the driver through the runtime
static cudaError_t state_map(const Ctx& c, const float* v, int maps, CUtensorMap* m) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[3] = {(cuuint64_t)sp::kPix, (cuuint64_t)sp::kPix, (cuuint64_t)c.N * c.K};
  const cuuint64_t strides[2] = {(cuuint64_t)sp::kPix * 4, (cuuint64_t)sp::kPix * sp::kPix * 4};
  const cuuint32_t box[3] = {(cuuint32_t)sp::kPix, 1u, (cuuint32_t)maps};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(v), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_spatial_conv(const Ctx& c, const float* v) {
  const sp::SpArgs a = sp_args(c, c.sp_bc, const_cast<float*>(v), nullptr);
  CUtensorMap vmap;
  cudaError_t e = state_map(c, v, sp::kAK, &vmap);
  if (e != cudaSuccess) return e;
  // at least 116 KB, so that one CTA holds an SM and its 512 TMEM columns
  const int smem = (int)std::max<size_t>(conv_smem(c), 116 * 1024);
  // 11 x 11 (the benchmark's support) with compile-time taps; every other support reads tap tables
  auto kern = (c.fh == 11 && c.fw == 11) ? sp::k_sp_conv<11, 11> : sp::k_sp_conv<0, 0>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<sp_grid(c), sp::kThreads, smem, c.stream>>>(a, vmap);
  return cudaGetLastError();
}

cudaError_t launch_spatial_lambda(const Ctx& c, const float* x) {
  auto kern = sp::k_sp_lambda<kLamThreads>;
  const int smem = (int)lambda_smem();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<c.N, kLamThreads, smem, c.stream>>>(c.sp_r, x, c.pdiag, c.tw, (float)(1.0 / c.p.rho), c.sp_lam, c.cerr);
  return cudaGetLastError();
}

cudaError_t launch_spatial_corr(const Ctx& c, float* v, float* z, bool last) {
  const sp::SpArgs a = sp_args(c, c.sp_bt, v, z);
  CUtensorMap vmap;
  cudaError_t e = state_map(c, v, sp::kCh, &vmap);
  if (e != cudaSuccess) return e;
  const int smem = (int)std::max<size_t>(corr_smem(c), 116 * 1024);
  const bool t11 = (c.fh == 11 && c.fw == 11);
  auto kern = last ? (t11 ? sp::k_sp_corr<true, 11, 11> : sp::k_sp_corr<true, 0, 0>)
                   : (t11 ? sp::k_sp_corr<false, 11, 11> : sp::k_sp_corr<false, 0, 0>);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<sp_grid(c), sp::kThreads, smem, c.stream>>>(a, vmap);
  return cudaGetLastError();
}

}  // namespace csc
