// Grid-wide exchanges of the persistent CG launches (the 2-D learning's k_learn_cg and the video
// learning's k_vl_cg): one cooperative launch, no grid barrier primitive. Every value that crosses
// CTAs is stored as a 64-bit word (float bits | epoch << 32) with relaxed GPU-scope stores, so a
// reader polls exactly the words it needs until they carry the current epoch; partial sums go to
// per-CTA slot words that alternate between two banks by epoch parity and are summed in CTA order
// (every CTA forms the same totals). Every wait is bounded (a context's wait limit, else kSpinLimit
// SM clocks) and sets the context's error word on running out.
#pragma once
#include "csc_internal.cuh"

namespace csc {

// default bound of every spin-wait of the CG launches (~1 s of SM clocks); a context can lower it
// (csc_set_wait_limit) so that a test can make a wait run out
constexpr long long kSpinLimit = 2000000000LL;

constexpr int kSlotWords = 4 * kMaxJ;   // words of one CTA's slot in one exchange

// Sums vals[0..N) over the block in float32 (the device's float64 rate is a few operations per
// clock per SM, so per-thread float64 work is kept out of the CG loop); the totals are valid in
// thread 0 only. scratch: [NT/32][kSlotWords] floats, free on entry.
template <int NT, int N>
__device__ __forceinline__ void block_reduce_to0(float (&vals)[N], float* scratch) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float v = vals[i];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) scratch[(threadIdx.x >> 5) * kSlotWords + i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float v = (threadIdx.x < NT / 32) ? scratch[threadIdx.x * kSlotWords + i] : 0.f;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      vals[i] = v;
    }
  }
}

// vals[idx] += v for a run-time idx with every slot kept in registers
template <int N>
__device__ __forceinline__ void add_at(float (&vals)[N], int idx, float v) {
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i == idx) vals[i] += v;
}

// 64-bit words exchanged between CTAs: relaxed, GPU scope (single-copy atomic; no fences implied)
__device__ __forceinline__ void st_volatile_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long tag(float v, unsigned ep) {
  return ((unsigned long long)ep << 32) | __float_as_uint(v);
}

// thread 0: make the CTA's earlier global writes visible, then publish vals[0..N) with epoch ep.
// The caller has synchronised the block since those writes. N == 0: one word without a sum.
template <int N>
__device__ __forceinline__ void publish(unsigned long long* slots, int G, const float* vals, unsigned ep,
                                        bool fence = false) {
  if (threadIdx.x != 0) return;
  if (fence) asm volatile("fence.acq_rel.gpu;" ::: "memory");   // release: plain stores before the words
  unsigned long long* s = slots + ((size_t)(ep & 1) * G + blockIdx.x) * kSlotWords;
#pragma unroll
  for (int i = 0; i < (N > 0 ? N : 1); ++i)
    st_volatile_u64(s + i, ((unsigned long long)ep << 32) | __float_as_uint(N > 0 ? vals[i] : 0.f));
}

// Waits until this block's words carry epoch ep, in two phases: first the exchange's slot words
// (G CTAs x nw <= US NT; thread t polls words t, t + NT, ..., values parked in vals, [G][nw] floats of
// shared memory), when slots is not null; after a block barrier the data words t + u NT < ndata (left in
// wd[u]; the value is the low half), which the publishers wrote before their slot words and so are
// almost always complete by then (any that are not are polled again). Must be called by the whole
// block. false when a CTA flagged an error or the wait ran out (flag set).
template <int NT, int U, int US = 2>
__device__ bool wait_words(const unsigned long long* slots, int G, int nw, unsigned ep, float* vals,
                           const unsigned long long* data, int ndata, unsigned long long (&wd)[U], int* err,
                           long long limit) {
  __shared__ int s_bad;
  const long long t0 = clock64();
  bool ok = true;
  if (slots) {
    if (threadIdx.x == 0) s_bad = 0;
    const unsigned long long* sb = slots + (size_t)(ep & 1) * G * kSlotWords;
    const int nsw = G * nw;
#pragma unroll
    for (int u = 0; u < US; ++u) {
      const int i = threadIdx.x + u * NT;
      if (i < nsw) {
        const unsigned long long* wp = sb + (size_t)(i / nw) * kSlotWords + i % nw;
        unsigned long long w = ld_volatile_u64(wp);
        while ((unsigned)(w >> 32) != ep) {
          if (*(volatile int*)err || clock64() - t0 > limit) { ok = false; break; }
          w = ld_volatile_u64(wp);
        }
        vals[i] = __uint_as_float((unsigned)w);
      }
    }
    if (!ok) s_bad = 1;
    __syncthreads();
    if (s_bad) {
      if (!*(volatile int*)err) atomicExch(err, (int)CSC_ERR_TIMEOUT);
      return false;
    }
  }
  unsigned pend = 0;
#pragma unroll
  for (int u = 0; u < U; ++u)
    if ((int)threadIdx.x + u * NT < ndata) pend |= 1u << u;
  while (pend) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (pend & (1u << u)) wd[u] = ld_volatile_u64(data + threadIdx.x + u * NT);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if ((pend & (1u << u)) && (unsigned)(wd[u] >> 32) == ep) pend &= ~(1u << u);
    if (!pend) break;
    if (*(volatile int*)err) return false;
    if (clock64() - t0 > limit) {
      atomicExch(err, (int)CSC_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ float word_value(unsigned long long w) { return __uint_as_float((unsigned)w); }

// totals[i] = sum over CTAs of vals[b * nw + i], i < n, in a fixed order (one warp per value, float32).
// Call after a barrier that follows wait_words; ends with a barrier. then() runs on thread 0 once the
// totals are known: the scalars of the iteration are formed there and broadcast through shared memory.
// All of it stays in float32: the device's float64 rate is a few operations per clock per SM, and
// float64 on the path of every exchange cost microseconds.
template <int NT, class F>
__device__ __forceinline__ void sum_slots(const float* vals, int G, int nw, int n, float* totals, F then) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < n; i += NT / 32) {
    float v = 0.f;
    for (int b = lane; b < G; b += 32) v += vals[b * nw + i];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) totals[i] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) then();
  __syncthreads();
}

}  // namespace csc
