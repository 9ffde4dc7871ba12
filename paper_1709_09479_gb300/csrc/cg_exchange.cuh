// Helpers of the grid-wide exchanges of the persistent CG launches (the 2-D learning's k_learn_cg and
// the video learning's k_vl_cg): one cooperative launch, no grid barrier primitive; each exchange is a
// counter of arrivals that every CTA increments with release semantics after its plain stores, and
// that the readers poll with acquire loads, bounded by a context's wait limit (else kSpinLimit SM
// clocks). Partial sums go to per-CTA slots and are summed in a fixed order, so every CTA forms the
// same totals.
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

// totals[i] = sum over CTAs of vals[b * nw + i], i < n, in a fixed order (one warp per value, float32).
// Call after a barrier that follows the loads of vals; ends with a barrier. then() runs on thread 0 once the
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
