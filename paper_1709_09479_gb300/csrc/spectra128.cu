// Forward 2-D spectra of real 128 x 128 maps with the per-thread passes of f128_common.cuh (the
// code spectra of a learning call, Sec. 3.2: z_hat_nk = F z_nk).
#include <cuda_runtime.h>

#include <algorithm>

#include "csc_internal.cuh"
#include "f128_common.cuh"

namespace csc {
namespace f128 {

// Forward spectra of real 128 x 128 maps (the codes of a learning call): per map the forward column
// and row passes and the real split of the coding sweep, each thread's 16 (+2) bins put back into
// the shared-memory map in the half-spectrum order (kh * 65 + kw), and the map copied out with
// 16-byte coalesced stores: out[m][Omega].
__global__ void __launch_bounds__(NT, 1) k_spectra_f128(const float* __restrict__ in, long long nmaps,
                                                        float2* __restrict__ out, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  float2* buf = sm;                  // [128][P]; P = 65, so the half spectrum is buf[0 .. OM)
  float2* twt = buf + H * P;         // twiddle tables (kTwEntries)
  const int t = threadIdx.x;
  const Tw T = build_tw<NT>(twt, tw + W / 2);
  const Roles R = roles_of(t);
  const int wc = R.wc, g = R.g;
  const long long m0 = (long long)blockIdx.x * nmaps / gridDim.x;
  const long long m1 = (long long)(blockIdx.x + 1) * nmaps / gridDim.x;
  for (long long m = m0; m < m1; ++m) {
    if (threadIdx.x < 4 && m + 1 < m1) prefetch_l2_f128(in + (m + 1) * D + threadIdx.x * (D / 4), (unsigned)D);
    float2 zc[16];   // rows h = g + 8 j of column wc
    const float* src = in + m * D;
#pragma unroll
    for (int j = 0; j < 16; ++j) zc[j] = __ldcs(reinterpret_cast<const float2*>(src + (g + 8 * j) * W + 2 * wc));
    __syncthreads();   // the twiddle tables are built; the previous map's copy-out precedes these writes
    fwd_cols1(buf, T, R, zc);
    __syncthreads();
    fwd_cols2(buf, R);
    __syncthreads();
    fwd_rows1(buf, T, R);
    __syncthreads();
    float2 y[18];
    fwd_rows2_split(buf, T, R, [&](int s, float2 x) { y[s] = x; });
    __syncthreads();   // every thread's row reads precede the spectrum writes
#pragma unroll
    for (int s = 0; s < 18; ++s)
      if (s < 16 || R.nyq) buf[canonical_of(slot_pos(s, t))] = y[s];
    __syncthreads();
    const float4* b4 = reinterpret_cast<const float4*>(buf);
    float4* o4 = reinterpret_cast<float4*>(out + m * OM);
    for (int i = t; i < OM / 2; i += NT) __stcs(o4 + i, b4[i]);
  }
}

}  // namespace f128

cudaError_t launch_spectra_f128(const Ctx& c, const float* in, long long nmaps, float2* out) {
  if (nmaps <= 0) return cudaSuccess;
  const size_t smem = ((size_t)f128::H * f128::P + f128::kTwEntries) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(f128::k_spectra_f128, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<long long>(nmaps, (long long)c.nsm);
  f128::k_spectra_f128<<<grid, f128::NT, smem, c.stream>>>(in, nmaps, out, c.tw);
  return cudaGetLastError();
}

}  // namespace csc
