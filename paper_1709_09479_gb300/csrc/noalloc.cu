// csc_code_noalloc: the coding call of csc_code without a context and without any device
// allocation. Some callers cannot allocate device memory at the point where they want to code
// images: code inside a framework whose caching allocator owns every byte of the device pool (a
// cudaMalloc there fails or fragments the pool), plugins and extension points that are handed only a
// stream and device pointers and have no right to allocate, and latency-bound paths where the
// implicit synchronisation of cudaMalloc/cudaFree is not acceptable. For them the workspace (filter
// and image spectra, the per-frequency system, the partial sums of the ADMM sweeps, the twiddle
// table) lives in one file-scope __device__ array of fixed size, reserved when the library is loaded
// and held by every GPU that loads it until the process exits.
//
// Set-up: the array's name is only a host-side stand-in in host code, so its device address is
// looked up with cudaGetSymbolAddress once per device (with that device current) on the first
// call made on it, cached, and passed to the kernels. The twiddle table is written by a kernel, so
// a call copies nothing from host memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "csc_internal.cuh"

using namespace csc;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;   // 64 MiB per device
constexpr int kNoAllocMaxDevices = 64;
constexpr int kNoAllocMaxTwiddles = 8192;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

csc_status noalloc_fail(csc_status s, const char* msg) {
  set_global_error(msg);
  return s;
}

// device address of the scratch array on `device` (current), looked up once per device
csc_status scratch_on(int device, unsigned char** out) {
  if (device < 0 || device >= kNoAllocMaxDevices)
    return noalloc_fail(CSC_ERR_UNSUPPORTED, "csc_code_noalloc: device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return noalloc_fail(CSC_ERR_CUDA, "csc_code_noalloc: cudaGetSymbolAddress of the scratch array failed");
    }
    g_noalloc_addr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[device]);
  return CSC_OK;
}

bool device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// tw[t] = exp(-2 pi i t / n) for the three sections of the table: n = W/2 (t < W/2), n = H
// (t < H) and n = W (t <= W/2), computed in float64 and rounded once
__global__ void k_noalloc_twiddles(float2* tw, int Wh, int H, int W) {
  const int n_all = Wh + H + Wh + 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_all; i += gridDim.x * blockDim.x) {
    int t = i, n = Wh;
    if (i >= Wh + H) { t = i - Wh - H; n = W; }
    else if (i >= Wh) { t = i - Wh; n = H; }
    double s, c;
    sincospi(2.0 * (double)t / (double)n, &s, &c);
    tw[i] = make_float2((float)c, (float)-s);
  }
}

cudaError_t launch_noalloc_twiddles(float2* tw, int Wh, int H, int W, cudaStream_t stream) {
  const int n_all = Wh + H + Wh + 1;
  k_noalloc_twiddles<<<(n_all + 255) / 256, 256, 0, stream>>>(tw, Wh, H, W);
  return cudaGetLastError();
}

}  // namespace

extern "C" csc_status csc_code_noalloc(const csc_params* params, int n_images, const int* dims, void* stream,
                                       const float* x, const float* d, float* v, float* z, int iters) {
  if (!params || !dims || !x || !d || !v) return noalloc_fail(CSC_ERR_ARG, "csc_code_noalloc: null argument");
  const csc_params& p = *params;
  if (n_images < 1 || iters < 0) return noalloc_fail(CSC_ERR_ARG, "csc_code_noalloc: n_images >= 1, iters >= 0");
  if (p.J < 1 || p.J > kMaxJ) return noalloc_fail(CSC_ERR_SHAPE, "csc_code_noalloc: J must be 1..3");
  if (p.K < 1) return noalloc_fail(CSC_ERR_ARG, "csc_code_noalloc: K must be >= 1");
  if (!(p.beta > 0) || !(p.rho > 0) || !std::isfinite(p.beta) || !std::isfinite(p.rho))
    return noalloc_fail(CSC_ERR_ARG, "csc_code_noalloc: beta and rho must be finite and > 0");
  if (p.precision != CSC_FP32) return noalloc_fail(CSC_ERR_UNSUPPORTED, "csc_code_noalloc: CSC_FP32 only");
  const int fh = p.fs[0], fw = p.fs[1];
  if (fh < 1 || fw < 1 || !(fh & 1) || !(fw & 1))
    return noalloc_fail(CSC_ERR_SHAPE, "csc_code_noalloc: filter support must be odd and >= 1");
  const int H = dims[0], W = dims[1];
  if (H < 8 || W < 8 || (W & 1)) return noalloc_fail(CSC_ERR_SHAPE, "csc_code_noalloc: need H, W >= 8 and W even");
  if (fh > H || fw > W) return noalloc_fail(CSC_ERR_SHAPE, "csc_code_noalloc: filter larger than the image");

  Ctx c;
  c.p = p;
  c.N = n_images; c.J = p.J; c.K = p.K; c.fh = fh; c.fw = fw; c.S2 = fh * fw;
  Geometry& g = c.g;
  g.H = H; g.W = W; g.Wh = W / 2; g.Wc = W / 2 + 1; g.P = odd_pitch(g.Wc);
  g.Omega = H * g.Wc; g.D = H * W;
  g.ct_id = (H == 128 && W == 128) ? 1 : (H == 100 && W == 100) ? 2 : (H == 64 && W == 64) ? 3 : 0;
  g.rt.H = H; g.rt.W = W; g.rt.Wh = g.Wh; g.rt.Wc = g.Wc; g.rt.P = g.P; g.rt.Omega = g.Omega; g.rt.D = g.D;
  g.rt.rrow = factorize(g.Wh);
  g.rt.rcol = factorize(H);
  for (int i = 0; i < g.rt.rrow.n_st; ++i)
    if (!radix_supported_rt(g.rt.rrow.r[i])) return noalloc_fail(CSC_ERR_SHAPE, "csc_code_noalloc: W/2 must factor into 2, 3, 5 and 7");
  for (int i = 0; i < g.rt.rcol.n_st; ++i)
    if (!radix_supported_rt(g.rt.rcol.r[i])) return noalloc_fail(CSC_ERR_SHAPE, "csc_code_noalloc: H must factor into 2, 3, 5 and 7");
  if (sweep_smem_bytes(g, p.J, kIter) > kSmemLimit)
    return noalloc_fail(CSC_ERR_SHAPE, "csc_code_noalloc: image too large for one map per CTA in shared memory");
  const int ntw = g.Wh + g.H + g.Wc;
  if (ntw > kNoAllocMaxTwiddles) return noalloc_fail(CSC_ERR_SHAPE, "csc_code_noalloc: image sides too long");

  c.stream = (cudaStream_t)stream;
  if (cudaGetDevice(&c.device) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(CSC_ERR_CUDA, "csc_code_noalloc: cudaGetDevice failed");
  }
  if (cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(CSC_ERR_CUDA, "csc_code_noalloc: cudaDeviceGetAttribute failed");
  }
  if (!device_pointer(x) || !device_pointer(d) || !device_pointer(v) || (z && !device_pointer(z)))
    return noalloc_fail(CSC_ERR_ARG, "csc_code_noalloc: x, d, v and z must be device pointers");
  const long long NK = (long long)c.N * c.K;
  c.G = (int)(NK < c.nsm ? NK : c.nsm);

  // carve the scratch array: twiddles, d_hat, x_hat, per-frequency system, two partial-sum buffers
  const size_t Om = g.Omega;
  const size_t b_tw = up256((size_t)ntw * sizeof(float2));
  const size_t b_dhat = up256((size_t)c.K * c.J * Om * sizeof(float2));
  const size_t b_xhat = up256((size_t)c.N * c.J * Om * sizeof(float2));
  const size_t b_pd = up256(Om * sizeof(float));
  const size_t b_pm = up256(Om * c.J * c.J * sizeof(float2));
  const size_t b_part = up256((size_t)(c.G + c.N) * c.J * Om * sizeof(float2));
  const size_t need = b_tw + b_dhat + b_xhat + b_pd + b_pm + 2 * b_part;
  if (need > kNoAllocScratchBytes) {
    char msg[200];
    std::snprintf(msg, sizeof(msg),
                  "csc_code_noalloc: problem needs %zu bytes of workspace, above the fixed 64 MiB scratch "
                  "(use csc_init/csc_code)", need);
    return noalloc_fail(CSC_ERR_SHAPE, msg);
  }
  unsigned char* base = nullptr;
  csc_status s = scratch_on(c.device, &base);
  if (s != CSC_OK) return s;
  size_t off = 0;
  auto take = [&](size_t bytes) { unsigned char* q = base + off; off += bytes; return q; };
  c.tw = reinterpret_cast<float2*>(take(b_tw));
  c.dhat = reinterpret_cast<float2*>(take(b_dhat));
  c.xhat = reinterpret_cast<float2*>(take(b_xhat));
  c.pdiag = reinterpret_cast<float*>(take(b_pd));
  c.pmat = reinterpret_cast<float2*>(take(b_pm));
  c.part[0] = reinterpret_cast<float2*>(take(b_part));
  c.part[1] = reinterpret_cast<float2*>(take(b_part));

  // twiddles (the table csc_init builds on the host), written by a kernel so that nothing is
  // copied from host memory
  cudaError_t e = launch_noalloc_twiddles(c.tw, g.Wh, g.H, g.W, c.stream);
  if (e == cudaSuccess && iters == 0) {
    if (z) e = launch_codes_from_state(c, v, z);
  } else if (e == cudaSuccess) {
    e = launch_fft_maps(c, d, c.K * c.J, 1, c.dhat);
    if (e == cudaSuccess) e = launch_solve_prep(c);
    if (e == cudaSuccess) e = launch_fft_maps(c, x, c.N * c.J, 0, c.xhat);
    if (e == cudaSuccess) e = launch_sweep(c, kPrologue, nullptr, c.part[0], v, nullptr);
    for (int t = 0; t < iters && e == cudaSuccess; ++t) {
      const int mode = (t == iters - 1) ? kLast : kIter;
      e = launch_sweep(c, mode, c.part[t & 1], c.part[(t + 1) & 1], v, z);
    }
  }
  if (e != cudaSuccess) {
    char msg[200];
    std::snprintf(msg, sizeof(msg), "csc_code_noalloc: %s", cudaGetErrorString(e));
    return noalloc_fail(CSC_ERR_CUDA, msg);
  }
  return CSC_OK;
}
