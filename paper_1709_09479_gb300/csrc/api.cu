// C ABI of libcsc.so (include/csc.h): argument checks, workspace, host/device staging, and the
// order of launches for each entry point. All compute runs in the kernels of coding.cu and
// learning.cu on the context's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <mutex>
#include <type_traits>
#include <new>
#include <string>
#include <vector>

#include "csc_internal.cuh"

using namespace csc;

struct csc_ctx {
  Ctx c;
};

namespace {

thread_local std::string g_init_error;

const char* kVersion = "csc-gb300 0.1 (sm_103a)";

csc_status fail(Ctx* c, csc_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  else g_init_error = msg;
  return s;
}

csc_status cuda_fail(Ctx* c, cudaError_t e, const char* where) {
  return fail(c, CSC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CSC_CHECK_CUDA(ctx, call, where)               \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t ensure_alloc(T** p, size_t count) {
  if (*p) return cudaSuccess;
  return cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
}

bool radices_ok(const Radices& r) {
  for (int i = 0; i < r.n_st; ++i)
    if (!radix_supported_rt(r.r[i])) return false;
  return true;
}

// Resolve an array argument to a device pointer, staging host memory into *stage.
template <class T>
csc_status stage_in(Ctx* c, const T* user, T** stage, size_t count, const T** dev, bool copy) {
  if (is_device_ptr(user)) {
    *dev = user;
    return CSC_OK;
  }
  CSC_CHECK_CUDA(c, ensure_alloc(stage, count), "staging allocation");
  if (copy)
    CSC_CHECK_CUDA(c, cudaMemcpyAsync(*stage, user, count * sizeof(T), cudaMemcpyHostToDevice, c->stream),
                   "host-to-device copy");
  *dev = *stage;
  return CSC_OK;
}

// benchmarking aid: open an event bracket (returns its index, or -1 when timing is off)
int bracket_open(Ctx* c, int kind) {
  if (!c->timing) return -1;
  if (c->events_used == c->events.size()) {
    Ctx::EventPair ep{nullptr, nullptr, kind};
    if (cudaEventCreate(&ep.a) != cudaSuccess || cudaEventCreate(&ep.b) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    c->events.push_back(ep);
  }
  const int i = (int)c->events_used++;
  c->events[i].kind = kind;
  cudaEventRecord(c->events[i].a, c->stream);
  return i;
}

void bracket_close(Ctx* c, int i) {
  if (i >= 0) cudaEventRecord(c->events[i].b, c->stream);
}

void free_all(Ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
  void* uptrs[] = {c->U.d_cls, c->U.d_img, c->U.d_mstart, c->U.d_slot, c->U.d_bcls, c->U.d_bimg, c->U.d_bcol,
                   c->U.d_brow, c->U.d_bfreq, c->U.d_btabs, c->U.d_by, c->U.d_blam, c->U.d_be, c->U.d_bl1,
                   c->U.d_bsetup, c->U.d_bprep, c->U.d_scol, c->U.d_srow, c->U.d_stile, c->U.d_sy, c->U.d_sq};
  for (void* p : uptrs)
    if (p) cudaFree(p);
  for (auto& ep : c->events) {
    cudaEventDestroy(ep.a);
    cudaEventDestroy(ep.b);
  }
  c->events.clear();
  void* ptrs[] = {c->xext, c->tw, c->dhat, c->dhatp, c->dhatp16, c->dhat16, c->L.rspec, c->L.zt, c->L.lagT, c->xhat, c->pdiag, c->pmat, c->part[0], c->part[1], c->l1, c->objimg,
                  c->err, c->L.zhat, c->L.gram, c->L.lags, c->L.chat, c->L.yw, c->L.zw, c->L.b, c->L.vec, c->L.mu, c->L.slots,
                  c->L.iters, c->st_x, c->st_d, c->st_v, c->st_z, c->st_mu, c->B.seg, c->B.vbar,
                  c->B.gspec, c->B.S, c->B.Xb, c->B.part[0], c->B.part[1], c->B.spec,
                  c->vS, c->vd2, c->vx3, c->vp3, c->vtmp, c->vobj, c->vl1,
                  c->VL.z3, c->VL.zt, c->VL.x2, c->VL.x3, c->VL.gram, c->VL.rspec, c->VL.rspecT, c->VL.U, c->VL.tab, c->VL.lags,
                  c->VL.chat, c->VL.vec, c->VL.phat, c->VL.yhat, c->VL.mu, c->VL.active, c->VL.fscal, c->VL.part, c->VL.st, c->VL.iters,
                  c->VL.words, c->sp_bt, c->sp_bc, c->sp_r, c->sp_lam};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}


// checks one image size against what the per-map kernels support; fills the geometry
csc_status check_size(const csc_params& p, int H, int W, Geometry& g, const char* who) {
  const int fh = p.fs[0], fw = p.fs[1];
  char msg[160];
  if (H < 8 || W < 8 || (W & 1)) {
    std::snprintf(msg, sizeof(msg), "%s: image %dx%d: need H, W >= 8 and W even", who, H, W);
    return fail(nullptr, CSC_ERR_SHAPE, msg);
  }
  if (fh > H || fw > W) {
    std::snprintf(msg, sizeof(msg), "%s: filter larger than the %dx%d image", who, H, W);
    return fail(nullptr, CSC_ERR_SHAPE, msg);
  }
  g.H = H; g.W = W; g.Wh = W / 2; g.Wc = W / 2 + 1; g.P = odd_pitch(g.Wc);
  g.Omega = H * g.Wc; g.D = H * W;
  g.ct_id = (H == 128 && W == 128) ? 1 : (H == 100 && W == 100) ? 2 : (H == 64 && W == 64) ? 3 : 0;
  g.rt.H = H; g.rt.W = W; g.rt.Wh = g.Wh; g.rt.Wc = g.Wc; g.rt.P = g.P; g.rt.Omega = g.Omega; g.rt.D = g.D;
  g.rt.rrow = factorize(g.Wh);
  g.rt.rcol = factorize(H);
  if (!radices_ok(g.rt.rrow) || !radices_ok(g.rt.rcol)) {
    std::snprintf(msg, sizeof(msg), "%s: image %dx%d: H and W/2 must factor into 2, 3, 5 and 7", who, H, W);
    return fail(nullptr, CSC_ERR_SHAPE, msg);
  }
  if (sweep_smem_bytes(g, p.J, kIter) > kSmemLimit) {
    std::snprintf(msg, sizeof(msg), "%s: image %dx%d too large for one map per CTA in shared memory", who, H, W);
    return fail(nullptr, CSC_ERR_SHAPE, msg);
  }
  return CSC_OK;
}

// a context view on one size class of an uneven batch, for the per-map setup launchers
void class_view(const Ctx& c, int ci, Ctx& v) {
  const UClass& uc = c.U.cls[ci];
  v.p = c.p; v.N = c.N; v.J = c.J; v.K = c.K; v.fh = c.fh; v.fw = c.fw; v.S2 = c.S2;
  v.stream = c.stream; v.device = c.device; v.nsm = c.nsm; v.G = c.G;
  Geometry g;
  check_size(c.p, c.U.cls_H[ci], c.U.cls_W[ci], g, "class");
  g.ct_id = 0;
  v.g = g;
  v.tw = c.tw + uc.tw;
  v.dhat = c.dhat + uc.dhat;
  v.pdiag = c.pdiag + uc.pd;
  v.pmat = c.pmat + uc.pm;
}

// cost-balanced CTA map ranges and partial-sum slots for G CTAs
void uneven_partition(Ctx* c, int G) {
  UnevenLayout& U = c->U;
  const int N = U.n_small, K = c->K, J = c->J;
  std::vector<double> cost(N);
  double total = 0.0;
  for (int n = 0; n < N; ++n) {
    const UClass& uc = U.cls[U.img[n].cls];
    cost[n] = (double)uc.g.D;
    total += cost[n] * K;
  }
  const long long NK = (long long)N * K;
  U.mstart.assign(G + 1, 0);
  long long m = 0;
  double acc = 0.0;
  for (int cta = 1; cta < G; ++cta) {
    const double target = total * cta / G;
    while (m < NK && acc + cost[m / K] * 0.5 < target) { acc += cost[m / K]; ++m; }
    long long lo = U.mstart[cta - 1] + 1, hi = NK - (G - cta);
    U.mstart[cta] = std::min(std::max(m, lo), hi);
    if (U.mstart[cta] != m) {   // keep acc consistent with the clamped boundary
      acc = 0.0;
      for (long long q = 0; q < U.mstart[cta]; ++q) acc += cost[q / K];
      m = U.mstart[cta];
    }
  }
  U.mstart[G] = NK;
  auto cta_of = [&](long long map) {
    int lo = 0, hi = G - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (U.mstart[mid] <= map) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  U.slot.assign(G + N, 0);
  long long off = 0;
  for (int n = 0; n < N; ++n) {
    UImage& im = U.img[n];
    im.c0 = cta_of((long long)n * K);
    im.c1 = cta_of((long long)(n + 1) * K - 1);
    const long long om = U.cls[im.cls].g.Omega;
    for (int cc = im.c0; cc <= im.c1; ++cc) {
      U.slot[cc + n] = off;
      off += (long long)J * om;
    }
  }
  U.n_slot = off;
  c->G = G;
}

csc_status upload_uneven(Ctx* c) {
  UnevenLayout& U = c->U;
  auto put = [&](auto** dptr, const auto& vec) {
    using T = typename std::remove_reference<decltype(vec)>::type::value_type;
    if (*dptr) cudaFree(*dptr);
    *dptr = nullptr;
    if (cudaMalloc((void**)dptr, std::max<size_t>(vec.size(), 1) * sizeof(T)) != cudaSuccess) return false;
    return cudaMemcpy(*dptr, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
  };
  if (!put(&U.d_cls, U.cls) || !put(&U.d_img, U.img) || !put(&U.d_mstart, U.mstart) || !put(&U.d_slot, U.slot)) {
    cudaGetLastError();
    return fail(c, CSC_ERR_WORKSPACE, "uneven batch: descriptor upload failed");
  }
  for (int i = 0; i < 2; ++i) {
    if (c->part[i]) cudaFree(c->part[i]);
    c->part[i] = nullptr;
    if (cudaMalloc((void**)&c->part[i], std::max<long long>(U.n_slot, 1) * sizeof(float2)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, CSC_ERR_WORKSPACE, "uneven batch: partial-sum allocation failed");
    }
  }
  if (c->l1) cudaFree(c->l1);
  c->l1 = nullptr;
  if (cudaMalloc((void**)&c->l1, c->G * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CSC_ERR_WORKSPACE, "uneven batch: allocation failed");
  }
  return CSC_OK;
}

UnevenArgs uneven_args(const Ctx& c, const float2* part_in, float2* part_out, float* v, float* z) {
  UnevenArgs a;
  a.N = c.U.n_small; a.K = c.K; a.J = c.J; a.G = c.G;
  a.beta = (float)c.p.beta; a.rho = (float)c.p.rho;
  a.buf_elems = c.U.buf_elems; a.max_omega = c.U.max_omega;
  a.cls = c.U.d_cls; a.img = c.U.d_img; a.mstart = c.U.d_mstart; a.slot = c.U.d_slot;
  a.tw = c.tw; a.dhat = c.dhat; a.pdiag = c.pdiag; a.pmat = c.pmat; a.xhat = c.xhat;
  a.dhat16 = c.p.precision == CSC_MIXED_BF16 ? c.dhat16 : nullptr;
  a.part_in = part_in; a.part_out = part_out; a.v = v; a.z = z; a.l1 = c.l1;
  return a;
}

BigArgs big_args(const Ctx& c, float* v, float* z) {
  const UnevenLayout& U = c.U;
  BigArgs a{};
  a.K = c.K; a.J = c.J;
  a.beta = (float)c.p.beta; a.rho = (float)c.p.rho;
  a.cls = U.d_bcls; a.img = U.d_bimg;
  a.col_items = U.d_bcol; a.row_items = U.d_brow; a.freq_items = U.d_bfreq;
  a.n_col_items = (int)U.bcol.size(); a.n_row_items = (int)U.brow.size(); a.n_freq_items = (int)U.bfreq.size();
  a.col_smem = U.bcol_smem; a.row_smem = U.brow_smem; a.tw_max = U.btw_max;
  a.tabs = U.d_btabs; a.dhat = c.dhat; a.pdiag = c.pdiag; a.pmat = c.pmat; a.xhat = c.xhat;
  a.dhat16 = c.p.precision == CSC_MIXED_BF16 ? c.dhat16 : nullptr;
  a.Y = U.d_by; a.lam = U.d_blam; a.v = v; a.z = z; a.e_items = U.d_be; a.l1_items = U.d_bl1;
  return a;
}

// kernel launches of one launch_big_sweep call
int big_launches(int mode) { return mode == kPrologue ? 3 : mode == kLast ? 2 : mode == kIter ? 4 : 3; }

csc_status upload_big(Ctx* c, const std::vector<BigSetupItem>& setup) {
  UnevenLayout& U = c->U;
  auto put = [&](auto** dptr, const auto& vec) {
    using T = typename std::remove_reference<decltype(vec)>::type::value_type;
    if (cudaMalloc((void**)dptr, std::max<size_t>(vec.size(), 1) * sizeof(T)) != cudaSuccess) return false;
    return cudaMemcpy(*dptr, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
  };
  std::vector<PrepArgs> prep;
  U.bprep_max_omega = 0;
  for (const BigCls& bc : U.bcls) {
    PrepArgs a{c->K, c->J, bc.H * bc.Wc, c->p.rho, 1.0 / ((double)bc.H * bc.W), c->dhat + bc.dhat,
               c->pdiag + bc.pd, c->pmat + bc.pm};
    prep.push_back(a);
    U.bprep_max_omega = std::max(U.bprep_max_omega, a.Omega);
  }
  if (!put(&U.d_bcls, U.bcls) || !put(&U.d_bimg, U.bimg) || !put(&U.d_bcol, U.bcol) || !put(&U.d_brow, U.brow) ||
      !put(&U.d_bfreq, U.bfreq) || !put(&U.d_btabs, U.btabs) || !put(&U.d_bsetup, setup) || !put(&U.d_bprep, prep) ||
      cudaMalloc((void**)&U.d_by, std::max<long long>(U.n_by, 1) * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&U.d_blam, std::max<long long>(U.n_blam, 1) * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&U.d_be, std::max<size_t>(U.bfreq.size(), 1) * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&U.d_bl1, std::max<size_t>(U.brow.size(), 1) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CSC_ERR_WORKSPACE, "uneven batch: allocation of the large-image workspace failed");
  }
  return CSC_OK;
}

// the spatial route's work items and buffers: one half spectrum and one plane per image
csc_status upload_usp(Ctx* c) {
  UnevenLayout& U = c->U;
  auto put = [&](auto** dptr, const auto& vec) {
    using T = typename std::remove_reference<decltype(vec)>::type::value_type;
    if (cudaMalloc((void**)dptr, std::max<size_t>(vec.size(), 1) * sizeof(T)) != cudaSuccess) return false;
    return cudaMemcpy(*dptr, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
  };
  if (!put(&U.d_scol, U.scol) || !put(&U.d_srow, U.srow) || !put(&U.d_stile, U.stile) ||
      cudaMalloc((void**)&U.d_sy, std::max<long long>(U.n_xh, 1) * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&U.d_sq, std::max<long long>(U.n_x, 1) * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CSC_ERR_WORKSPACE, "uneven batch: allocation of the spatial route's workspace failed");
  }
  return CSC_OK;
}

// spectra of the filters (per class) and of the images (per image) of an uneven batch
cudaError_t uneven_setup(Ctx* c, const float* d, const float* x, bool solve) {
  for (int ci = 0; ci < (int)c->U.cls.size(); ++ci) {
    Ctx v;
    class_view(*c, ci, v);
    cudaError_t e = launch_fft_maps(v, d, c->K * c->J, 1, v.dhat);
    if (e == cudaSuccess && solve) e = launch_solve_prep(v);
    if (e != cudaSuccess) return e;
    c->launches += solve ? 2 : 1;
  }
  for (int n = 0; n < c->U.n_small; ++n) {
    const UImage& im = c->U.img[n];
    Ctx v;
    class_view(*c, im.cls, v);
    cudaError_t e = launch_fft_maps(v, x + im.x, c->J, 0, c->xhat + im.xh);
    if (e != cudaSuccess) return e;
    c->launches += 1;
  }
  if (!c->U.bimg.empty()) {
    const UnevenLayout& U = c->U;
    cudaError_t e = launch_big_setup(big_args(*c, nullptr, nullptr), U.d_bsetup, U.n_bsetup_rows,
                                     U.d_bsetup + U.n_bsetup_rows, U.n_bsetup_cols, d, x, c->dhat, c->xhat, c->fh,
                                     c->fw, (int)U.bcls.size(), c->stream);
    c->launches += 3;
    if (solve && e == cudaSuccess) {
      e = launch_solve_prep_batch(U.d_bprep, (int)U.bcls.size(), U.bprep_max_omega, c->nsm, c->stream);
      c->launches += 1;
    }
    if (e != cudaSuccess) return e;
  }
  if (c->dhat16) {
    cudaError_t e = launch_to_bf16(*c, c->dhat, c->dhat16, (size_t)c->U.n_dhat);
    if (e != cudaSuccess) return e;
    c->launches += 1;
  }
  return cudaSuccess;
}

// the sweeps of one coding call on an uneven batch
cudaError_t uneven_sweeps(Ctx* c, float* v, float* z, int iters) {
  const bool small = c->U.n_small > 0, big = !c->U.bimg.empty();
  const BigArgs ba = big_args(*c, v, z);
  cudaError_t e = cudaSuccess;
  if (small) {
    e = launch_sweep_uneven(uneven_args(*c, nullptr, c->part[0], v, nullptr), kPrologue, c->G, c->U.nt,
                            uneven_smem_bytes(c->U, c->J, kPrologue), c->stream);
    c->launches += 1;
  }
  if (big && e == cudaSuccess) {
    e = launch_big_sweep(ba, kPrologue, c->stream);
    c->launches += big_launches(kPrologue);
  }
  for (int t = 0; t < iters && e == cudaSuccess; ++t) {
    const int mode = (t == iters - 1) ? kLast : kIter;
    const int br = (mode == kIter) ? bracket_open(c, 0) : -1;
    if (small) {
      e = launch_sweep_uneven(uneven_args(*c, c->part[t & 1], c->part[(t + 1) & 1], v, z), mode, c->G, c->U.nt,
                              uneven_smem_bytes(c->U, c->J, mode), c->stream);
      c->launches += 1;
    }
    if (big && e == cudaSuccess) {
      e = launch_big_sweep(ba, mode, c->stream);
      c->launches += big_launches(mode);
    }
    bracket_close(c, br);
  }
  return e;
}

// the direct spatial route on an uneven batch (CSC_FLAG_SPATIAL): per iteration D on the tiles
// (q = sum_k d_k * u_k - x / rho), lambda = F^-1(P F(q)) by the one-channel transforms, then D^T and the
// state update on the tiles; P and the spectra of the setup as for the Fourier route
UspArgs usp_args(const Ctx& c, const float* x, const float* d, float* v, float* z) {
  const UnevenLayout& U = c.U;
  UspArgs a{};
  a.K = c.K; a.fh = c.fh; a.fw = c.fw;
  a.beta = (float)c.p.beta; a.rho = (float)c.p.rho;
  a.cls = U.d_bcls; a.img = U.d_bimg; a.tiles = U.d_stile; a.n_tiles = (int)U.stile.size();
  a.d = d; a.x = x; a.q = U.d_sq; a.v = v; a.z = z;
  return a;
}

cudaError_t uneven_spatial_sweeps(Ctx* c, const float* x, const float* d, float* v, float* z, int iters) {
  const UnevenLayout& U = c->U;
  BigArgs la = big_args(*c, U.d_sq, nullptr);
  la.one = 1;
  la.K = 1;
  la.col_items = U.d_scol; la.row_items = U.d_srow;
  la.n_col_items = (int)U.scol.size(); la.n_row_items = (int)U.srow.size();
  la.Y = U.d_sy;
  const UspArgs ua = usp_args(*c, x, d, v, z);
  cudaError_t e = launch_usp_conv(ua, c->stream);
  if (e == cudaSuccess) e = launch_big_lambda1(la, c->stream);
  c->launches += 4;
  for (int t = 0; t < iters && e == cudaSuccess; ++t) {
    const bool last = (t == iters - 1);
    const int br = last ? -1 : bracket_open(c, 0);
    e = launch_usp_corr(ua, last, c->stream);
    c->launches += 1;
    if (!last && e == cudaSuccess) {
      e = launch_usp_conv(ua, c->stream);
      if (e == cudaSuccess) e = launch_big_lambda1(la, c->stream);
      c->launches += 4;
    }
    bracket_close(c, br);
  }
  return e;
}

// launch shapes the autotuner picked, per (sizes, K, J, precision, device): later contexts on the
// same batch shape reuse them without timing
struct TuneKey {
  std::vector<int> dims;
  int K, J, precision, device;
  bool operator<(const TuneKey& o) const {
    if (K != o.K) return K < o.K;
    if (J != o.J) return J < o.J;
    if (precision != o.precision) return precision < o.precision;
    if (device != o.device) return device < o.device;
    return dims < o.dims;
  }
};
std::mutex g_tune_mutex;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;   // key -> (threads per CTA, CTAs per SM)

// pick threads per CTA and CTAs per SM for this batch by timing two sweeps of each candidate
csc_status uneven_autotune(Ctx* c, float* v) {
  if (c->U.n_small == 0) {
    c->U.tuned = true;
    return CSC_OK;
  }
  const TuneKey key{c->U.dims, c->K, c->J, (int)c->p.precision, c->device};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const auto hit = g_tune_cache.find(key);
    if (hit != g_tune_cache.end()) {
      const int G = (int)std::min<long long>((long long)c->nsm * hit->second.second, (long long)c->U.n_small * c->K);
      uneven_partition(c, G);
      csc_status st = upload_uneven(c);
      if (st != CSC_OK) return st;
      c->U.nt = hit->second.first;
      c->U.tuned = true;
      c->U.tune_cached = true;
      return CSC_OK;
    }
  }
  struct Cand { int nt, per_sm; };
  const Cand cands[] = {{512, 1}, {256, 1}, {256, 2}, {512, 2}};
  const size_t smem = uneven_smem_bytes(c->U, c->J, kIter);
  float best = 1e30f;
  Cand pick{512, 1};
  float* vs = nullptr;
  const size_t nv = (size_t)c->U.n_v;
  CSC_CHECK_CUDA(c, cudaMalloc((void**)&vs, nv * sizeof(float)), "autotune scratch");
  {
    const cudaError_t ec = cudaMemcpyAsync(vs, v, nv * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    if (ec != cudaSuccess) {
      cudaFree(vs);
      return cuda_fail(c, ec, "autotune copy");
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  bool timed = false;
  for (const Cand& cd : cands) {
    if (cd.per_sm * (smem + 1024) > (size_t)228 * 1024) continue;
    const int G = (int)std::min<long long>((long long)c->nsm * cd.per_sm, (long long)c->U.n_small * c->K);
    uneven_partition(c, G);
    csc_status st = upload_uneven(c);
    if (st != CSC_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cudaFree(vs);
      return st;
    }
    c->U.nt = cd.nt;
    cudaError_t e = launch_sweep_uneven(uneven_args(*c, nullptr, c->part[0], vs, nullptr), kPrologue, G, cd.nt,
                                        uneven_smem_bytes(c->U, c->J, kPrologue), c->stream);
    e = (e == cudaSuccess) ? launch_sweep_uneven(uneven_args(*c, c->part[0], c->part[1], vs, nullptr), kIter, G,
                                                 cd.nt, smem, c->stream) : e;
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r)
      e = launch_sweep_uneven(uneven_args(*c, c->part[(r + 1) & 1], c->part[r & 1], vs, nullptr), kIter, G, cd.nt,
                              smem, c->stream);
    cudaEventRecord(e1, c->stream);
    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); continue; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    timed = true;
    if (ms < best) { best = ms; pick = cd; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(vs);
  // no candidate ran: report it rather than caching an untimed default
  if (!timed) return fail(c, CSC_ERR_CUDA, "uneven autotune: no launch shape ran on this batch");
  const int G = (int)std::min<long long>((long long)c->nsm * pick.per_sm, (long long)c->U.n_small * c->K);
  uneven_partition(c, G);
  csc_status st = upload_uneven(c);
  if (st != CSC_OK) return st;
  c->U.nt = pick.nt;
  c->U.tuned = true;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[key] = {pick.nt, pick.per_sm};
  return CSC_OK;
}

}  // namespace

namespace csc {
void set_global_error(const char* msg) { g_init_error = msg; }
}  // namespace csc

extern "C" {

const char* csc_version(void) { return kVersion; }

const char* csc_last_error(const csc_ctx* ctx) {
  return ctx ? ctx->c.last_error.c_str() : g_init_error.c_str();
}

static csc_status init_ctx(const csc_params* params, int n_images, const int* dims, void* stream, csc_ctx** out,
                           bool video);

csc_status csc_init(const csc_params* params, int n_images, const int* dims, void* stream, csc_ctx** out) {
  return init_ctx(params, n_images, dims, stream, out, false);
}

// video contexts run their own frame and bin kernels: the 2-D sweep and learning limits do not apply
static csc_status init_ctx(const csc_params* params, int n_images, const int* dims, void* stream, csc_ctx** out,
                           bool video) {
  if (!params || !dims || !out) return fail(nullptr, CSC_ERR_ARG, "csc_init: null argument");
  *out = nullptr;
  const csc_params& p = *params;
  if (n_images < 1) return fail(nullptr, CSC_ERR_ARG, "csc_init: n_images must be >= 1");
  if (p.J < 1 || p.J > kMaxJ) return fail(nullptr, CSC_ERR_SHAPE, "csc_init: J must be 1..3");
  if (p.K < 1) return fail(nullptr, CSC_ERR_ARG, "csc_init: K must be >= 1");
  if (!(p.beta > 0) || !(p.rho > 0) || !std::isfinite(p.beta) || !std::isfinite(p.rho))
    return fail(nullptr, CSC_ERR_ARG, "csc_init: beta and rho must be finite and > 0");
  if (p.cg_max < 1 || !(p.cg_tol > 0)) return fail(nullptr, CSC_ERR_ARG, "csc_init: cg_max >= 1, cg_tol > 0");
  if (p.precision != CSC_FP32 && p.precision != CSC_MIXED_BF16 && p.precision != CSC_MIXED_TF32)
    return fail(nullptr, CSC_ERR_ARG, "csc_init: unknown precision");
  if (p.precision == CSC_MIXED_BF16) {
    if (p.K > 128) return fail(nullptr, CSC_ERR_SHAPE, "csc_init: CSC_MIXED_BF16 needs K <= 128");
  }
  const int fh = p.fs[0], fw = p.fs[1];
  if (fh < 1 || fw < 1 || !(fh & 1) || !(fw & 1))
    return fail(nullptr, CSC_ERR_SHAPE, "csc_init: filter support must be odd and >= 1");
  if (fw > 15) return fail(nullptr, CSC_ERR_SHAPE, "csc_init: filter width must be <= 15");
  // symmetric boundary: the context codes the half-sample symmetric extension (2H x 2W)
  const bool sym = !video && (p.flags & CSC_FLAG_SYMMETRIC_BOUNDARY);
  if (video && (p.flags & CSC_FLAG_SYMMETRIC_BOUNDARY))
    return fail(nullptr, CSC_ERR_UNSUPPORTED, "csc_init_video: no symmetric boundary on video contexts");
  const int H0 = dims[0], W0 = dims[1];
  if (sym && (H0 < 4 || W0 < 4)) return fail(nullptr, CSC_ERR_SHAPE, "csc_init: symmetric boundary needs H, W >= 4");
  const int H = sym ? 2 * H0 : H0, W = sym ? 2 * W0 : W0;
  if (H < 8 || W < 8 || (W & 1)) return fail(nullptr, CSC_ERR_SHAPE, "csc_init: need H, W >= 8 and W even");
  if (fh > H || fw > W) return fail(nullptr, CSC_ERR_SHAPE, "csc_init: filter larger than the image");

  Ctx tmp;
  tmp.sym = sym;
  tmp.H0 = H0;
  tmp.W0 = W0;
  tmp.p = p;
  tmp.N = n_images; tmp.J = p.J; tmp.K = p.K; tmp.fh = fh; tmp.fw = fw; tmp.S2 = fh * fw;
  Geometry& g = tmp.g;
  g.H = H; g.W = W; g.Wh = W / 2; g.Wc = W / 2 + 1; g.P = odd_pitch(g.Wc);
  g.Omega = H * g.Wc; g.D = H * W;
  g.ct_id = (H == 128 && W == 128) ? 1 : (H == 100 && W == 100) ? 2 : (H == 64 && W == 64) ? 3 : 0;
  g.rt.H = H; g.rt.W = W; g.rt.Wh = g.Wh; g.rt.Wc = g.Wc; g.rt.P = g.P; g.rt.Omega = g.Omega; g.rt.D = g.D;
  g.rt.rrow = factorize(g.Wh);
  g.rt.rcol = factorize(H);
  if (!radices_ok(g.rt.rrow) || !radices_ok(g.rt.rcol))
    return fail(nullptr, CSC_ERR_SHAPE, "csc_init: H and W/2 must factor into 2, 3, 5 and 7");
  if (!video && sweep_smem_bytes(g, p.J, kIter) > kSmemLimit)
    return fail(nullptr, CSC_ERR_SHAPE, "csc_init: image too large for one map per CTA in shared memory");
  tmp.stream = (cudaStream_t)stream;
  if (cudaGetDevice(&tmp.device) != cudaSuccess) return cuda_fail(nullptr, cudaGetLastError(), "cudaGetDevice");
  cudaError_t e = cudaDeviceGetAttribute(&tmp.nsm, cudaDevAttrMultiProcessorCount, tmp.device);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
  const size_t cg_smem = learn_cg_smem_bytes(tmp, false);
  if (!video && (cg_smem > kSmemLimit || !learn_cg_shape_ok(tmp)))
    return fail(nullptr, CSC_ERR_SHAPE, "csc_init: K * J * fh * fw too large for the learning kernel");
  const long long NK = (long long)tmp.N * tmp.K;
  tmp.G = (int)std::min<long long>(tmp.nsm, NK);

  csc_ctx* ctx = new (std::nothrow) csc_ctx;
  if (!ctx) return fail(nullptr, CSC_ERR_WORKSPACE, "csc_init: out of host memory");
  ctx->c = tmp;
  Ctx* c = &ctx->c;
  auto bail = [&](csc_status s) {
    g_init_error = c->last_error;
    free_all(c);
    delete ctx;
    return s;
  };
  const size_t Om = g.Omega;
  std::vector<float2> tw(g.Wh + g.H + g.Wc);
  const double pi2 = 6.283185307179586476925286766559;
  for (int t = 0; t < g.Wh; ++t) tw[t] = make_float2((float)cos(pi2 * t / g.Wh), (float)-sin(pi2 * t / g.Wh));
  for (int t = 0; t < g.H; ++t)
    tw[g.Wh + t] = make_float2((float)cos(pi2 * t / g.H), (float)-sin(pi2 * t / g.H));
  for (int t = 0; t < g.Wc; ++t)
    tw[g.Wh + g.H + t] = make_float2((float)cos(pi2 * t / g.W), (float)-sin(pi2 * t / g.W));
  if (cudaMalloc((void**)&c->tw, tw.size() * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->dhat, (size_t)p.K * p.J * Om * sizeof(float2)) != cudaSuccess ||
      (g.ct_id == 1 && p.J == 1 &&
       cudaMalloc((void**)&c->dhatp, (size_t)p.K * Om * sizeof(float2)) != cudaSuccess) ||
      (p.precision == CSC_MIXED_BF16 &&
       cudaMalloc((void**)&c->dhat16, (size_t)p.K * p.J * Om * sizeof(__nv_bfloat162)) != cudaSuccess) ||
      (p.precision == CSC_MIXED_BF16 && g.ct_id == 1 && p.J == 1 &&
       cudaMalloc((void**)&c->dhatp16, (size_t)p.K * Om * sizeof(__nv_bfloat162)) != cudaSuccess) ||
      cudaMalloc((void**)&c->xhat, (size_t)tmp.N * p.J * Om * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->pdiag, Om * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&c->pmat, Om * p.J * p.J * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->part[0], (size_t)(tmp.G + tmp.N) * p.J * Om * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->part[1], (size_t)(tmp.G + tmp.N) * p.J * Om * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->l1, tmp.G * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&c->objimg, tmp.N * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&c->err, 2 * sizeof(int)) != cudaSuccess ||
      (sym && cudaMalloc((void**)&c->xext, (size_t)tmp.N * p.J * g.D * sizeof(float)) != cudaSuccess)) {
    cudaGetLastError();
    c->last_error = "csc_init: device workspace allocation failed";
    return bail(CSC_ERR_WORKSPACE);
  }
  if (p.flags & CSC_FLAG_SPATIAL) {
    std::string why;
    if (video || !spatial_applies(*c, &why)) {
      c->last_error = "csc_init: " + (video ? std::string("direct spatial coding is for 2-D images") : why);
      return bail(CSC_ERR_UNSUPPORTED);
    }
    const size_t ob = spatial_operand_bytes(*c), plane = (size_t)tmp.N * g.D * sizeof(float);
    if (cudaMalloc((void**)&c->sp_bt, ob) != cudaSuccess || cudaMalloc((void**)&c->sp_bc, ob) != cudaSuccess ||
        cudaMalloc((void**)&c->sp_r, plane) != cudaSuccess || cudaMalloc((void**)&c->sp_lam, plane) != cudaSuccess) {
      cudaGetLastError();
      c->last_error = "csc_init: device workspace allocation failed";
      return bail(CSC_ERR_WORKSPACE);
    }
    c->spatial = true;
  }
  e = cudaMemcpy(c->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->err, 0, 2 * sizeof(int));
  if (e == cudaSuccess && c->dhatp) e = upload_f128_twiddles();
  c->cerr = c->err + 1;
  if (e != cudaSuccess) {
    c->last_error = std::string("csc_init: ") + cudaGetErrorString(e);
    return bail(CSC_ERR_CUDA);
  }
  *out = ctx;
  return CSC_OK;
}

csc_status csc_init_uneven(const csc_params* params, int n_images, const int* dims, void* stream,
                           csc_ctx** out) {
  if (!params || !dims || !out) return fail(nullptr, CSC_ERR_ARG, "csc_init_uneven: null argument");
  *out = nullptr;
  const csc_params& p = *params;
  if (n_images < 1) return fail(nullptr, CSC_ERR_ARG, "csc_init_uneven: n_images must be >= 1");
  if (p.J < 1 || p.J > kMaxJ) return fail(nullptr, CSC_ERR_SHAPE, "csc_init_uneven: J must be 1..3");
  if (p.K < 1) return fail(nullptr, CSC_ERR_ARG, "csc_init_uneven: K must be >= 1");
  if (!(p.beta > 0) || !(p.rho > 0) || !std::isfinite(p.beta) || !std::isfinite(p.rho))
    return fail(nullptr, CSC_ERR_ARG, "csc_init_uneven: beta and rho must be finite and > 0");
  if (p.precision == CSC_MIXED_TF32)
    return fail(nullptr, CSC_ERR_UNSUPPORTED, "csc_init_uneven: CSC_MIXED_TF32 is for uniform batches");
  if (p.precision != CSC_FP32 && p.precision != CSC_MIXED_BF16)
    return fail(nullptr, CSC_ERR_ARG, "csc_init_uneven: unknown precision");
  const int fh = p.fs[0], fw = p.fs[1];
  if (fh < 1 || fw < 1 || !(fh & 1) || !(fw & 1))
    return fail(nullptr, CSC_ERR_SHAPE, "csc_init_uneven: filter support must be odd and >= 1");
  const bool spatial = (p.flags & CSC_FLAG_SPATIAL) != 0;
  if (spatial) {
    if (p.J != 1 || p.precision != CSC_FP32)
      return fail(nullptr, CSC_ERR_UNSUPPORTED, "csc_init_uneven: direct spatial coding is for grey images in CSC_FP32");
    if (fh > kUspF || fw > kUspF)
      return fail(nullptr, CSC_ERR_UNSUPPORTED, "csc_init_uneven: direct spatial coding needs fh, fw <= 11");
    if (usp_smem_bytes(p.K) > kSmemLimit)
      return fail(nullptr, CSC_ERR_UNSUPPORTED, "csc_init_uneven: direct spatial coding: K filters do not fit shared memory");
    if (p.flags & CSC_FLAG_SYMMETRIC_BOUNDARY)
      return fail(nullptr, CSC_ERR_UNSUPPORTED, "csc_init_uneven: direct spatial coding takes circular boundaries");
  }
  csc_ctx* ctx = new (std::nothrow) csc_ctx;
  if (!ctx) return fail(nullptr, CSC_ERR_WORKSPACE, "csc_init_uneven: out of host memory");
  Ctx* c = &ctx->c;
  c->p = p;
  c->N = n_images; c->J = p.J; c->K = p.K; c->fh = fh; c->fw = fw; c->S2 = fh * fw;
  c->uneven = true;
  c->spatial = spatial;
  c->stream = (cudaStream_t)stream;
  auto bail = [&](csc_status st) {
    if (c->last_error.size()) g_init_error = c->last_error;
    free_all(c);
    delete ctx;
    return st;
  };
  UnevenLayout& U = c->U;
  U.dims.assign(dims, dims + 2 * (size_t)n_images);
  std::vector<Geometry> geos;
  std::vector<float2> tw;
  const double pi2 = 6.283185307179586476925286766559;
  for (int n = 0; n < n_images; ++n) {
    const int H = dims[2 * n], W = dims[2 * n + 1];
    int ci = -1, bi = -1;
    for (int q = 0; q < (int)U.cls.size(); ++q)
      if (U.cls_H[q] == H && U.cls_W[q] == W) { ci = q; break; }
    for (int q = 0; ci < 0 && q < (int)U.bcls.size(); ++q)
      if (U.bcls_H[q] == H && U.bcls_W[q] == W) { bi = q; break; }
    Geometry g;
    if (ci < 0 && bi < 0 && (spatial || check_size(p, H, W, g, "csc_init_uneven") != CSC_OK)) {
      // not one map per CTA (or the direct spatial route, whose lambda transforms are the engine's):
      // the multi-pass engine (any side up to kBigMaxSide, any factorisation)
      if (H < 8 || W < 8 || fh > H || fw > W || !big_add_class(U, H, W)) {
        char msg[160];
        std::snprintf(msg, sizeof(msg), "csc_init_uneven: image %dx%d: need 8 <= H, W <= %d and the filter inside",
                      H, W, kBigMaxSide);
        delete ctx;
        return fail(nullptr, CSC_ERR_SHAPE, msg);
      }
      g_init_error.clear();
      bi = (int)U.bcls.size() - 1;
      BigCls& bc = U.bcls[bi];
      const long long Om = (long long)H * bc.Wc;
      bc.dhat = U.n_dhat; bc.pd = U.n_pd; bc.pm = U.n_pm;
      U.n_dhat += (long long)p.K * p.J * Om;
      U.n_pd += Om;
      U.n_pm += Om * p.J * p.J;
    }
    if (bi >= 0) {
      const BigCls& bc = U.bcls[bi];
      const long long Om = (long long)H * bc.Wc;
      BigImg im;
      im.cls = bi;
      im.x = U.n_x; im.v = U.n_v; im.xh = U.n_xh;
      im.y = U.n_by; im.lam = U.n_blam;
      U.n_x += (long long)p.J * H * W;
      U.n_v += (long long)p.K * H * W;
      U.n_xh += (long long)p.J * Om;
      U.n_by += (long long)p.K * Om;
      U.n_blam += (long long)p.J * Om;
      U.bimg.push_back(im);
      continue;
    }
    if (ci < 0) {
      UClass uc;
      uc.g = g.rt;
      uc.tw = U.n_tw; uc.dhat = U.n_dhat; uc.pd = U.n_pd; uc.pm = U.n_pm;
      U.n_tw += g.Wh + g.H + g.Wc;
      U.n_dhat += (long long)p.K * p.J * g.Omega;
      U.n_pd += g.Omega;
      U.n_pm += (long long)g.Omega * p.J * p.J;
      for (int t = 0; t < g.Wh; ++t) tw.push_back(make_float2((float)cos(pi2 * t / g.Wh), (float)-sin(pi2 * t / g.Wh)));
      for (int t = 0; t < g.H; ++t) tw.push_back(make_float2((float)cos(pi2 * t / g.H), (float)-sin(pi2 * t / g.H)));
      for (int t = 0; t < g.Wc; ++t) tw.push_back(make_float2((float)cos(pi2 * t / g.W), (float)-sin(pi2 * t / g.W)));
      U.buf_elems = std::max(U.buf_elems, g.H * g.P);
      U.max_omega = std::max(U.max_omega, g.Omega);
      U.max_tw = std::max(U.max_tw, g.Wh + g.H + g.Wc);
      U.cls.push_back(uc);
      U.cls_H.push_back(H);
      U.cls_W.push_back(W);
      geos.push_back(g);
      ci = (int)U.cls.size() - 1;
    }
    UImage im;
    im.cls = ci; im.c0 = im.c1 = 0;
    im.x = U.n_x; im.v = U.n_v; im.xh = U.n_xh;
    U.n_x += (long long)p.J * geos[ci].D;
    U.n_v += (long long)p.K * geos[ci].D;
    U.n_xh += (long long)p.J * geos[ci].Omega;
    U.img.push_back(im);
  }
  U.n_small = (int)U.img.size();
  std::vector<BigSetupItem> bsetup;
  if (!U.bimg.empty()) big_build_items(U, p.K, p.J, fh, fw, bsetup);
  if (spatial) big_build_one_channel(U);
  if (uneven_smem_bytes(U, p.J, kIter) > kSmemLimit) {
    delete ctx;
    return fail(nullptr, CSC_ERR_SHAPE, "csc_init_uneven: the largest image and the largest spectrum do not fit one CTA");
  }
  c->g = geos.empty() ? Geometry{} : geos[0];
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    c->last_error = "csc_init_uneven: no CUDA device";
    return bail(CSC_ERR_CUDA);
  }
  uneven_partition(c, (int)std::min<long long>(c->nsm, (long long)U.n_small * p.K));
  if (cudaMalloc((void**)&c->tw, std::max<size_t>(tw.size(), 1) * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->dhat, U.n_dhat * sizeof(float2)) != cudaSuccess ||
      (p.precision == CSC_MIXED_BF16 &&
       cudaMalloc((void**)&c->dhat16, U.n_dhat * sizeof(__nv_bfloat162)) != cudaSuccess) ||
      cudaMalloc((void**)&c->pdiag, U.n_pd * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&c->pmat, U.n_pm * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->xhat, U.n_xh * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->objimg, n_images * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&c->err, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    c->last_error = "csc_init_uneven: device workspace allocation failed";
    return bail(CSC_ERR_WORKSPACE);
  }
  c->cerr = c->err + 1;
  if (cudaMemcpy(c->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->err, 0, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    c->last_error = "csc_init_uneven: upload failed";
    return bail(CSC_ERR_CUDA);
  }
  if (upload_uneven(c) != CSC_OK) return bail(CSC_ERR_WORKSPACE);
  if (!U.bimg.empty() && upload_big(c, bsetup) != CSC_OK) return bail(CSC_ERR_WORKSPACE);
  if (spatial && upload_usp(c) != CSC_OK) return bail(CSC_ERR_WORKSPACE);
  *out = ctx;
  return CSC_OK;
}

// ---- video tensors --------------------------------------------------------------------------

csc_status csc_init_video(const csc_params* params, int ft, int n_videos, const int* dims, void* stream,
                          csc_ctx** out) {
  if (!params || !dims || !out) return fail(nullptr, CSC_ERR_ARG, "csc_init_video: null argument");
  *out = nullptr;
  const int T = dims[0], H = dims[1], W = dims[2];
  if (H != 128 || W != 128) return fail(nullptr, CSC_ERR_SHAPE, "csc_init_video: frames must be 128 x 128");
  if (T < 1 || T > video_max_T()) return fail(nullptr, CSC_ERR_SHAPE, "csc_init_video: T must be 1..64");
  if (ft < 1 || !(ft & 1) || ft > 7 || ft > T)
    return fail(nullptr, CSC_ERR_SHAPE, "csc_init_video: time support must be odd, <= 7 and <= T");
  if (params->precision != CSC_FP32) return fail(nullptr, CSC_ERR_UNSUPPORTED, "csc_init_video: CSC_FP32 only");
  if (params->flags & CSC_FLAG_SYMMETRIC_BOUNDARY)
    return fail(nullptr, CSC_ERR_UNSUPPORTED, "csc_init_video: the symmetric boundary is for 2-D batches");
  const int hw[2] = {H, W};
  csc_status s = init_ctx(params, n_videos, hw, stream, out, true);
  if (s != CSC_OK) return s;
  Ctx* c = &(*out)->c;
  c->video = true;
  c->T = T;
  c->ft = ft;
  const size_t OM = (size_t)c->g.Omega;
  const size_t nmaps = std::max((size_t)c->K * c->J * ft, (size_t)c->N * c->J * T);
  if (cudaMalloc((void**)&c->vS, (size_t)c->N * c->K * T * OM * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->vd2, (size_t)c->K * c->J * ft * OM * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->vx3, (size_t)c->N * c->J * T * OM * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->vp3, (size_t)T * OM * c->J * c->J * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->vtmp, nmaps * OM * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->vobj, (size_t)c->N * video_bin_blocks() * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&c->vl1, (size_t)c->nsm * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    csc_destroy(*out);
    *out = nullptr;
    return fail(nullptr, CSC_ERR_WORKSPACE, "csc_init_video: device workspace allocation failed");
  }
  return CSC_OK;
}

static VideoArgs video_args(const Ctx* c, float* v, float* z) {
  VideoArgs a;
  a.N = c->N; a.K = c->K; a.J = c->J; a.T = c->T; a.ft = c->ft;
  a.beta = (float)c->p.beta; a.rho = (float)c->p.rho;
  a.tw = c->tw; a.S = c->vS; a.v = v; a.z = z; a.l1 = c->vl1;
  a.d2 = c->vd2; a.xh3 = c->vx3; a.p3 = c->vp3; a.objpart = c->vobj;
  return a;
}

// filter tap spectra, x_hat at the 3-D frequencies and the per-frequency systems
static cudaError_t video_setup(Ctx* c, const VideoArgs& a, const float* dd, const float* xd) {
  cudaError_t e = launch_fft_maps(*c, dd, c->K * c->J * c->ft, 1, c->vtmp);
  if (e == cudaSuccess) e = launch_permute_f128(c->vtmp, c->vd2, c->K * c->J * c->ft, *c);
  if (e == cudaSuccess) e = launch_fft_maps(*c, xd, c->N * c->J * c->T, 0, c->vtmp);
  if (e == cudaSuccess) e = launch_video_setup(a, c->vtmp, c->stream);
  c->launches += 4;
  return e;
}

static csc_status video_code(Ctx* c, const float* x, const float* d, float* v, float* z, int iters) {
  const size_t D = (size_t)c->g.D;
  const size_t nx = (size_t)c->N * c->J * c->T * D, nd = (size_t)c->K * c->J * c->ft * c->S2;
  const size_t nv = (size_t)c->N * c->K * c->T * D;
  const float *xd = nullptr, *dd = nullptr, *vd_c = nullptr;
  csc_status s;
  if ((s = stage_in(c, v, &c->st_v, nv, &vd_c, true)) != CSC_OK) return s;
  float* vd = const_cast<float*>(vd_c);
  const bool v_host = (vd != v);
  float* zd = nullptr;
  bool z_host = false;
  if (z) {
    if (is_device_ptr(z)) zd = z;
    else {
      CSC_CHECK_CUDA(c, ensure_alloc(&c->st_z, nv), "staging allocation");
      zd = c->st_z;
      z_host = true;
    }
  }
  if (iters == 0) {
    if (zd) {
      CSC_CHECK_CUDA(c, launch_codes_from_state_n(*c, vd, zd, nv), "codes");
      c->launches += 1;
    }
  } else {
    if ((s = stage_in(c, x, &c->st_x, nx, &xd, true)) != CSC_OK) return s;
    if ((s = stage_in(c, d, &c->st_d, nd, &dd, true)) != CSC_OK) return s;
    const VideoArgs a = video_args(c, vd, zd);
    const int G = c->nsm;
    CSC_CHECK_CUDA(c, video_setup(c, a, dd, xd), "video setup");
    CSC_CHECK_CUDA(c, launch_video_frames(a, kPrologue, G, c->stream), "video prologue");
    c->launches += 1;
    for (int t = 0; t < iters; ++t) {
      const int br = (t < iters - 1) ? bracket_open(c, 0) : -1;
      CSC_CHECK_CUDA(c, launch_video_bins(a, kIter, c->stream), "video bins");
      CSC_CHECK_CUDA(c, launch_video_frames(a, t == iters - 1 ? kLast : kIter, G, c->stream), "video frames");
      bracket_close(c, br);
      c->launches += 2;
    }
  }
  if (v_host) CSC_CHECK_CUDA(c, cudaMemcpyAsync(v, vd, nv * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "v copy");
  if (z_host) CSC_CHECK_CUDA(c, cudaMemcpyAsync(z, zd, nv * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "z copy");
  if (v_host || z_host || (xd && xd != x) || (dd && dd != d))
    CSC_CHECK_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
  return CSC_OK;
}

static csc_status video_objective(Ctx* c, const float* x, const float* d, const float* z, double* out) {
  const size_t D = (size_t)c->g.D;
  const size_t nx = (size_t)c->N * c->J * c->T * D, nd = (size_t)c->K * c->J * c->ft * c->S2;
  const size_t nz = (size_t)c->N * c->K * c->T * D;
  const float *xd, *dd, *zd;
  csc_status s;
  if ((s = stage_in(c, x, &c->st_x, nx, &xd, true)) != CSC_OK) return s;
  if ((s = stage_in(c, d, &c->st_d, nd, &dd, true)) != CSC_OK) return s;
  if ((s = stage_in(c, z, &c->st_z, nz, &zd, true)) != CSC_OK) return s;
  const VideoArgs a = video_args(c, nullptr, const_cast<float*>(zd));
  const int G = c->nsm;
  CSC_CHECK_CUDA(c, video_setup(c, a, dd, xd), "video setup");
  CSC_CHECK_CUDA(c, launch_video_frames(a, kObjective, G, c->stream), "video codes spectra");
  CSC_CHECK_CUDA(c, launch_video_bins(a, kObjective, c->stream), "video residual");
  c->launches += 2;
  const int nb = c->N * video_bin_blocks();
  std::vector<double> parts(nb), l1(G);
  CSC_CHECK_CUDA(c, cudaMemcpyAsync(parts.data(), c->vobj, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                 "objective copy");
  CSC_CHECK_CUDA(c, cudaMemcpyAsync(l1.data(), c->vl1, G * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                 "objective copy");
  CSC_CHECK_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
  double e2 = 0.0, a1 = 0.0;
  for (double p : parts) e2 += p;
  for (double p : l1) a1 += p;
  *out = 0.5 * e2 + c->p.beta * a1;
  return CSC_OK;
}

csc_status csc_describe(const csc_ctx* ctx, char* buf, int len) {
  if (!ctx || !buf || len < 1) return fail(nullptr, CSC_ERR_ARG, "csc_describe: null argument");
  const Ctx& c = ctx->c;
  const int n_cls = c.uneven ? (int)c.U.cls.size() : 1;
  const int n_big = c.uneven ? (int)c.U.bcls.size() : 0;
  std::snprintf(buf, (size_t)len,
                "{\"N\": %d, \"K\": %d, \"J\": %d, \"uneven\": %s, \"size_classes\": %d, "
                "\"large_size_classes\": %d, \"large_images\": %d, \"ctas\": %d, "
                "\"threads_per_cta\": %d, \"autotuned\": %s, \"autotune_cached\": %s, \"graph\": %s, "
                "\"graph_recorded\": %s, "
                "\"video\": %s, \"T\": %d, \"ft\": %d, \"spatial\": %s}",
                c.N, c.K, c.J, c.uneven ? "true" : "false", n_cls, n_big, c.uneven ? (int)c.U.bimg.size() : 0, c.G,
                c.uneven ? c.U.nt : (int)kNTSweep,
                (c.uneven && c.U.tuned) ? "true" : "false", (c.uneven && c.U.tune_cached) ? "true" : "false",
                (c.p.flags & CSC_FLAG_GRAPH) ? "true" : "false",
                c.graph ? "true" : "false", c.video ? "true" : "false", c.T, c.ft, c.spatial ? "true" : "false");
  return CSC_OK;
}

void csc_destroy(csc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->c.device);
  cudaStreamSynchronize(ctx->c.stream);
  free_all(&ctx->c);
  delete ctx;
}

// symmetric-boundary contexts: stage the caller's H x W images (host or device) and write their
// half-sample symmetric extension into the context's 2H x 2W image buffer, which the call then uses
static csc_status sym_images(Ctx* c, const float** x) {
  if (!c->sym) return CSC_OK;
  const float* xd = nullptr;
  csc_status s = stage_in(c, *x, &c->st_x, (size_t)c->N * c->J * c->H0 * c->W0, &xd, true);
  if (s != CSC_OK) return s;
  CSC_CHECK_CUDA(c, launch_symmetric_extend(*c, xd, c->xext), "symmetric extension");
  c->launches += 1;
  *x = c->xext;
  return CSC_OK;
}

csc_status csc_code(csc_ctx* ctx, const float* x, const float* d, float* v, float* z, int iters) {
  if (!ctx) return fail(nullptr, CSC_ERR_ARG, "csc_code: null context");
  Ctx* c = &ctx->c;
  if (!x || !d || !v) return fail(c, CSC_ERR_ARG, "csc_code: x, d and v must be non-null");
  if (iters < 0) return fail(c, CSC_ERR_ARG, "csc_code: iters must be >= 0");
  CSC_CHECK_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  {
    const csc_status s0 = (iters > 0) ? sym_images(c, &x) : CSC_OK;
    if (s0 != CSC_OK) return s0;
  }
  if (c->video) return video_code(c, x, d, v, z, iters);
  const size_t nx = c->uneven ? (size_t)c->U.n_x : (size_t)c->N * c->J * c->g.D;
  const size_t nd = (size_t)c->K * c->J * c->S2;
  const size_t nv = c->uneven ? (size_t)c->U.n_v : (size_t)c->N * c->K * c->g.D;
  const float *xd = nullptr, *dd = nullptr, *vd_c = nullptr;
  csc_status s;
  if ((s = stage_in(c, v, &c->st_v, nv, &vd_c, true)) != CSC_OK) return s;
  float* vd = const_cast<float*>(vd_c);
  const bool v_host = (vd != v);
  float* zd = nullptr;
  bool z_host = false;
  if (z) {
    if (is_device_ptr(z)) zd = z;
    else {
      CSC_CHECK_CUDA(c, ensure_alloc(&c->st_z, nv), "staging allocation");
      zd = c->st_z;
      z_host = true;
    }
  }
  if (iters > 0) {
    if ((s = stage_in(c, x, &c->st_x, nx, &xd, true)) != CSC_OK) return s;
    if ((s = stage_in(c, d, &c->st_d, nd, &dd, true)) != CSC_OK) return s;
  }
  if (c->spatial && !c->uneven && iters > 0 && (reinterpret_cast<uintptr_t>(vd) & 15))
    return fail(c, CSC_ERR_ARG, "csc_code: direct spatial coding needs v 16-byte aligned (its rows are bulk copies)");
  if (c->uneven && iters > 0 && !c->U.tuned) {
    if (c->U.n_small > 0) CSC_CHECK_CUDA(c, uneven_setup(c, dd, xd, true), "uneven setup");
    if ((s = uneven_autotune(c, vd)) != CSC_OK) return s;
  }
  // the launch sequence of this call
  auto enqueue = [&]() -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(c->cerr, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    if (iters == 0) {
      if (!zd) return cudaSuccess;
      c->launches += 1;
      return launch_codes_from_state_n(*c, vd, zd, nv);
    }
    if (c->uneven) {
      e = uneven_setup(c, dd, xd, true);
      if (e == cudaSuccess) e = c->spatial ? uneven_spatial_sweeps(c, xd, dd, vd, zd, iters) : uneven_sweeps(c, vd, zd, iters);
      return e;
    }
    e = launch_fft_maps(*c, dd, c->K * c->J, 1, c->dhat);
    if (e == cudaSuccess) e = launch_solve_prep(*c);
    if (e == cudaSuccess) e = launch_fft_maps(*c, xd, c->N * c->J, 0, c->xhat);
    if (c->spatial) {
      // direct spatial D and D^T on the tensor cores; P from the filter spectra as above
      if (e == cudaSuccess) e = launch_spatial_operands(*c, dd);
      c->launches += 4;
      for (int t = 0; t < iters && e == cudaSuccess; ++t) {
        const bool last = (t == iters - 1);
        const int br = last ? -1 : bracket_open(c, 0);
        e = launch_spatial_conv(*c, vd);
        if (e == cudaSuccess) e = launch_spatial_lambda(*c, xd);
        if (e == cudaSuccess) e = launch_spatial_corr(*c, vd, zd, last);
        bracket_close(c, br);
        c->launches += 3;
      }
      return e;
    }
    if (e == cudaSuccess && c->p.precision == CSC_MIXED_BF16) {
      e = launch_to_bf16(*c, c->dhat, c->dhat16, (size_t)c->K * c->J * c->g.Omega);
      // and the copy in the thread order of the fused 128 x 128 sweep
      if (e == cudaSuccess && c->dhatp16) {
        e = launch_to_bf16(*c, c->dhatp, c->dhatp16, (size_t)c->K * c->g.Omega);
        c->launches += 1;
      }
      c->launches += 1;
    }
    if (e == cudaSuccess) e = launch_sweep(*c, kPrologue, nullptr, c->part[0], vd, nullptr);
    c->launches += 4;
    for (int t = 0; t < iters && e == cudaSuccess; ++t) {
      const int mode = (t == iters - 1) ? kLast : kIter;
      const int br = (mode == kIter) ? bracket_open(c, 0) : -1;
      e = launch_sweep(*c, mode, c->part[t & 1], c->part[(t + 1) & 1], vd, zd);
      bracket_close(c, br);
      c->launches += 1;
    }
    return e;
  };
  const bool all_dev = !v_host && !z_host && (iters == 0 || (xd == x && dd == d));
  const void* key[5] = {x, d, v, z, nullptr};
  const bool same = c->graph && c->graph_iters == iters && key[0] == c->graph_key[0] && key[1] == c->graph_key[1] &&
                    key[2] == c->graph_key[2] && key[3] == c->graph_key[3];
  if ((c->p.flags & CSC_FLAG_GRAPH) && all_dev && same) {
    CSC_CHECK_CUDA(c, cudaGraphLaunch(c->graph, c->stream), "graph launch");
  } else {
    CSC_CHECK_CUDA(c, enqueue(), "coding launch");
    if ((c->p.flags & CSC_FLAG_GRAPH) && all_dev) {
      // record the sequence for later calls with the same arrays
      if (c->graph) cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
      if (!c->cap_stream) CSC_CHECK_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "stream");
      cudaStream_t user = c->stream;
      const bool timing = c->timing;
      const long long launches = c->launches;
      c->timing = false;
      c->stream = c->cap_stream;
      cudaGraph_t gr = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
      cudaError_t e2 = (e == cudaSuccess) ? enqueue() : e;
      cudaError_t e3 = (e == cudaSuccess) ? cudaStreamEndCapture(c->cap_stream, &gr) : e;
      c->stream = user;
      c->timing = timing;
      c->launches = launches;
      if (e2 == cudaSuccess && e3 == cudaSuccess && gr) {
        if (cudaGraphInstantiate(&c->graph, gr, 0) == cudaSuccess) {
          for (int i = 0; i < 4; ++i) c->graph_key[i] = key[i];
          c->graph_iters = iters;
        } else {
          c->graph = nullptr;
        }
      }
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
    }
  }
  if (v_host) CSC_CHECK_CUDA(c, cudaMemcpyAsync(v, vd, nv * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "v copy");
  if (z_host) CSC_CHECK_CUDA(c, cudaMemcpyAsync(z, zd, nv * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "z copy");
  const bool sync = v_host || z_host || (xd && xd != x) || (dd && dd != d);
  if (sync || (c->p.flags & CSC_FLAG_CHECK_FINITE)) {
    // a synchronous call reports the sweeps' non-finite flag at its end
    int herr = 0;
    CSC_CHECK_CUDA(c, cudaMemcpyAsync(&herr, c->cerr, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flag copy");
    CSC_CHECK_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    if (herr == CSC_ERR_TIMEOUT) return fail(c, CSC_ERR_TIMEOUT, "csc_code: a bounded wait of the spatial products gave up");
    if (herr) return fail(c, (csc_status)herr, "csc_code: a non-finite value reached the dual variable");
  }
  return CSC_OK;
}

csc_status csc_check(csc_ctx* ctx) {
  if (!ctx) return fail(nullptr, CSC_ERR_ARG, "csc_check: null context");
  Ctx* c = &ctx->c;
  CSC_CHECK_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  int herr[2] = {0, 0};
  CSC_CHECK_CUDA(c, cudaMemcpyAsync(herr, c->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flag copy");
  CSC_CHECK_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
  if (herr[1]) return fail(c, (csc_status)herr[1], "csc_check: a non-finite value reached the dual variable in csc_code");
  return CSC_OK;
}

csc_status csc_set_wait_limit(csc_ctx* ctx, long long clocks) {
  if (!ctx) return fail(nullptr, CSC_ERR_ARG, "csc_set_wait_limit: null context");
  if (clocks < 0) return fail(&ctx->c, CSC_ERR_ARG, "csc_set_wait_limit: clocks must be >= 0");
  ctx->c.wait_limit = clocks;
  return CSC_OK;
}

csc_status csc_objective(csc_ctx* ctx, const float* x, const float* d, const float* z, double* out) {
  if (!ctx) return fail(nullptr, CSC_ERR_ARG, "csc_objective: null context");
  Ctx* c = &ctx->c;
  if (!x || !d || !z || !out) return fail(c, CSC_ERR_ARG, "csc_objective: null argument");
  CSC_CHECK_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  {
    const csc_status s0 = sym_images(c, &x);
    if (s0 != CSC_OK) return s0;
  }
  if (c->video) return video_objective(c, x, d, z, out);
  const size_t nx = c->uneven ? (size_t)c->U.n_x : (size_t)c->N * c->J * c->g.D;
  const size_t nd = (size_t)c->K * c->J * c->S2;
  const size_t nz = c->uneven ? (size_t)c->U.n_v : (size_t)c->N * c->K * c->g.D;
  const float *xd, *dd, *zd;
  csc_status s;
  if ((s = stage_in(c, x, &c->st_x, nx, &xd, true)) != CSC_OK) return s;
  if ((s = stage_in(c, d, &c->st_d, nd, &dd, true)) != CSC_OK) return s;
  if ((s = stage_in(c, z, &c->st_z, nz, &zd, true)) != CSC_OK) return s;
  std::vector<double> big_e, big_l1;
  if (c->uneven) {
    CSC_CHECK_CUDA(c, uneven_setup(c, dd, xd, false), "uneven setup");
    if (c->U.n_small > 0) {
      UnevenArgs ua = uneven_args(*c, nullptr, c->part[0], nullptr, const_cast<float*>(zd));
      ua.dhat16 = nullptr;   // the objective stays float32 in every mode
      CSC_CHECK_CUDA(c, launch_sweep_uneven(ua, kObjective, c->G, c->U.nt,
                                            uneven_smem_bytes(c->U, c->J, kObjective), c->stream), "objective sweep");
      CSC_CHECK_CUDA(c, launch_objective_final_uneven(uneven_args(*c, c->part[0], nullptr, nullptr, nullptr),
                                                      c->objimg, c->stream), "objective reduction");
      c->launches += 2;
    }
    if (!c->U.bimg.empty()) {
      CSC_CHECK_CUDA(c, launch_big_sweep(big_args(*c, nullptr, const_cast<float*>(zd)), kObjective, c->stream),
                     "objective sweep (large images)");
      c->launches += big_launches(kObjective);
      big_e.resize(c->U.bfreq.size());
      big_l1.resize(c->U.brow.size());
      CSC_CHECK_CUDA(c, cudaMemcpyAsync(big_e.data(), c->U.d_be, big_e.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                        c->stream), "objective copy");
      CSC_CHECK_CUDA(c, cudaMemcpyAsync(big_l1.data(), c->U.d_bl1, big_l1.size() * sizeof(double),
                                        cudaMemcpyDeviceToHost, c->stream), "objective copy");
    }
  } else {
    CSC_CHECK_CUDA(c, launch_fft_maps(*c, dd, c->K * c->J, 1, c->dhat), "filter spectra");
    CSC_CHECK_CUDA(c, launch_fft_maps(*c, xd, c->N * c->J, 0, c->xhat), "image spectra");
    CSC_CHECK_CUDA(c, launch_sweep(*c, kObjective, nullptr, c->part[0], nullptr, const_cast<float*>(zd)),
                   "objective sweep");
    CSC_CHECK_CUDA(c, launch_objective_final(*c, c->part[0], c->objimg), "objective reduction");
    c->launches += 4;
  }
  const int n_img = c->uneven ? c->U.n_small : c->N;
  std::vector<double> img(n_img), l1(c->G);
  if (n_img > 0) {
    CSC_CHECK_CUDA(c, cudaMemcpyAsync(img.data(), c->objimg, n_img * sizeof(double), cudaMemcpyDeviceToHost,
                                      c->stream), "objective copy");
    CSC_CHECK_CUDA(c, cudaMemcpyAsync(l1.data(), c->l1, c->G * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                   "objective copy");
  }
  CSC_CHECK_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
  double data = 0.0, reg = 0.0;
  for (double v : img) data += v;
  for (double v : l1) reg += v;
  for (double v : big_e) data += v;
  for (double v : big_l1) reg += v;
  const double f = 0.5 * data + c->p.beta * reg;
  if (!std::isfinite(f)) return fail(c, CSC_ERR_NONFINITE, "csc_objective: non-finite objective");
  *out = f;
  return CSC_OK;
}

// workspace of the 2-D learning path (allocated on first use) and the per-step iteration buffer
static csc_status learn_prepare(Ctx* c, int steps, const char* who) {
  const int K = c->K, J = c->J;
  const size_t nd = (size_t)K * J * c->S2, Om = c->g.Omega;
  const size_t npairs = (size_t)K * (K + 1) / 2;
  const int La = 2 * c->fh - 1, Lb = 2 * c->fw - 1;
  LearnBuffers& L = c->L;
  if (!L.ready) {
    if (ensure_alloc(&L.zhat, (size_t)c->N * K * Om) != cudaSuccess ||
        ensure_alloc(&L.gram, npairs * Om) != cudaSuccess ||
        ensure_alloc(&L.lags, (size_t)K * K * La * Lb) != cudaSuccess ||
        ensure_alloc(&L.chat, (size_t)La * c->fw * K * (K + 1) / 2) != cudaSuccess ||
        ensure_alloc(&L.yw, (size_t)2 * K * J * La * c->fw) != cudaSuccess ||
        ensure_alloc(&L.zw, nd) != cudaSuccess ||
        ensure_alloc(&L.b, nd) != cudaSuccess || ensure_alloc(&L.vec, 4 * nd) != cudaSuccess ||
        ensure_alloc(&L.mu, (size_t)K) != cudaSuccess ||
        (gram_tc_applies(*c) && (ensure_alloc(&L.rspec, (size_t)K * J * Om) != cudaSuccess ||
                                 ensure_alloc(&L.zt, (size_t)c->N * K * Om) != cudaSuccess ||
                                 ensure_alloc(&L.lagT, lag_sep_T_count(*c)) != cudaSuccess)) ||
        ensure_alloc(&L.slots, (size_t)2 * c->nsm * 4 * kMaxJ) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, CSC_ERR_WORKSPACE, std::string(who) + ": device workspace allocation failed");
    }
    L.ready = true;
  }
  if (steps > L.steps_cap) {
    if (L.iters) cudaFree(L.iters);
    L.iters = nullptr;
    CSC_CHECK_CUDA(c, ensure_alloc(&L.iters, (size_t)steps), "iteration buffer");
    L.steps_cap = steps;
  }
  return CSC_OK;
}

// the sums over this context's images: code Gram -> lags L.lags (and their spectra L.chat), and the
// right-hand side L.b = S Z^T x
static csc_status learn_stats_enqueue(Ctx* c, const float* xd, const float* zd) {
  const int K = c->K, J = c->J;
  LearnBuffers& L = c->L;
  CSC_CHECK_CUDA(c, launch_fft_maps(*c, xd, c->N * J, 0, c->xhat), "image spectra");
  // the per-frequency Gram on the tensor cores (3xTF32 in float32, BF16 in the mixed mode), with the
  // right-hand-side spectra as J extra columns, when K + J <= 128; otherwise on the CUDA cores
  if (gram_tc_applies(*c)) {
    CSC_CHECK_CUDA(c, launch_code_spectra(*c, zd, c->N * K, L.zhat), "code spectra");
    CSC_CHECK_CUDA(c, launch_spectra_transpose(*c, L.zhat, c->N * K, L.zt), "code spectra transpose");
    CSC_CHECK_CUDA(c, launch_learn_gram_tc(*c, c->p.precision, L.rspec, c->err),
                   "code Gram (tensor cores)");
    CSC_CHECK_CUDA(c, launch_learn_rhs(*c, L.rspec), "learning right-hand side");
    CSC_CHECK_CUDA(c, launch_learn_lags_sep(*c), "code lags");
    c->launches += 4;
  } else {
    CSC_CHECK_CUDA(c, launch_code_spectra(*c, zd, c->N * K, L.zhat), "code spectra");
    CSC_CHECK_CUDA(c, launch_learn_gram(*c), "code Gram");
    CSC_CHECK_CUDA(c, launch_learn_rhs(*c, nullptr), "learning right-hand side");
    CSC_CHECK_CUDA(c, launch_learn_lags(*c), "code lags");
    c->launches += 3;
  }
  c->launches += 1;   // image spectra (the lag kernels count themselves)
  return CSC_OK;
}

// the CG steps from L.lags / L.chat / L.b, then d, mu and the iteration counts back to the caller
static csc_status learn_solve_finish(Ctx* c, float* dd, float* d, double* mu, int steps, int* cg_iters, int br) {
  const int K = c->K;
  const size_t nd = (size_t)K * c->J * c->S2;
  LearnBuffers& L = c->L;
  const bool mu_dev = is_device_ptr(mu);
  CSC_CHECK_CUDA(c, cudaMemcpyAsync(L.mu, mu, K * sizeof(double),
                                    mu_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
                 "mu copy");
  CSC_CHECK_CUDA(c, launch_learn_cg(*c, dd, steps, c->err), "learning CG");
  bracket_close(c, br);
  c->launches += 1;
  if (dd != d) CSC_CHECK_CUDA(c, cudaMemcpyAsync(d, dd, nd * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "d copy");
  CSC_CHECK_CUDA(c, cudaMemcpyAsync(mu, L.mu, K * sizeof(double),
                                    mu_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
                 "mu copy");
  int herr = 0;
  CSC_CHECK_CUDA(c, cudaMemcpyAsync(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flag copy");
  std::vector<int> its(std::max(steps, 1));
  if ((cg_iters || (c->p.flags & CSC_FLAG_CG_STRICT)) && steps > 0)
    CSC_CHECK_CUDA(c, cudaMemcpyAsync(its.data(), L.iters, steps * sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                   "iteration copy");
  CSC_CHECK_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
  if (herr == CSC_ERR_NONFINITE) return fail(c, CSC_ERR_NONFINITE, "csc_learn: a code, CG residual or step was not finite");
  if (herr) return fail(c, (csc_status)herr, "csc_learn: grid barrier timed out");
  if (cg_iters && steps > 0) std::memcpy(cg_iters, its.data(), steps * sizeof(int));
  if (c->p.flags & CSC_FLAG_CG_STRICT)
    for (int i = 0; i < steps; ++i)
      if (its[i] >= c->p.cg_max)
        return fail(c, CSC_ERR_NOT_CONVERGED, "csc_learn: a CG solve stopped at cg_max iterations");
  return CSC_OK;
}

csc_status csc_learn(csc_ctx* ctx, const float* x, const float* z, float* d, double* mu, int steps,
                     int* cg_iters) {
  if (!ctx) return fail(nullptr, CSC_ERR_ARG, "csc_learn: null context");
  Ctx* c = &ctx->c;
  if (c->uneven) return fail(c, CSC_ERR_UNSUPPORTED, "csc_learn: not available on an uneven-batch context");
  if (!x || !z || !d || !mu) return fail(c, CSC_ERR_ARG, "csc_learn: null argument");
  if (steps < 0) return fail(c, CSC_ERR_ARG, "csc_learn: steps must be >= 0");
  CSC_CHECK_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (c->video) {
    if (!video_learn_shape_ok(*c))
      return fail(c, CSC_ERR_SHAPE, "csc_learn: video learning needs fh, fw <= 12, K + J <= 128, T <= 64");
    const size_t D3 = (size_t)c->T * c->g.D;
    const size_t vx = (size_t)c->N * c->J * D3, vz = (size_t)c->N * c->K * D3;
    const size_t vd = (size_t)c->K * c->J * c->ft * c->fh * c->fw;
    const float *xd, *zd, *dd_c;
    csc_status s;
    if ((s = stage_in(c, x, &c->st_x, vx, &xd, true)) != CSC_OK) return s;
    if ((s = stage_in(c, z, &c->st_z, vz, &zd, true)) != CSC_OK) return s;
    if ((s = stage_in(c, (const float*)d, &c->st_d, vd, &dd_c, true)) != CSC_OK) return s;
    float* dd = const_cast<float*>(dd_c);
    CSC_CHECK_CUDA(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream), "memset");
    const int br = bracket_open(c, 1);
    if ((s = video_learn(c, xd, zd, dd, mu, steps)) != CSC_OK) return s;
    bracket_close(c, br);
    if (dd != d) CSC_CHECK_CUDA(c, cudaMemcpyAsync(d, dd, vd * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "d copy");
    int herr = 0;
    CSC_CHECK_CUDA(c, cudaMemcpyAsync(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flag copy");
    std::vector<int> its(std::max(steps, 1));
    if (steps > 0)
      CSC_CHECK_CUDA(c, cudaMemcpyAsync(its.data(), c->VL.iters, steps * sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                     "iteration copy");
    CSC_CHECK_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    if (herr == CSC_ERR_NONFINITE) return fail(c, CSC_ERR_NONFINITE, "csc_learn: a code or image value was not finite");
    if (herr) return fail(c, (csc_status)herr, "csc_learn: a device wait (tensor-core Gram or CG exchange) timed out");
    if (cg_iters && steps > 0) std::memcpy(cg_iters, its.data(), steps * sizeof(int));
    if (c->p.flags & CSC_FLAG_CG_STRICT)
      for (int i = 0; i < steps; ++i)
        if (its[i] >= c->p.cg_max)
          return fail(c, CSC_ERR_NOT_CONVERGED, "csc_learn: a CG solve stopped at cg_max iterations");
    return CSC_OK;
  }
  csc_status s;
  if ((s = sym_images(c, &x)) != CSC_OK) return s;
  if ((s = learn_prepare(c, steps, "csc_learn")) != CSC_OK) return s;
  const size_t nx = (size_t)c->N * c->J * c->g.D, nd = (size_t)c->K * c->J * c->S2;
  const size_t nz = (size_t)c->N * c->K * c->g.D;
  const float *xd, *zd, *dd_c;
  if ((s = stage_in(c, x, &c->st_x, nx, &xd, true)) != CSC_OK) return s;
  if ((s = stage_in(c, z, &c->st_z, nz, &zd, true)) != CSC_OK) return s;
  if ((s = stage_in(c, (const float*)d, &c->st_d, nd, &dd_c, true)) != CSC_OK) return s;
  CSC_CHECK_CUDA(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream), "memset");
  const int br = bracket_open(c, 1);
  if ((s = learn_stats_enqueue(c, xd, zd)) != CSC_OK) return s;
  return learn_solve_finish(c, const_cast<float*>(dd_c), d, mu, steps, cg_iters, br);
}

csc_status csc_learn_stats(csc_ctx* ctx, const float* x, const float* z, float* C, float* b) {
  if (!ctx) return fail(nullptr, CSC_ERR_ARG, "csc_learn_stats: null context");
  Ctx* c = &ctx->c;
  if (c->uneven || c->video)
    return fail(c, CSC_ERR_UNSUPPORTED, "csc_learn_stats: uniform 2-D batches only");
  if (!x || !z || !C || !b) return fail(c, CSC_ERR_ARG, "csc_learn_stats: null argument");
  CSC_CHECK_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  csc_status s;
  if ((s = sym_images(c, &x)) != CSC_OK) return s;
  if ((s = learn_prepare(c, 0, "csc_learn_stats")) != CSC_OK) return s;
  const size_t nx = (size_t)c->N * c->J * c->g.D, nz = (size_t)c->N * c->K * c->g.D;
  const size_t nd = (size_t)c->K * c->J * c->S2;
  const size_t nC = (size_t)c->K * c->K * (2 * c->fh - 1) * (2 * c->fw - 1);
  const float *xd, *zd;
  if ((s = stage_in(c, x, &c->st_x, nx, &xd, true)) != CSC_OK) return s;
  if ((s = stage_in(c, z, &c->st_z, nz, &zd, true)) != CSC_OK) return s;
  CSC_CHECK_CUDA(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream), "memset");
  if ((s = learn_stats_enqueue(c, xd, zd)) != CSC_OK) return s;
  CSC_CHECK_CUDA(c, cudaMemcpyAsync(C, c->L.lags, nC * sizeof(float), cudaMemcpyDefault, c->stream), "C copy");
  CSC_CHECK_CUDA(c, cudaMemcpyAsync(b, c->L.b, nd * sizeof(float), cudaMemcpyDefault, c->stream), "b copy");
  int herr = 0;
  CSC_CHECK_CUDA(c, cudaMemcpyAsync(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flag copy");
  CSC_CHECK_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
  if (herr) return fail(c, (csc_status)herr, "csc_learn_stats: tensor-core Gram wait timed out");
  return CSC_OK;
}

csc_status csc_learn_solve(csc_ctx* ctx, const float* C, const float* b, float* d, double* mu, int steps,
                           int* cg_iters) {
  if (!ctx) return fail(nullptr, CSC_ERR_ARG, "csc_learn_solve: null context");
  Ctx* c = &ctx->c;
  if (c->uneven || c->video)
    return fail(c, CSC_ERR_UNSUPPORTED, "csc_learn_solve: uniform 2-D batches only");
  if (!C || !b || !d || !mu) return fail(c, CSC_ERR_ARG, "csc_learn_solve: null argument");
  if (steps < 0) return fail(c, CSC_ERR_ARG, "csc_learn_solve: steps must be >= 0");
  CSC_CHECK_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  csc_status s;
  if ((s = learn_prepare(c, steps, "csc_learn_solve")) != CSC_OK) return s;
  const size_t nd = (size_t)c->K * c->J * c->S2;
  const size_t nC = (size_t)c->K * c->K * (2 * c->fh - 1) * (2 * c->fw - 1);
  const float* dd_c;
  if ((s = stage_in(c, (const float*)d, &c->st_d, nd, &dd_c, true)) != CSC_OK) return s;
  CSC_CHECK_CUDA(c, cudaMemcpyAsync(c->L.lags, C, nC * sizeof(float), cudaMemcpyDefault, c->stream), "C copy");
  CSC_CHECK_CUDA(c, cudaMemcpyAsync(c->L.b, b, nd * sizeof(float), cudaMemcpyDefault, c->stream), "b copy");
  CSC_CHECK_CUDA(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream), "memset");
  const int br = bracket_open(c, 1);
  CSC_CHECK_CUDA(c, launch_lag_spectra(*c), "lag spectra");
  return learn_solve_finish(c, const_cast<float*>(dd_c), d, mu, steps, cg_iters, br);
}

// ------------------------------------------------------------------------------------------------
// reverse mode through unrolled coding iterations, and the reconstruction D z
// ------------------------------------------------------------------------------------------------
namespace {

struct TapeLayout {
  size_t ckpt, vT, lam, total;
  int n_ckpt;
};

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

TapeLayout tape_layout(const Ctx& c, int iters, int every) {
  TapeLayout t;
  const size_t state = (size_t)c.N * c.K * c.g.D * sizeof(float);
  const size_t lam = (size_t)c.N * c.J * c.g.Omega * sizeof(float2);
  t.n_ckpt = (iters + every - 1) / every;
  t.ckpt = 0;
  t.vT = up256((size_t)t.n_ckpt * state);
  t.lam = t.vT + up256(state);
  t.total = t.lam + up256((size_t)iters * lam);
  return t;
}

csc_status check_device_arrays(Ctx* c, std::initializer_list<const void*> ptrs, const char* who) {
  for (const void* p : ptrs)
    if (p && !is_device_ptr(p))
      return fail(c, CSC_ERR_ARG, std::string(who) + ": arrays must be device memory");
  return CSC_OK;
}

csc_status ensure_backward(Ctx* c, int seg) {
  BackwardBuffers& B = c->B;
  const size_t state = (size_t)c->N * c->K * c->g.D;
  const size_t Om = c->g.Omega;
  if (seg > B.seg_cap) {
    if (B.seg) cudaFree(B.seg);
    B.seg = nullptr;
    B.seg_cap = 0;
    CSC_CHECK_CUDA(c, cudaMalloc((void**)&B.seg, (size_t)seg * state * sizeof(float)), "backward workspace");
    B.seg_cap = seg;
  }
  if (ensure_alloc(&B.vbar, state) != cudaSuccess || ensure_alloc(&B.gspec, (size_t)c->N * c->K * Om) != cudaSuccess ||
      ensure_alloc(&B.S, (size_t)c->N * Om) != cudaSuccess || ensure_alloc(&B.Xb, (size_t)c->N * Om) != cudaSuccess ||
      ensure_alloc(&B.part[0], (size_t)(c->G + c->N) * Om) != cudaSuccess ||
      ensure_alloc(&B.part[1], (size_t)(c->G + c->N) * Om) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CSC_ERR_WORKSPACE, "backward workspace allocation failed");
  }
  return CSC_OK;
}

csc_status ensure_spec(Ctx* c) {
  if (ensure_alloc(&c->B.spec, (size_t)c->N * c->J * c->g.Omega) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CSC_ERR_WORKSPACE, "spectrum workspace allocation failed");
  }
  return CSC_OK;
}

}  // namespace

size_t csc_tape_bytes(const csc_ctx* ctx, int iters, int every) {
  if (!ctx || iters < 1 || every < 1 || ctx->c.uneven || ctx->c.video || ctx->c.sym) return 0;   // no reverse mode there
  return tape_layout(ctx->c, iters, every).total;
}

csc_status csc_code_unrolled(csc_ctx* ctx, const float* x, const float* d, float* v, float* z, int iters,
                             int every, void* tape) {
  if (!ctx) return fail(nullptr, CSC_ERR_ARG, "csc_code_unrolled: null context");
  Ctx* c = &ctx->c;
  if (c->uneven || c->sym)
    return fail(c, CSC_ERR_UNSUPPORTED, "csc_code_unrolled: not available on uneven-batch or symmetric-boundary contexts");
  if (c->video) return fail(c, CSC_ERR_UNSUPPORTED, "csc_code_unrolled: not available on a video context");
  if (!x || !d || !v || !tape || iters < 1 || every < 1)
    return fail(c, CSC_ERR_ARG, "csc_code_unrolled: null array, iters < 1 or every < 1");
  if (c->J != 1) return fail(c, CSC_ERR_UNSUPPORTED, "csc_code_unrolled: J = 1 only");
  if (c->p.precision != CSC_FP32) return fail(c, CSC_ERR_UNSUPPORTED, "csc_code_unrolled: CSC_FP32 only");
  CSC_CHECK_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  csc_status s = check_device_arrays(c, {x, d, v, z, tape}, "csc_code_unrolled");
  if (s != CSC_OK) return s;
  const TapeLayout T = tape_layout(*c, iters, every);
  unsigned char* tp = static_cast<unsigned char*>(tape);
  const size_t state = (size_t)c->N * c->K * c->g.D;
  float* ckpt = reinterpret_cast<float*>(tp + T.ckpt);
  float* vT = reinterpret_cast<float*>(tp + T.vT);
  float2* lam = reinterpret_cast<float2*>(tp + T.lam);
  const size_t lam_n = (size_t)c->N * c->J * c->g.Omega;
  CSC_CHECK_CUDA(c, launch_fft_maps(*c, d, c->K * c->J, 1, c->dhat), "filter spectra");
  CSC_CHECK_CUDA(c, launch_solve_prep(*c), "per-frequency solve setup");
  CSC_CHECK_CUDA(c, launch_fft_maps(*c, x, c->N * c->J, 0, c->xhat), "image spectra");
  CSC_CHECK_CUDA(c, launch_sweep(*c, kPrologue, nullptr, c->part[0], v, nullptr), "coding prologue");
  c->launches += 4;
  for (int t = 0; t < iters; ++t) {
    if (t % every == 0)
      CSC_CHECK_CUDA(c, cudaMemcpyAsync(ckpt + (size_t)(t / every) * state, v, state * sizeof(float),
                                        cudaMemcpyDeviceToDevice, c->stream), "checkpoint copy");
    const int mode = (t == iters - 1) ? kLast : kIter;
    CSC_CHECK_CUDA(c, launch_sweep_ex(*c, mode, c->part[t & 1], c->part[(t + 1) & 1], v, z, nullptr,
                                      lam + (size_t)t * lam_n), "coding sweep");
    c->launches += 1;
  }
  CSC_CHECK_CUDA(c, cudaMemcpyAsync(vT, v, state * sizeof(float), cudaMemcpyDeviceToDevice, c->stream), "state copy");
  return CSC_OK;
}

csc_status csc_code_backward(csc_ctx* ctx, const float* x, const float* d, const void* tape, int iters, int every,
                             const float* gz, float* gx, float* gd) {
  if (!ctx) return fail(nullptr, CSC_ERR_ARG, "csc_code_backward: null context");
  Ctx* c = &ctx->c;
  if (c->uneven || c->sym)
    return fail(c, CSC_ERR_UNSUPPORTED, "csc_code_backward: not available on uneven-batch or symmetric-boundary contexts");
  if (c->video) return fail(c, CSC_ERR_UNSUPPORTED, "csc_code_backward: not available on a video context");
  if (!x || !d || !tape || !gz || !gx || !gd || iters < 1 || every < 1)
    return fail(c, CSC_ERR_ARG, "csc_code_backward: null array, iters < 1 or every < 1");
  if (c->J != 1) return fail(c, CSC_ERR_UNSUPPORTED, "csc_code_backward: J = 1 only");
  if (c->p.precision != CSC_FP32) return fail(c, CSC_ERR_UNSUPPORTED, "csc_code_backward: CSC_FP32 only");
  CSC_CHECK_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  csc_status s = check_device_arrays(c, {x, d, tape, gz, gx, gd}, "csc_code_backward");
  if (s != CSC_OK) return s;
  if ((s = ensure_backward(c, std::min(every, iters))) != CSC_OK) return s;
  const TapeLayout T = tape_layout(*c, iters, every);
  const unsigned char* tp = static_cast<const unsigned char*>(tape);
  const size_t state = (size_t)c->N * c->K * c->g.D;
  const float* ckpt = reinterpret_cast<const float*>(tp + T.ckpt);
  const float* vT = reinterpret_cast<const float*>(tp + T.vT);
  const float2* lam = reinterpret_cast<const float2*>(tp + T.lam);
  const size_t lam_n = (size_t)c->N * c->g.Omega;
  BackwardBuffers& B = c->B;
  CSC_CHECK_CUDA(c, launch_fft_maps(*c, d, c->K, 1, c->dhat), "filter spectra");
  CSC_CHECK_CUDA(c, launch_solve_prep(*c), "per-frequency solve setup");
  CSC_CHECK_CUDA(c, launch_fft_maps(*c, x, c->N, 0, c->xhat), "image spectra");
  CSC_CHECK_CUDA(c, cudaMemsetAsync(B.S, 0, (size_t)c->N * c->g.Omega * sizeof(float), c->stream), "memset");
  CSC_CHECK_CUDA(c, cudaMemsetAsync(B.Xb, 0, (size_t)c->N * c->g.Omega * sizeof(float2), c->stream), "memset");
  c->launches += 3;
  BwdArgs a;
  a.N = c->N; a.K = c->K; a.G = c->G;
  a.beta = (float)c->p.beta; a.rho = (float)c->p.rho; a.dsize = (float)c->g.D;
  a.dhat = c->dhat; a.pdiag = c->pdiag; a.vbar = B.vbar; a.gz = gz; a.gspec = B.gspec; a.S = B.S; a.Xb = B.Xb;
  a.tw = c->tw;
  const GeoOps& ops = geo_ops(*c);
  // seed: vbar^T = rho (m_T - 1) z_bar
  a.part_in = nullptr; a.part_out = B.part[0]; a.vt = vT; a.lam_t = nullptr;
  a.lam_prev = lam + (size_t)(iters - 1) * lam_n;
  CSC_CHECK_CUDA(c, ops.bwd(*c, kBSeed, a), "backward seed");
  c->launches += 1;
  int cur = 0;
  for (int sgm = T.n_ckpt - 1; sgm >= 0; --sgm) {
    const int t0 = sgm * every, t1 = std::min(iters, t0 + every);
    // recompute the forward states v^t0 .. v^(t1-1) of the segment from its checkpoint
    CSC_CHECK_CUDA(c, cudaMemcpyAsync(B.seg, ckpt + (size_t)sgm * state, state * sizeof(float),
                                      cudaMemcpyDeviceToDevice, c->stream), "checkpoint restore");
    if (t1 - t0 > 1) {
      CSC_CHECK_CUDA(c, launch_sweep(*c, kPrologue, nullptr, c->part[0], B.seg, nullptr), "recompute prologue");
      c->launches += 1;
      for (int t = t0; t < t1 - 1; ++t) {
        const int i = t - t0;
        CSC_CHECK_CUDA(c, launch_sweep_ex(*c, kIter, c->part[i & 1], c->part[(i + 1) & 1], B.seg + (size_t)i * state,
                                          nullptr, B.seg + (size_t)(i + 1) * state, nullptr), "recompute sweep");
        c->launches += 1;
      }
    }
    for (int t = t1 - 1; t >= t0; --t) {
      a.part_in = B.part[cur];
      a.part_out = B.part[cur ^ 1];
      a.vt = B.seg + (size_t)(t - t0) * state;
      a.lam_t = lam + (size_t)t * lam_n;
      a.lam_prev = t >= 1 ? lam + (size_t)(t - 1) * lam_n : nullptr;
      CSC_CHECK_CUDA(c, ops.bwd(*c, t == 0 ? kBLast : kBIter, a), "backward sweep");
      c->launches += 1;
      cur ^= 1;
    }
  }
  CSC_CHECK_CUDA(c, ops.spec_maps(*c, B.Xb, c->N, 1.0f, gx), "input gradient");
  CSC_CHECK_CUDA(c, ops.dgrad(*c, B.gspec, B.S, gd), "filter gradient");
  c->launches += 2;
  return CSC_OK;
}

csc_status csc_synthesize(csc_ctx* ctx, const float* d, const float* z, float* out) {
  if (!ctx) return fail(nullptr, CSC_ERR_ARG, "csc_synthesize: null context");
  Ctx* c = &ctx->c;
  if (c->uneven) return fail(c, CSC_ERR_UNSUPPORTED, "csc_synthesize: not available on an uneven-batch context");
  if (c->video) return fail(c, CSC_ERR_UNSUPPORTED, "csc_synthesize: not available on a video context");
  if (!d || !z || !out) return fail(c, CSC_ERR_ARG, "csc_synthesize: null argument");
  if (c->p.precision != CSC_FP32) return fail(c, CSC_ERR_UNSUPPORTED, "csc_synthesize: CSC_FP32 only");
  CSC_CHECK_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  csc_status s = check_device_arrays(c, {d, z, out}, "csc_synthesize");
  if (s != CSC_OK) return s;
  if ((s = ensure_spec(c)) != CSC_OK) return s;
  CSC_CHECK_CUDA(c, launch_fft_maps(*c, d, c->K * c->J, 1, c->dhat), "filter spectra");
  CSC_CHECK_CUDA(c, launch_sweep(*c, kObjective, nullptr, c->part[0], nullptr, const_cast<float*>(z)), "synthesis");
  CSC_CHECK_CUDA(c, launch_sum_slots(*c, c->part[0], c->B.spec), "synthesis sum");
  CSC_CHECK_CUDA(c, geo_ops(*c).spec_maps(*c, c->B.spec, c->N * c->J, 1.0f / (float)c->g.D, out), "synthesis inverse");
  c->launches += 4;
  return CSC_OK;
}

csc_status csc_synthesize_backward(csc_ctx* ctx, const float* d, const float* z, const float* gout, float* gz,
                                   float* gd) {
  if (!ctx) return fail(nullptr, CSC_ERR_ARG, "csc_synthesize_backward: null context");
  Ctx* c = &ctx->c;
  if (c->uneven) return fail(c, CSC_ERR_UNSUPPORTED, "csc_synthesize_backward: not available on an uneven-batch context");
  if (c->video) return fail(c, CSC_ERR_UNSUPPORTED, "csc_synthesize_backward: not available on a video context");
  if (!d || !z || !gout || !gz || !gd) return fail(c, CSC_ERR_ARG, "csc_synthesize_backward: null argument");
  if (c->J != 1) return fail(c, CSC_ERR_UNSUPPORTED, "csc_synthesize_backward: J = 1 only");
  if (c->p.precision != CSC_FP32) return fail(c, CSC_ERR_UNSUPPORTED, "csc_synthesize_backward: CSC_FP32 only");
  CSC_CHECK_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  csc_status s = check_device_arrays(c, {d, z, gout, gz, gd}, "csc_synthesize_backward");
  if (s != CSC_OK) return s;
  if ((s = ensure_spec(c)) != CSC_OK) return s;
  if (ensure_alloc(&c->L.zhat, (size_t)c->N * c->K * c->g.Omega) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CSC_ERR_WORKSPACE, "csc_synthesize_backward: workspace allocation failed");
  }
  const GeoOps& ops = geo_ops(*c);
  CSC_CHECK_CUDA(c, launch_fft_maps(*c, d, c->K, 1, c->dhat), "filter spectra");
  CSC_CHECK_CUDA(c, launch_fft_maps(*c, gout, c->N, 0, c->B.spec), "gradient spectra");
  CSC_CHECK_CUDA(c, ops.expand(*c, c->B.spec, 1.0f / (float)c->g.D, gz), "code gradient");
  CSC_CHECK_CUDA(c, launch_code_spectra(*c, z, c->N * c->K, c->L.zhat), "code spectra");
  CSC_CHECK_CUDA(c, ops.rhs_ex(*c, c->L.zhat, c->B.spec, gd), "filter gradient");
  c->launches += 5;
  return CSC_OK;
}

csc_status csc_timing_enable(csc_ctx* ctx, int enable) {
  if (!ctx) return fail(nullptr, CSC_ERR_ARG, "csc_timing_enable: null context");
  ctx->c.timing = enable != 0;
  return CSC_OK;
}

csc_status csc_timing_read(csc_ctx* ctx, csc_timing* out) {
  if (!ctx || !out) return fail(ctx ? &ctx->c : nullptr, CSC_ERR_ARG, "csc_timing_read: null argument");
  Ctx* c = &ctx->c;
  CSC_CHECK_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  CSC_CHECK_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
  csc_timing t{0.0, 0, 0.0, 0, c->launches};
  for (size_t i = 0; i < c->events_used; ++i) {
    float ms = 0.f;
    CSC_CHECK_CUDA(c, cudaEventElapsedTime(&ms, c->events[i].a, c->events[i].b), "cudaEventElapsedTime");
    if (c->events[i].kind == 0) { t.sweep_ms += ms; t.sweep_launches += 1; }
    else { t.learn_ms += ms; t.learn_calls += 1; }
  }
  c->events_used = 0;
  c->launches = 0;
  *out = t;
  return CSC_OK;
}

}  // extern "C"
