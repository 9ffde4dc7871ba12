// Internal declarations shared by the translation units of libcsc.so.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/csc.h"
#include "fft.cuh"

namespace csc {

constexpr int kNT = 512;              // threads of the per-map kernels
constexpr int kNTSweep = 512;         // threads of the coding sweep
constexpr int kMaxJ = 3;
constexpr size_t kSmemLimit = 232448; // 227 KB opt-in shared memory per CTA
constexpr double kMuFloor = 1e-8;

enum SweepMode { kPrologue = 0, kIter = 1, kLast = 2, kObjective = 3 };

// arguments of the coding sweep (one launch = one pass over all N*K maps)
struct SweepArgs {
  int N, K, J, G;        // images, filters, channels, CTAs in the launch
  float beta, rho;
  const float2* dhat;    // [K][J][Omega]
  const float2* xhat;    // [N][J][Omega]
  const float* pdiag;    // J == 1: [Omega] 1/(sum_k |dhat_k|^2 + 1/rho) / D
  const float2* pmat;    // J > 1: [Omega][J][J] (A + I/rho)^{-1} / D
  const float2* part_in; // [(G+N)][J][Omega] partial sums of the previous sweep
  float2* part_out;      // [(G+N)][J][Omega]
  float* v;              // [N][K][D] ADMM state
  float* z;              // [N][K][D] codes: written by kLast (may be null), read by kObjective
  double* l1;            // [G] per-CTA sum |z| (kObjective)
  const float2* tw;      // twiddles [Wh | H | Wc]
  int vec4;              // v, z 16-byte aligned and D % 16 == 0: 4-pixel vector path + L2 prefetch
  float* v_out;          // iterate/last: new state written here instead of over v (may be null)
  const __nv_bfloat162* dhat16;  // mixed precision: d_hat in bf16; contraction operands rounded to bf16
  float2* lam_store;     // iterate/last: lambda_hat / D of each image stored here [N][J][Omega] (may be null)
  int* err;              // set to CSC_ERR_NONFINITE when a lambda_hat formed by the sweep is not finite (may be null)
  int tf32;              // CSC_MIXED_TF32: contraction operands rounded to TF32 (float32 accumulation)
};

struct Ctx;

// ---- video tensors (video.cu): J x T x 128 x 128, filters ft x fh x fw ---------------------------
struct VideoArgs {
  int N, K, J, T, ft;
  float beta, rho;
  const float2* tw;    // the context's twiddles [Wh | H | Wc]
  float2* S;           // [N][K][T][8320] per-frame 2-D spectra, thread-major bins
  float* v;            // [N][K][T][128][128]
  float* z;            // [N][K][T][128][128]
  double* l1;          // [grid] per-CTA sum |z| (objective)
  const float2* d2;    // [K][J][ft][8320] 2-D spectra of the filters' time taps
  float2* xh3;         // [N][J][T][8320] x_hat at the 3-D frequencies (time frequency tau)
  float2* p3;          // [T][8320][J][J] (A + I/rho)^{-1} / (128 * 128)
  double* objpart;     // [N][bin blocks] residual energy (objective)
};
size_t video_frames_smem_bytes();
int video_max_T();
int video_bin_blocks();
cudaError_t launch_video_frames(const VideoArgs& a, int mode, int G, cudaStream_t st);
cudaError_t launch_video_bins(const VideoArgs& a, int mode, cudaStream_t st);
cudaError_t launch_video_setup(const VideoArgs& a, const float2* x2, cudaStream_t st);
cudaError_t launch_permute_f128(const float2* in, float2* out, int nmaps, const Ctx& c);

// ---- batches of images of different sizes (uneven.cu) ------------------------------------------
struct UClass {            // one image size: run-time FFT plan and offsets of its per-class data
  GeoRT g;
  long long tw, dhat, pd, pm;   // element offsets into the twiddle, d_hat, P (diag / J x J) buffers
};
struct UImage {
  int cls, c0, c1;         // size class; first and last CTA whose map range covers the image
  long long x, v, xh;      // element offsets of its images (x), maps (v, z) and image spectra
};
struct UnevenArgs {
  int N, K, J, G;
  float beta, rho;
  int buf_elems, max_omega;
  const UClass* cls;
  const UImage* img;
  const long long* mstart;  // [G+1] map range of each CTA (global map index n*K + k)
  const long long* slot;    // [G+N] partial-sum slot offset (float2) of (cta, image), indexed by cta + n
  const float2* tw;
  const float2* dhat;
  const __nv_bfloat162* dhat16;   // mixed precision: bf16 copy of dhat (contraction operands), else null
  const float* pdiag;
  const float2* pmat;
  const float2* xhat;
  const float2* part_in;
  float2* part_out;
  float* v;
  float* z;
  double* l1;
};
// the per-frequency system (A(w) + I/rho)^{-1} / D of one filter spectrum (coding.cu)
struct PrepArgs {
  int K, J, Omega;
  double rho, invD;
  const float2* dhat;
  float* pdiag;
  float2* pmat;
};
cudaError_t launch_solve_prep_batch(const PrepArgs* list, int n, int max_omega, int nsm, cudaStream_t st);

// ---- uneven-batch images beyond the one-map-per-CTA sweep (uneven_big.cu) -------------------------
struct BigPlan {          // a length-n complex DFT
  int n;
  int M;                  // 0: Stockham plan of n (7-smooth); else Bluestein length M >= 2n - 1 (a power of two)
  Radices rad;            // radices of n, or of M
  long long tw;           // twiddles exp(-2 pi i t / L), L = n or M: element offset into the tables
  long long chirp, bhat;  // Bluestein: w_j = exp(-pi i j^2 / n) (n), FFT_M of the conjugate chirp / M (M)
  long long twn;          // exp(-2 pi i t / n), t < n (direct DFTs of the filters)
};
struct BigCls {
  int H, W, Wc;           // Wc = W/2 + 1 stored columns (both parities)
  int col_ls, row_ls;     // line pitch of the column / row passes in shared memory (>= n and >= M)
  BigPlan pcol, prow;     // lengths H and W
  long long dhat, pd, pm; // offsets of the class's d_hat, P diagonal, P blocks (the uneven buffers)
};
struct BigImg {
  int cls;
  long long x, v, xh;     // offsets in the uneven batch's arrays (user order)
  long long y, lam;       // offsets of its K map spectra and its J lambda_hat in the big workspaces
};
struct BigItem {          // an image's map (or, for frequency items, the image) and a range
  int img, map, first, count;
};
struct BigSetupItem {      // rows or columns [first, first + count) of one map of the setup transforms
  int cls, first, count, filter;
  long long src;          // filter: element offset of its [fh][fw] taps in d; image: of its [H][W] plane in x
  long long dst;          // element offset of its half spectrum [H][Wc] in d_hat (filter) or x_hat (image)
};
struct BigArgs {
  int K, J;
  float beta, rho;
  const BigCls* cls;
  const BigImg* img;
  const BigItem* col_items;
  const BigItem* row_items;
  const BigItem* freq_items;
  int n_col_items, n_row_items, n_freq_items;
  size_t col_smem, row_smem;   // bytes of the lines of a column / row work item; the twiddles follow
  int tw_max;                   // longest twiddle table of the plans
  const float2* tabs;
  const float2* dhat;
  const __nv_bfloat162* dhat16;   // mixed precision: bf16 copy of dhat (contraction operands), else null
  const float* pdiag;
  const float2* pmat;
  const float2* xhat;
  float2* Y;
  float2* lam;
  float* v;
  float* z;
  double* e_items;        // [n_freq_items] residual energy (objective)
  double* l1_items;       // [n_row_items] sum |z| (objective)
  int one;                // one-channel item lists (direct spatial route): Y at the image's x_hat offset,
                          // the spatial plane (v) at its x offset
};
constexpr int kBigMaxSide = 1024;
cudaError_t launch_big_sweep(const BigArgs& a, int mode, cudaStream_t st);
cudaError_t launch_big_setup(const BigArgs& a, const BigSetupItem* row_items, int n_rows,
                             const BigSetupItem* col_items, int n_cols, const float* d, const float* x,
                             float2* dhat, float2* xhat, int fh, int fw, int n_classes, cudaStream_t st);
struct UnevenLayout;
// plans (and their tables, appended to L.btabs) of a new H x W class; false if a side is out of range
bool big_add_class(UnevenLayout& L, int H, int W);
// the work-item lists of the sweeps and of the setup, from L.bcls / L.bimg
void big_build_items(UnevenLayout& L, int K, int J, int fh, int fw, std::vector<BigSetupItem>& setup);

// ---- direct spatial coding of an uneven batch (uneven_spatial.cu, CSC_FLAG_SPATIAL, J = 1) -------
// D and D^T as correlations on the CUDA cores over output tiles of kUspTileH x kUspTileW pixels,
// filters zero-padded to kUspF x kUspF about their centre; lambda by the engine's one-channel transforms
constexpr int kUspTileH = 32, kUspTileW = 64, kUspF = 11;
struct UspTile {
  int img, y0, x0, pad;
};
struct UspArgs {
  int K, fh, fw;
  float beta, rho;
  const BigCls* cls;
  const BigImg* img;
  const UspTile* tiles;
  int n_tiles;
  const float* d;     // [K][fh][fw] filters
  const float* x;     // images (offset im.x)
  float* q;           // conv: q = sum_k d_k * u_k - x / rho (offset im.x); then lambda, in place
  float* v;           // [K][H][W] per image (offset im.v) ADMM state
  float* z;           // corr, last iteration: codes (may be null)
};
size_t usp_smem_bytes(int K);
cudaError_t launch_usp_conv(const UspArgs& a, cudaStream_t st);
cudaError_t launch_usp_corr(const UspArgs& a, bool last, cudaStream_t st);
// lambda = F^-1(P F(q)) per image in place on q: the one-channel row and column passes (3 launches)
cudaError_t launch_big_lambda1(const BigArgs& a, cudaStream_t st);
// the one-channel column and row work items and the output tiles of the spatial route, from L.bimg
void big_build_one_channel(UnevenLayout& L);

struct UnevenLayout {
  std::vector<UClass> cls;
  std::vector<UImage> img;
  std::vector<int> cls_H, cls_W;
  std::vector<long long> mstart, slot;
  int buf_elems = 0, max_omega = 0, max_tw = 0;
  int n_small = 0;          // images coded by the one-map-per-CTA sweep (U.img); the rest are in bimg
  // images the one-map-per-CTA sweep cannot hold, coded by uneven_big.cu
  std::vector<BigCls> bcls;
  std::vector<BigImg> bimg;
  std::vector<int> bcls_H, bcls_W;
  std::vector<float2> btabs;
  std::vector<BigPlan> bplans;   // one per transform length, shared by the classes
  std::vector<BigItem> bcol, brow, bfreq;
  size_t bcol_smem = 0, brow_smem = 0;
  int btw_max = 0;
  long long n_by = 0, n_blam = 0;
  BigCls* d_bcls = nullptr;
  BigImg* d_bimg = nullptr;
  BigItem* d_bcol = nullptr;
  BigItem* d_brow = nullptr;
  BigItem* d_bfreq = nullptr;
  float2* d_btabs = nullptr;
  float2* d_by = nullptr;
  float2* d_blam = nullptr;
  double* d_be = nullptr;
  double* d_bl1 = nullptr;
  BigSetupItem* d_bsetup = nullptr;
  PrepArgs* d_bprep = nullptr;   // the classes' per-frequency systems, one launch
  int bprep_max_omega = 0;
  int n_bsetup_rows = 0, n_bsetup_cols = 0;
  // direct spatial route (CSC_FLAG_SPATIAL): one-channel transform items, output tiles, buffers
  std::vector<BigItem> scol, srow;
  std::vector<UspTile> stile;
  BigItem* d_scol = nullptr;
  BigItem* d_srow = nullptr;
  UspTile* d_stile = nullptr;
  float2* d_sy = nullptr;     // one half spectrum per image (x_hat offsets)
  float* d_sq = nullptr;      // q, then lambda, one plane per image (x offsets)
  long long n_tw = 0, n_dhat = 0, n_pd = 0, n_pm = 0, n_x = 0, n_v = 0, n_xh = 0, n_slot = 0;
  UClass* d_cls = nullptr;
  UImage* d_img = nullptr;
  long long* d_mstart = nullptr;
  long long* d_slot = nullptr;
  int nt = 512;             // threads per CTA of the sweep (autotuned)
  bool tuned = false;
  bool tune_cached = false;  // the launch shape came from an earlier batch with the same key
  std::vector<int> dims;    // (H, W) per image in user order: the autotuner cache key with K, J, precision
};
size_t uneven_smem_bytes(const UnevenLayout& L, int J, int mode);
cudaError_t launch_sweep_uneven(const UnevenArgs& a, int mode, int G, int nt, size_t smem, cudaStream_t st);
cudaError_t launch_objective_final_uneven(const UnevenArgs& a, double* out, cudaStream_t st);

// geometry of the (uniform) batch, chosen at csc_init
struct Geometry {
  int H, W, Wh, Wc, P, Omega, D;
  int ct_id;     // 0: run-time geometry; 1: 128x128; 2: 100x100; 3: 64x64
  GeoRT rt;
};

struct LearnBuffers {
  bool ready = false;
  float2* zhat = nullptr;   // [N][K][Omega]
  float2* gram = nullptr;   // [npairs][Omega], pairs k <= k' (CUDA-core Gram), or [Omega][npairs] in
                            // column order k'(k'+1)/2 + k (tensor-core Gram)
  float* lags = nullptr;    // [K][K][L*L]
  float2* chat = nullptr;   // [NF][K(K+1)/2] lag spectra / (La Lb), NF = La * fw
  unsigned long long* yw = nullptr;   // the CG product spectrum, [K][J][NF] c64 (allocated as 2x that)
  unsigned long long* zw = nullptr;   // the CG's z = M^-1 r, [K][J][S2] f32 (allocated as 2x that)
  float* b = nullptr;       // [K][J][S2]
  float* vec = nullptr;     // r, z, p, Ap: 4 x [K][J][S2]
  double* mu = nullptr;     // [K]
  unsigned long long* slots = nullptr;   // CG partial sums [2][G][4 kMaxJ] f32, then the arrival counter
  int* iters = nullptr;     // [steps_cap]
  int steps_cap = 0;
  float2* rspec = nullptr;  // [K][J][Omega] right-hand-side spectra from the tensor-core Gram
  float2* zt = nullptr;     // [Omega][N K] frequency-major code spectra for the tensor-core Gram
  float2* lagT = nullptr;   // [H][2 fw - 1][npairs] row sums of the separable lag transform
};

// video learning workspace (video_learn.cu), allocated on the first csc_learn of a video context
struct VideoLearnBuffers {
  float2* z3 = nullptr;      // [N K][T][Omega] codes' 3-D spectra
  float2* zt = nullptr;      // [T Omega][N K] frequency-major
  float2* x2 = nullptr;      // [N J T][Omega] images' per-frame spectra
  float2* x3 = nullptr;      // [N J][T][Omega]
  float2* gram = nullptr;    // [T Omega][K(K+1)/2] (column pair order)
  float2* rspec = nullptr;   // [K J][T Omega]
  float2* rspecT = nullptr;  // [T Omega][K J]
  float2* U = nullptr;       // [T][items][window] partial inverse DFTs
  float2* tab = nullptr;     // twiddle tables of the partial inverse DFTs
  float* lags = nullptr;     // [K][K][2ft-1][2fh-1][2fw-1]
  float2* chat = nullptr;    // [(2ft-1)(2fh-1) fw][K(K+1)/2]
  float* vec = nullptr;      // b, r, z, p, y: 5 x [K][J][ft fh fw]
  float2* phat = nullptr;    // [K J][bins]
  float2* yhat = nullptr;
  double* mu = nullptr;
  int* active = nullptr;
  float* fscal = nullptr;    // [2][K] per-step float scalars of the CG
  double* part = nullptr;    // per-block partial sums of the CG iterations
  void* st = nullptr;        // CG scalars and flags
  int* iters = nullptr;
  int iters_cap = 0;
  unsigned long long* words = nullptr;   // exchange words of the persistent CG (video_cg.cu)
};

struct BackwardBuffers {
  int seg_cap = 0;          // states the segment buffer holds
  float* seg = nullptr;     // [seg_cap][N][K][D] recomputed forward states
  float* vbar = nullptr;    // [N][K][D]
  float2* gspec = nullptr;  // [N][K][Omega]
  float* S = nullptr;       // [N][Omega]
  float2* Xb = nullptr;     // [N][Omega]
  float2* part[2] = {nullptr, nullptr};
  float2* spec = nullptr;   // [N][J][Omega] scratch spectra
};

struct Ctx {
  csc_params p;
  int N, J, K, fh, fw, S2;
  // symmetric image boundary (CSC_FLAG_SYMMETRIC_BOUNDARY): the caller's images are H0 x W0, the
  // context codes their half-sample symmetric extension (g = 2 H0 x 2 W0) from xext
  bool sym = false;
  int H0 = 0, W0 = 0;
  float* xext = nullptr;
  Geometry g;
  cudaStream_t stream;
  int device = 0, nsm = 0;
  int G;                    // CTAs of the coding sweep
  size_t sweep_smem;
  // workspace
  float2* tw = nullptr;
  float2* dhat = nullptr;
  float2* dhatp = nullptr;            // 128 x 128, J = 1: d_hat in the thread order of the fused sweep
  __nv_bfloat162* dhatp16 = nullptr;  // its bf16 copy (mixed precision)
  __nv_bfloat162* dhat16 = nullptr;   // mixed precision copy of dhat
  float2* xhat = nullptr;
  float* pdiag = nullptr;
  float2* pmat = nullptr;
  float2* part[2] = {nullptr, nullptr};
  double* l1 = nullptr;
  double* objimg = nullptr;
  int* err = nullptr;        // learning: CSC_ERR_TIMEOUT / CSC_ERR_NONFINITE raised by the kernels
  int* cerr = nullptr;       // coding: CSC_ERR_NONFINITE raised by the sweeps of the latest csc_code
  long long wait_limit = 0;  // bound of the CG exchange waits in SM clocks (0: the default, ~1 s)
  LearnBuffers L;
  BackwardBuffers B;
  VideoLearnBuffers VL;
  bool uneven = false;
  UnevenLayout U;
  // video tensors (csc_init_video)
  bool video = false;
  int T = 1, ft = 1;
  float2* vS = nullptr;     // [N][K][T][8320]
  float2* vd2 = nullptr;    // [K][J][ft][8320]
  float2* vx3 = nullptr;    // [N][J][T][8320]
  float2* vp3 = nullptr;    // [T][8320][J][J]
  float2* vtmp = nullptr;   // canonical 2-D spectra scratch [max(K J ft, N J T)][Omega]
  double* vobj = nullptr;   // [N][bin blocks]
  double* vl1 = nullptr;    // [frame CTAs]
  // direct spatial coding (CSC_FLAG_SPATIAL, spatial.cu)
  bool spatial = false;
  uint8_t* sp_bt = nullptr;   // filter operand of D^T, TF32 hi | lo
  uint8_t* sp_bc = nullptr;   // filter operand of D, TF32 hi | lo
  float* sp_r = nullptr;      // [N][128][128] sum_k d_k * u_k
  float* sp_lam = nullptr;    // [N][128][128] dual variable
  // CUDA graph of the last csc_code launch sequence (flag CSC_FLAG_GRAPH)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  const void* graph_key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int graph_iters = -1;
  // staging of host arrays
  float* st_x = nullptr;
  float* st_d = nullptr;
  float* st_v = nullptr;
  float* st_z = nullptr;
  double* st_mu = nullptr;
  std::string last_error;
  // benchmarking aid: event pairs around sweeps (kind 0) and learning calls (kind 1)
  bool timing = false;
  struct EventPair { cudaEvent_t a, b; int kind; };
  std::vector<EventPair> events;
  size_t events_used = 0;
  mutable long long launches = 0;
};

// per-geometry launchers of the per-map kernels (geo_*.cu)
enum BwdMode { kBSeed = 0, kBIter = 1, kBLast = 2 };

// arguments of the reverse-mode sweep (geo_kernels.cuh, k_bwd_sweep)
struct BwdArgs {
  int N, K, G;
  float beta, rho, dsize;
  const float2* dhat;      // [K][Omega]
  const float* pdiag;      // [Omega] P / D
  const float2* part_in;   // [(G+N)][Omega]
  float2* part_out;
  float* vbar;             // [N][K][D] in/out
  const float* vt;         // [N][K][D] forward state v^t (seed: v^T)
  const float* gz;         // [N][K][D] dL/dz_T (seed)
  const float2* lam_t;     // [N][Omega] lam_s^t (iterate, last)
  const float2* lam_prev;  // [N][Omega] lam_s^{t-1} (seed, iterate)
  float2* gspec;           // [N][K][Omega]
  float* S;                // [N][Omega]
  float2* Xb;              // [N][Omega]
  const float2* tw;
};

struct GeoOps {
  cudaError_t (*fft_maps)(const Ctx&, const float* in, int nmaps, int filter_mode, float2* out);
  cudaError_t (*sweep)(const Ctx&, int mode, const SweepArgs&);
  cudaError_t (*rhs)(const Ctx&, const float2* spec);
  cudaError_t (*lags)(const Ctx&);
  cudaError_t (*bwd)(const Ctx&, int mode, const BwdArgs&);
  cudaError_t (*spec_maps)(const Ctx&, const float2* spec, int nmaps, float scale, float* out);
  cudaError_t (*dgrad)(const Ctx&, const float2* gspec, const float* S, float* gd);
  cudaError_t (*rhs_ex)(const Ctx&, const float2* zhat, const float2* xhat, float* out);
  cudaError_t (*expand)(const Ctx&, const float2* spec, float scale, float* out);
};
const GeoOps& geo_ops_128();
const GeoOps& geo_ops_100();
const GeoOps& geo_ops_64();
const GeoOps& geo_ops_rt();
inline const GeoOps& geo_ops(const Ctx& c);

// launchers (coding.cu)
cudaError_t launch_fft_maps(const Ctx& c, const float* in, int nmaps, int filter_mode, float2* out);
// the fused 128 x 128 sweep (sweep128.cu)
bool fused128_applies(const Ctx& c, const SweepArgs& a);
cudaError_t launch_sweep_fused128(const Ctx& c, int mode, const SweepArgs& a);
cudaError_t launch_permute_dhat128(const Ctx& c);
cudaError_t upload_f128_twiddles();   // the fused sweep's constant twiddle tables, current device
cudaError_t launch_solve_prep(const Ctx& c);
cudaError_t launch_sweep(const Ctx& c, int mode, const float2* part_in, float2* part_out, float* v,
                         float* z);
cudaError_t launch_codes_from_state(const Ctx& c, const float* v, float* z);
// out [N J][2 H0][2 W0] = half-sample symmetric extension of in [N J][H0][W0] (symmetric boundary)
cudaError_t launch_symmetric_extend(const Ctx& c, const float* in, float* out);
cudaError_t launch_codes_from_state_n(const Ctx& c, const float* v, float* z, size_t n);
cudaError_t launch_objective_final(const Ctx& c, const float2* part, double* out_img);
cudaError_t launch_sweep_ex(const Ctx& c, int mode, const float2* part_in, float2* part_out, float* v,
                            float* z, float* v_out, float2* lam_store);
cudaError_t launch_sum_slots(const Ctx& c, const float2* part, float2* out);
size_t sweep_smem_bytes(const Geometry& g, int J, int mode);
inline size_t bwd_smem_bytes(const Geometry& g, bool rb, bool acc) {
  return ((size_t)g.H * g.P + (rb ? (size_t)g.Omega : 0) + (acc ? (size_t)g.Omega : 0) +
          (size_t)(g.Wh + g.H + g.Wc)) * sizeof(float2);
}

// direct spatial coding of 128 x 128 grey images on the tensor cores (spatial.cu): whether the
// context qualifies (else *why says what is missing), the bytes of each filter operand, the operand
// build from d, and the three launches of one iteration (D, the per-frequency solve of lambda, D^T with
// the state update; z written by the last iteration's D^T when non-null)
bool spatial_applies(const Ctx& c, std::string* why);
size_t spatial_operand_bytes(const Ctx& c);
cudaError_t launch_spatial_operands(const Ctx& c, const float* d);
cudaError_t launch_spatial_conv(const Ctx& c, const float* v);
cudaError_t launch_spatial_lambda(const Ctx& c, const float* x);
cudaError_t launch_spatial_corr(const Ctx& c, float* v, float* z, bool last);

// message returned by csc_last_error(NULL) (api.cu)
void set_global_error(const char* msg);

// launchers (learning.cu)
cudaError_t launch_learn_rhs(const Ctx& c, const float2* spec);
cudaError_t launch_learn_gram(const Ctx& c);
// learning on a video context (video_learn.cu): x, z, d device arrays; mu host or device; the
// steps' CG iteration counts in c->VL.iters
csc_status video_learn(Ctx* c, const float* x, const float* z, float* d, double* mu, int steps);
bool video_learn_shape_ok(const Ctx& c);
// the persistent cooperative CG of the video learning (video_cg.cu): whether the context's shape fits
// it, the exchange words it needs, and the launch (all learning steps, mu on the device)
bool video_cg_applies(const Ctx& c);
size_t video_cg_words(const Ctx& c);
cudaError_t launch_video_cg(const Ctx& c, unsigned long long* words, const float* lags, const float2* chat,
                            const float* b, float* x, double* mu, const int* active, int* iters, int steps);
cudaError_t launch_learn_lags(const Ctx& c);       // from gram [npairs][Omega] (CUDA-core Gram)
cudaError_t launch_learn_lags_sep(const Ctx& c);   // from the tensor-core Gram's gramT [Omega][npairs]
cudaError_t launch_lag_spectra(const Ctx& c);      // L.chat from L.lags (both lag launchers end with it)
size_t lag_sep_T_count(const Ctx& c);
cudaError_t launch_learn_cg(const Ctx& c, float* d, int steps, int* dev_err);
bool learn_cg_shape_ok(const Ctx& c);   // filters per CTA <= 8 and 2 J NF <= 6 NT
size_t learn_cg_smem_bytes(const Ctx& c, bool chat_smem);
// spectra of nmaps real maps (codes), out[m][Omega]: the fused-sweep passes for 128 x 128 maps,
// else the generic FFT
cudaError_t launch_code_spectra(const Ctx& c, const float* in, int nmaps, float2* out);
cudaError_t launch_spectra_f128(const Ctx& c, const float* in, long long nmaps, float2* out);
// out[o][m] = in[m][o] for nmaps spectra (frequency-major copy for the tensor-core Gram)
cudaError_t launch_spectra_transpose(const Ctx& c, const float2* in, int nmaps, float2* out);
// tensor-core Gram (K + J <= 128), reading the frequency-major code spectra L.zt; also writes the
// right-hand-side spectra [K][J][Omega]. prec: CSC_FP32 (3xTF32, float32-accurate), CSC_MIXED_BF16
// (BF16 operands) or CSC_MIXED_TF32 (one TF32 product)
cudaError_t launch_learn_gram_tc(const Ctx& c, int prec, float2* rspec, int* dev_err);
bool gram_tc_applies(const Ctx& c);
cudaError_t launch_to_bf16(const Ctx& c, const float2* in, __nv_bfloat162* out, size_t n);

inline const GeoOps& geo_ops(const Ctx& c) {
  switch (c.g.ct_id) {
    case 1: return geo_ops_128();
    case 2: return geo_ops_100();
    case 3: return geo_ops_64();
    default: return geo_ops_rt();
  }
}

}  // namespace csc
