/*
 * csc.h - C ABI of the GB300 dual-domain convolutional sparse coding library (libcsc.so).
 *
 * Method: Affara, Ghanem & Wonka, "Fast Convolutional Sparse Coding in the Dual Domain"
 * (arXiv 1709.09479). The problem (Eq. 1, summed over N images that share the dictionary):
 *
 *     min_{d,z}  1/2 sum_n || x_n - sum_k d_k * z_nk ||^2 + beta sum_{n,k} || z_nk ||_1
 *     s.t.       || d_k ||_2^2 <= 1,
 *
 * with circular convolution on the image grid (Sec. 3). Higher-order CSC (Sec. 3.3): J channels per
 * image share one code per filter; filter k has J channels.
 *
 * Layouts (all float32, C order, no padding):
 *   x  images       [N][J][H][W]
 *   d  filters      [K][J][fh][fw]  tap (a,b) sits at offset (a - (fh-1)/2, b - (fw-1)/2), wrapped
 *   v  ADMM state   [N][K][H][W]    v = D^T lambda - z / rho; v = 0 means z = theta = 0
 *   z  codes        [N][K][H][W]    z = rho (clamp(v, -beta, beta) - v)
 *   mu multipliers  [K] float64     (Eq. Learning_Lagrangian)
 *
 * Pointers: every array argument may be host memory or device memory of the context's device;
 * the library detects which (cudaPointerGetAttributes). Host arrays are staged through
 * library-owned device buffers inside the call, and such calls return only after their host
 * outputs are written. Calls whose arrays are all on the device are asynchronous on the
 * context's stream, except csc_learn and csc_objective, which synchronise to return host values.
 * The caller owns every array it passes; the library owns its workspace (allocated by csc_init
 * and on first use of csc_learn, released by csc_destroy).
 *
 * Errors: every call returns a csc_status. Shape and argument errors are detected before any
 * launch. A failed call leaves its output arrays unspecified but the context usable;
 * csc_last_error gives a one-line description. No exception or exit() crosses the ABI.
 */
#ifndef CSC_H_
#define CSC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct csc_ctx csc_ctx;

typedef enum {
  CSC_OK = 0,
  CSC_ERR_ARG = 1,           /* null or inconsistent argument */
  CSC_ERR_SHAPE = 2,         /* size outside what the kernels support */
  CSC_ERR_WORKSPACE = 3,     /* device allocation failed */
  CSC_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed */
  CSC_ERR_NONFINITE = 5,     /* a non-finite value appeared (device flag, see CSC_FLAG_CHECK_FINITE) */
  CSC_ERR_NOT_CONVERGED = 6, /* csc_learn with CSC_FLAG_CG_STRICT: a CG solve stopped at cg_max */
  CSC_ERR_TIMEOUT = 7,       /* a bounded grid barrier gave up; results unspecified */
  CSC_ERR_UNSUPPORTED = 8    /* valid request the library does not implement */
} csc_status;

typedef enum {
  CSC_FP32 = 0,        /* everything in float32 */
  CSC_MIXED_BF16 = 1,  /* FFTs, shrinkage and CG in float32; the per-frequency contractions with
                          bfloat16 operands and float32 accumulation: sum_k d_hat_k u_hat_k and
                          conj(d_hat_k) lambda_hat in the coding sweep (CUDA cores), and the code Gram
                          Z(w)^H Z(w) of csc_learn on the tensor cores (tcgen05 kind::f16). In
                          CSC_FP32 the Gram also runs on the tensor cores when K <= 128, as three
                          TF32 products of a hi + lo operand split (float32-accurate). The
                          per-frequency system (A(w) + I/rho)^{-1} is built in float64 in both modes.
                          csc_init needs K <= 128 in this mode. Uniform and uneven batches accept
                          it; video contexts,
                          csc_code_unrolled, csc_code_backward and the synthesis calls accept
                          CSC_FP32 only. */
  CSC_MIXED_TF32 = 2   /* as CSC_MIXED_BF16 with TF32 operands (10 explicit mantissa bits, rounded to
                          nearest, ties away from zero): both operands of sum_k d_hat_k u_hat_k and of
                          conj(d_hat_k) lambda_hat rounded to TF32 in the coding sweeps, float32
                          accumulation; the code Gram as one TF32 tensor-core product (kind::tf32)
                          instead of CSC_FP32's three. Uniform batches only (csc_init). */
} csc_precision;

typedef struct {
  int J;          /* channels per image sharing one code (1 grey, 3 colour), 1..3 */
  int K;          /* number of filters, >= 1 */
  int fs[2];      /* filter support (fh, fw), odd, each <= the image side */
  double beta;    /* l1 weight of Eq. 1, > 0 */
  double rho;     /* ADMM step of Eq. Inference_solution, > 0 */
  int cg_max;     /* CG iteration cap per learning step (csc_learn), >= 1 */
  double cg_tol;  /* CG stop: ||r|| <= cg_tol ||b|| (relative residual), > 0 */
  int precision;  /* csc_precision */
  int flags;      /* CSC_FLAG_* bits */
  int deterministic; /* 1: every reduction runs in a fixed order, so a call repeated on the same inputs
                        gives the same bits (partial sums per CTA slot added in slot order, float64 CG
                        dot products, no atomics on data). This build has no other mode: 0 is accepted
                        and gives the same bits. */
} csc_params;

/* csc_code records its launch sequence in a CUDA graph the first time it is called with a given
   (x, d, v, z, iters) on device memory, and replays the graph on later calls with the same
   arguments (the arrays' contents may change between calls; their addresses may not). */
#define CSC_FLAG_GRAPH 1
/* csc_code synchronises the stream at its end and returns CSC_ERR_NONFINITE when a sweep met a
   non-finite dual variable lambda_hat (any NaN or Inf in x, d or v reaches it within one
   iteration). Calls with host arrays always check; without the flag a device-array call stays
   asynchronous and csc_check reports the flag later. Uniform 2-D batches only (uneven and video
   contexts do not raise it). */
#define CSC_FLAG_CHECK_FINITE 2
/* csc_learn returns CSC_ERR_NOT_CONVERGED (after writing d, mu and cg_iters) when a step's CG stopped
   at params->cg_max iterations; without the flag that case returns CSC_OK and shows in cg_iters. */
#define CSC_FLAG_CG_STRICT 4
/* csc_init only: reflected image boundaries instead of circular ones - the DCT variant the paper
   mentions at the start of Sec. 3. dims = {H, W} is the size of the caller's images x [N][J][H][W];
   the context codes their half-sample symmetric extension (2H x 2W: rows H..2H-1 repeat rows
   H-1..0, columns likewise), whose circular convolution is convolution with reflected boundaries
   on the image, so v and z are [N][K][2H][2W] and csc_objective is the objective of the extended
   problem. For filters symmetric about their centre this is exactly the dual ADMM in the type-II DCT
   domain of the H x W images, and the extended codes are mirror symmetric (their [0, H) x [0, W)
   block holds all of them). 2H x 2W must satisfy csc_init's size conditions. csc_code, csc_learn,
   csc_learn_stats and csc_objective take x at H x W; the reverse-mode calls return
   CSC_ERR_UNSUPPORTED. */
#define CSC_FLAG_SYMMETRIC_BOUNDARY 8
/* csc_init: csc_code applies D and D^T as direct spatial convolutions on the tensor cores
   (tcgen05, float32 operands split into two TF32 parts, three products per pair: float32-accurate;
   one TF32 product under CSC_MIXED_TF32) instead of per-frequency products of K map spectra. The
   Fourier domain is kept only for the per-frequency solve lambda = (D D^T + I/rho)^{-1} r of one
   channel per image (Eq. Inference_solution; the complexity table of Sec. 4.2 counts the Fourier
   route's transforms, about log(H W) operations per pixel and filter, where the spatial products take
   fh fw multiply-adds on the tensor pipe). One iteration is three launches:
   r = D u with u = 2 clamp(v) - v, lambda from r - x/rho by two 2-D FFTs, and D^T lambda with the state
   update. Same state v and codes z as the Fourier route, equal up to rounding. Needs H = W = 128,
   J = 1, K <= 128, fh fw <= 128, fh <= 15, precision CSC_FP32 or CSC_MIXED_TF32, no symmetric
   boundary (CSC_ERR_UNSUPPORTED otherwise); csc_code needs v 16-byte aligned (CSC_ERR_ARG otherwise:
   its rows are moved by TMA tensor copies). On a GB300 at 100 images of 128 x 128 and 100 filters of
   11 x 11 an iteration takes about 1.25 times the Fourier route's (1.04 times with CSC_MIXED_TF32):
   it is a second route to the same iterates, not the faster one there. Only csc_code's iterations
   change; the other calls run as
   on any context. Every wait of the tensor-core kernels is bounded by csc_set_wait_limit's bound (or
   about one second); a wait that gives up makes a synchronising csc_code return CSC_ERR_TIMEOUT.
   csc_init_uneven: every image of the batch is coded with D and D^T as direct spatial correlations on
   the CUDA cores (float32; output tiles of 32 x 64 pixels, the filters zero-padded to 11 x 11 about
   their centre, circular boundaries on each image's own H x W grid) and lambda by one 2-D transform
   pair per image and iteration (the multi-pass transforms, Bluestein for sides with a prime factor
   above 7). One iteration is five launches: D^T with the state update, D (q = D u - x/rho), and three
   passes for lambda = F^-1(P F(q)). Needs J = 1, CSC_FP32, fh, fw <= 11, 496 K + 26 168 bytes of
   shared memory <= 232448 (K <= 415), no symmetric boundary (CSC_ERR_UNSUPPORTED otherwise); any
   alignment of v. On a GB300, 256 images with sides uniform in [64, 512] and 64 filters of 11 x 11
   take about 16 ms per iteration against 84 ms on the Fourier route. The objective on such a context
   is the Fourier engine's (its workspace is kept). */
#define CSC_FLAG_SPATIAL 16

/*
 * Create a context for n_images images, all of size H x W (dims = {H, W}), on the current CUDA
 * device, launching on `stream` (a cudaStream_t; NULL = legacy default stream). The context holds
 * one instance of the problem of Eq. 1 (N images sharing K filters; J channels per image sharing
 * one code per filter, the higher-order form of Sec. 3.3) with the parameters beta and rho of
 * Eq. 1 and Eq. Inference_solution.
 * Supported sizes: W even; H, W >= 8; H and W/2 factoring into 2, 3, 5 and 7; one map plus 2*J
 * half spectra in a CTA's shared memory: 8 * (H*P + 2*J*H*(W/2+1) + W + H + 1) <= 232448 bytes,
 * P = W/2+1 rounded up to odd (128 x 128 fits at J = 1). Filter width fw <= 15.
 * On success *out owns the workspace; release it with csc_destroy.
 */
csc_status csc_init(const csc_params* params, int n_images, const int* dims, void* stream,
                    csc_ctx** out);

/*
 * Like csc_init for a batch whose images have their own sizes: dims holds n_images (H, W) pairs.
 * Arrays are the per-image arrays of csc_init concatenated in image order: x holds
 * J*H_n*W_n floats for image n, v and z hold K*H_n*W_n. Any 8 <= H, W <= 1024 with the filter
 * inside the image (fh <= H, fw <= W) is accepted; other sizes give CSC_ERR_SHAPE. Images of one
 * size share one FFT plan, filter spectrum and per-frequency system. Images that satisfy
 * csc_init's conditions are coded by one launch per ADMM iteration over all of them, with the maps
 * split over the CTAs by pixel count; on the first coding call that launch's shape (threads per
 * CTA, CTAs per SM) is chosen by timing the candidates on this batch. Every other image (odd W,
 * sides with a prime factor above 7, spectra beyond one CTA's shared memory) is coded by four
 * launches per iteration that stage each 2-D transform through device memory (Bluestein's chirp
 * z-transform for lengths with a prime factor above 7), with a workspace of K*H_n*(W_n/2+1)
 * complex values per image. Supports csc_code and csc_objective (csc_learn and the reverse-mode
 * calls return CSC_ERR_UNSUPPORTED on such a context). With CSC_FLAG_SPATIAL every image takes the
 * direct spatial route described at that flag.
 */
csc_status csc_init_uneven(const csc_params* params, int n_images, const int* dims, void* stream,
                           csc_ctx** out);

/*
 * Like csc_init for videos: n_videos tensors of J channels x T frames x H x W (dims = {T, H, W}),
 * coded with K filters of support ft x fh x fw per channel (params->fs = {fh, fw}; ft odd, taps at
 * time offsets -(ft-1)/2 .. (ft-1)/2, circular like the spatial ones), 3-D DFTs: the higher-order
 * extension of Sec. 3.3 with a time axis. Arrays: x [N][J][T][H][W], d [K][J][ft][fh][fw],
 * v and z [N][K][T][H][W]. Supported: H = W = 128, 1 <= T <= 64, ft <= 7 and <= T, CSC_FP32; the
 * flags of csc_params but CSC_FLAG_SYMMETRIC_BOUNDARY (CSC_ERR_UNSUPPORTED).
 * Supports csc_code, csc_objective, csc_learn (fh <= 12, fw <= 16, K + J <= 128; the 3-D lag window
 * (2ft-1) x (2fh-1) x (2fw-1), Jacobi-preconditioned CG, params->cg_max, cg_tol and
 * CSC_FLAG_CG_STRICT as for csc_init; all learning steps in one persistent launch whose exchange
 * waits follow csc_set_wait_limit, where the shape fits the shared memory of an SM, else a
 * host-driven CG), csc_describe and csc_destroy; the reverse-mode calls return CSC_ERR_UNSUPPORTED
 * on such a context.
 */
csc_status csc_init_video(const csc_params* params, int ft, int n_videos, const int* dims, void* stream,
                          csc_ctx** out);

/* One-line JSON description of the context (sizes, size classes, launch shape) into buf (len bytes). */
csc_status csc_describe(const csc_ctx* ctx, char* buf, int len);

/*
 * Coding subproblem (Eq. 2) by `iters` iterations of the dual ADMM of Eq. Inference_solution
 * (Sec. 3.2), in the Fourier domain, with the filters d fixed:
 *     lambda = (D D^T + I/rho)^{-1} (D theta + D z / rho - x / rho)
 *     theta  = Pi_C(D^T lambda - z / rho)
 *     z      = z + rho (theta - D^T lambda)
 * carried in the single state v (in/out, [N][K][H][W]); pass v = 0 for the start of Algorithm 1
 * and the previous v to warm-start. If z is non-NULL it receives the codes of the final state.
 * iters >= 0 (0 only computes z from v).
 */
csc_status csc_code(csc_ctx* ctx, const float* x, const float* d, float* v, float* z, int iters);

/*
 * Learning subproblem (Eq. 3, Sec. 3.2) for fixed codes z: `steps` rounds of
 *     d(mu) = argmin_d 1/2 ||x - Z S^T d||^2 + sum_k mu_k ||d_k||^2   (Eqs. Learning_new..Solution)
 *     mu_k <- max(mu_k ||d_k||_2, 1e-8)                                (Eq. mu_update)
 * then d_k <- d_k / max(1, ||d_k||). d(mu) is the solution of the dual system of
 * Eq. Learning_gamma; the library reaches the same d by solving the filter-space normal equations
 * (S Z^T Z S^T + 2 diag(mu)) d = S Z^T x (strong duality) with CG warm-started from the current d.
 * A filter whose codes are all zero keeps its d_k and mu_k. Channels are solved separately with
 * one shared mu (Sec. 3.3). d is in/out [K][J][fh][fw] ([K][J][ft][fh][fw] on a video context);
 * mu is in/out [K] (float64).
 * If cg_iters is non-NULL it receives `steps` ints (host memory): the CG iterations of each step
 * (the maximum over channels). Synchronises the stream.
 */
csc_status csc_learn(csc_ctx* ctx, const float* x, const float* z, float* d, double* mu, int steps,
                     int* cg_iters);

/*
 * The learning subproblem split at its one reduction over images, for data-parallel learning over
 * several contexts (one per GPU, each holding its own images; Sec. 3.2: the dictionary d is shared,
 * the images only enter through sums over n). csc_learn is csc_learn_stats followed by
 * csc_learn_solve on the same context.
 *
 * csc_learn_stats writes this context's two sums for codes z:
 *   C [K][K][2fh-1][2fw-1]  the code cross-correlations on the lag window:
 *                           C[k][k'][ta + fh-1][tb + fw-1] = sum_n sum_p z_nk(p) z_nk'(p + (ta, tb))
 *                           (circular in p), i.e. the matrix S Z^T Z S^T of Eq. Learning_new in
 *                           block-Toeplitz form;
 *   b [K][J][fh][fw]        the right-hand side S Z^T x = sum_n S (z_nk correlated with x_nj).
 * Both are sums over images: the sums of several contexts' C and b (an all-reduce) are the C and b of
 * their images together. csc_learn_solve then runs `steps` learning steps (the CG of csc_learn
 * warm-started from d, the mu update, the final projection) from a given C and b: every context
 * given the same reduced C, b, d and mu computes the same d and mu. Arrays may be host or device
 * memory (float32; mu float64); csc_learn_stats synchronises and returns after C and b are written.
 * Uniform 2-D contexts only (CSC_ERR_UNSUPPORTED on uneven and video contexts).
 */
csc_status csc_learn_stats(csc_ctx* ctx, const float* x, const float* z, float* C, float* b);
csc_status csc_learn_solve(csc_ctx* ctx, const float* C, const float* b, float* d, double* mu, int steps,
                           int* cg_iters);

/*
 * Objective of Eq. 1 summed over images: *out (host) = 1/2 sum_n ||x_n - sum_k d_k * z_nk||^2
 * + beta sum |z|. Reductions run in float64 in a fixed order. Synchronises the stream.
 */
csc_status csc_objective(csc_ctx* ctx, const float* x, const float* d, const float* z, double* out);

/*
 * Reverse mode through unrolled coding iterations (not in the paper; J = 1 in this build).
 * csc_code_unrolled runs `iters` iterations of csc_code from the state v (in: v^0, out: v^T) and
 * writes z = z_T (nullable) like csc_code, and records on `tape` (device memory of
 * csc_tape_bytes(ctx, iters, every) bytes, owned by the caller): the state every `every`
 * iterations (checkpoints), v^T, and lambda of every iteration.
 * csc_code_backward then returns the vector-Jacobian products of z_T with respect to the images x
 * and the filters d for the cotangent gz = dL/dz_T ([N][K][H][W]): gx [N][J][H][W], gd [K][J][fh][fw].
 * It recomputes each segment's states from its checkpoint and runs the reverse recurrence
 *   lambar = D vbar', rbar = P lambar, ubar = D^T rbar, xbar -= rbar / rho,
 *   vbar = (1 - m) vbar' + (2m - 1) ubar,   m = 1[|v| < beta],
 *   dbar_k += G(vbar'_k, lambda) + G(u_k, rbar) - G(w_k, rbar) - G(ubar_k, lambda),
 * with G(a, b)(q) = sum_p b(p) a(p - q) on the filter support and the seed vbar^T = rho (m_T - 1) gz.
 * All arrays must be device memory. Asynchronous on the context's stream. csc_tape_bytes returns 0
 * for invalid arguments and for uneven-batch and video contexts (no reverse mode there).
 */
size_t csc_tape_bytes(const csc_ctx* ctx, int iters, int every);
csc_status csc_code_unrolled(csc_ctx* ctx, const float* x, const float* d, float* v, float* z, int iters,
                             int every, void* tape);
csc_status csc_code_backward(csc_ctx* ctx, const float* x, const float* d, const void* tape, int iters,
                             int every, const float* gz, float* gx, float* gd);

/*
 * Reconstruction (Eq. 1's model): out [N][J][H][W] = sum_k d_k * z_k. csc_synthesize_backward gives,
 * for the cotangent gout of out, gz = D^T gout and gd_k = S sum_n z_nk ⋆ gout_n (J = 1 in this
 * build). Device arrays only; asynchronous on the context's stream.
 */
csc_status csc_synthesize(csc_ctx* ctx, const float* d, const float* z, float* out);
csc_status csc_synthesize_backward(csc_ctx* ctx, const float* d, const float* z, const float* gout, float* gz,
                                   float* gd);

/*
 * Benchmarking aid (no counterpart in the paper). While enabled, each coding sweep launch (one ADMM
 * iteration over all N*K maps) and each csc_learn call are bracketed by CUDA events on the
 * context's stream. kernel_launches counts every kernel the library launched (enabled or not).
 */
typedef struct {
  double sweep_ms;           /* summed device time of the bracketed coding sweeps */
  int sweep_launches;        /* number of bracketed coding sweeps */
  double learn_ms;           /* summed device time of the bracketed csc_learn calls */
  int learn_calls;
  long long kernel_launches; /* kernels launched since the last csc_timing_read */
} csc_timing;

/* Turn event bracketing on (enable != 0) or off. */
csc_status csc_timing_enable(csc_ctx* ctx, int enable);

/* Read and reset the accumulated timing (synchronises the stream). */
csc_status csc_timing_read(csc_ctx* ctx, csc_timing* out);

/*
 * csc_code without a context and without allocating. The paper has no counterpart: this exists for
 * callers that cannot allocate device memory where they code images - code inside a framework whose
 * caching allocator owns the whole device pool, plugins that are handed only a stream and device
 * pointers, and latency-bound paths that cannot take the implicit synchronisation of cudaMalloc.
 * Same computation, arguments and layouts as csc_init(params, n_images, dims, stream) followed by
 * csc_code(x, d, v, z, iters), except that x, d, v and z must be device pointers, only CSC_FP32 is
 * accepted, and every geometry (128 x 128 included) runs the generic fused sweep, about 2.8x slower
 * than the 128 x 128 sweep csc_code takes (that one needs a second, thread-ordered copy of the filter
 * spectra). The workspace is a fixed 64 MiB file-scope __device__ array that every GPU loading the
 * library holds until the process exits; problems needing more return CSC_ERR_SHAPE with the byte
 * count in csc_last_error(NULL) (e.g. N = 100, K = 100, 128 x 128 needs about 47 MB and fits).
 * No cudaMalloc, cudaFree or other allocating call is made, and nothing is copied from host memory
 * (the twiddle table is written by a kernel). The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and caches it; make that first call before any stream
 * capture. Every call on a device shares that device's one array and leaves its contents behind
 * (each call rewrites everything it reads), so calls that may overlap on the same device race:
 * serialise them on one stream per device. Asynchronous on `stream`. Errors are reported through
 * the return value and csc_last_error(NULL).
 */
csc_status csc_code_noalloc(const csc_params* params, int n_images, const int* dims, void* stream,
                            const float* x, const float* d, float* v, float* z, int iters);

/*
 * Synchronise the context's stream and report the device flag of the most recent csc_code call:
 * CSC_ERR_NONFINITE if one of its sweeps met a non-finite lambda_hat, else CSC_OK (each csc_code
 * clears the flag when it starts). For asynchronous callers that did not set CSC_FLAG_CHECK_FINITE.
 */
csc_status csc_check(csc_ctx* ctx);

/*
 * Testing aid (no counterpart in the paper): bound every spin-wait of the learning CG's grid
 * exchanges to `clocks` SM clock cycles (0 restores the default of about one second). A wait that
 * runs out sets the context's error word; every CTA then returns and csc_learn returns
 * CSC_ERR_TIMEOUT with d and mu unspecified, leaving the context usable. A tiny bound makes a wait run
 * out on purpose; the tensor-core Gram's waits are not affected.
 */
csc_status csc_set_wait_limit(csc_ctx* ctx, long long clocks);

/* Release the context and its workspace. NULL is ignored. */
void csc_destroy(csc_ctx* ctx);

/* One-line description of the last error on ctx (or of the last csc_init failure if ctx is NULL). */
const char* csc_last_error(const csc_ctx* ctx);

/* Library version string. */
const char* csc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CSC_H_ */
