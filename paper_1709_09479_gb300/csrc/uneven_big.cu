// Coding of the images of an uneven batch whose maps do not fit the one-map-per-CTA sweep: sides up
// to kBigMaxSide (1024), odd widths, and lengths with prime factors above 7 (the dual ADMM of
// Eq. Inference_solution, the same arithmetic as uneven.cu).
//
// The map spectra live in HBM ([map][H][W/2+1], the half-spectrum layout of d_hat and x_hat) and each
// 2-D transform is two batched passes of 1-D transforms through shared memory:
//   columns (length H, complex) on the W/2+1 stored columns, and
//   rows (length W; two real rows as the real and imaginary parts of one complex transform, the
//   first W/2+1 bins of each kept; the inverse first completes each row by Hermitian symmetry,
//   X[W-k] = conj X[k]).
// A 1-D transform of a 7-smooth length is the run-time Stockham plan of fft.cuh; any other length n
// goes through Bluestein's chirp z-transform: with w_j = e^{-pi i j^2/n},
//     X_k = w_k sum_j (x_j w_j) conj(w_{k-j}),
// a circular convolution of length M >= 2n - 1 (M a power of two) done with two length-M transforms; the
// inverse transform is conj(DFT(conj x)).
// One ADMM iteration over all such images is four launches: the inverse column pass (building
// w_hat_k = sum_j conj(d_hat_jk) lambda_hat_j as it loads), the row pass (inverse row transform, the
// state update v <- w - (clamp(v) - v), u = 2 clamp(v) - v, forward row transform), the forward
// column pass, and the per-frequency pass that forms r_hat = sum_k d_hat_k u_hat_k - x_hat / rho and
// lambda_hat = P r_hat (P includes 1/D, so the transforms stay unnormalised). Work items are listed
// on the host; every sum is formed in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "csc_internal.cuh"

namespace csc {
namespace big {

constexpr int NT = 256;
constexpr int kMinCtas = 3;   // resident CTAs per SM the transform kernels are compiled for

// x / d for x * d < 2^32 from m = floor((2^32 - 1) / d) + 1 (d >= 2), by one high multiply
struct FastDiv {
  unsigned d, m;
  __device__ __forceinline__ explicit FastDiv(unsigned dd) : d(dd), m(dd > 1 ? 0xFFFFFFFFu / dd + 1u : 0u) {}
  __device__ __forceinline__ unsigned div(unsigned x) const { return d > 1 ? __umulhi(x, m) : x; }
};

__device__ __forceinline__ float bclamp(float v, float b) { return fminf(fmaxf(v, -b), b); }
// a complex value rounded to bfloat16 and back (operands of the mixed-precision contractions)
__device__ __forceinline__ float2 bbf16(float2 v) { return __bfloat1622float2(__floats2bfloat162_rn(v.x, v.y)); }

// A transform of nlines lines of length pl.n at buf + line * ls (ls >= pl.M) is: each element j < n
// stored through fin (Bluestein: the chirp w_j, after conjugation for the inverse), the padding [n, M)
// zeroed by fpad, a synchronisation, fcore, and each result element read through fout (Bluestein: the
// chirp again, and the conjugation for the inverse). Without Bluestein, fin and fout are the identity.
template <bool INV>
__device__ __forceinline__ float2 fin(float2 v, int j, const BigPlan& pl, const float2* tabs) {
  if (pl.M == 0) return v;
  if (INV) v.y = -v.y;
  return cmul(v, __ldg(tabs + pl.chirp + j));
}
template <bool INV>
__device__ __forceinline__ float2 fout(float2 v, int j, const BigPlan& pl, const float2* tabs) {
  if (pl.M == 0) return v;
  v = cmul(v, __ldg(tabs + pl.chirp + j));
  if (INV) v.y = -v.y;
  return v;
}
__device__ __forceinline__ void fpad(float2* buf, int nlines, int ls, const BigPlan& pl) {
  if (pl.M == 0) return;
  const int pad = pl.M - pl.n;
  for (int line = 0; line < nlines; ++line)
    for (int j = threadIdx.x; j < pad; j += NT) buf[(size_t)line * ls + pl.n + j] = make_float2(0.f, 0.f);
}
// One Stockham stage of radix R over nlines lines (line L element e at buf[L * ls + e]) in place:
// the butterflies of whole lines per round, read into registers before any is written. The same
// butterflies as the run-time stages of fft.cuh, with the index divisions by the round's line count
// and by Ns done as high multiplies.
template <int R, bool INV, int IPT>
__device__ __forceinline__ void big_stage_body(float2* buf, int nlines, int ls, int n, int Ns, const float2* tw) {
  const int nb = n / R;
  int lpr = (NT * IPT) / nb;
  lpr = lpr < 1 ? 1 : (lpr > nlines ? nlines : lpr);
  const int tsu = n / (Ns * R);
  const FastDiv dns((unsigned)Ns);
  for (int L0 = 0; L0 < nlines; L0 += lpr) {
    const int nl = min(lpr, nlines - L0);
    const FastDiv dnl((unsigned)nl);
    const int items = nl * nb;
    float2 v[IPT][R];
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      const int i = threadIdx.x + it * NT;
      if (i < items) {
        const int j = (int)dnl.div((unsigned)i);
        const int line = L0 + i - j * nl;
        const int k = j - (int)dns.div((unsigned)j) * Ns;
        const float2* src = buf + line * ls + j;
        const int ts = k * tsu;
        v[it][0] = src[0];
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const float2 x = src[r * nb];
          v[it][r] = ts ? cmul(x, tw_dir<INV>(tw[r * ts])) : x;
        }
        dft<R, INV>(v[it], tw, n);
      }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      const int i = threadIdx.x + it * NT;
      if (i < items) {
        const int j = (int)dnl.div((unsigned)i);
        const int line = L0 + i - j * nl;
        const int k = j - (int)dns.div((unsigned)j) * Ns;
        float2* dst = buf + line * ls + (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[r * Ns] = v[it][out_slot<R>(r)];
      }
    }
  }
  __syncthreads();
}
template <int R, bool INV, int IPT>
__device__ __noinline__ void big_stage(float2* buf, int nlines, int ls, int n, int Ns, const float2* tw) {
  big_stage_body<R, INV, IPT>(buf, nlines, ls, n, Ns, tw);
}

// the stages of a power-of-two length L >= 128 with compile-time radices (16 first, then what is
// left: 8, 16, 2 or 4), inlined one after the other: no calls, so no registers saved to local memory
// around them as for the run-time plans
template <int L, bool INV>
__device__ __forceinline__ void pow2_stages(float2* buf, int nlines, int ls, const float2* tw) {
  big_stage_body<16, INV, 1>(buf, nlines, ls, L, 1, tw);
  if constexpr (L == 128) {
    big_stage_body<8, INV, 1>(buf, nlines, ls, L, 16, tw);
  } else {
    big_stage_body<16, INV, 1>(buf, nlines, ls, L, 16, tw);
    if constexpr (L == 512) big_stage_body<2, INV, 4>(buf, nlines, ls, L, 256, tw);
    if constexpr (L == 1024) big_stage_body<4, INV, 2>(buf, nlines, ls, L, 256, tw);
  }
}
template <bool INV>
__device__ __forceinline__ bool pow2_dispatch(float2* buf, int nlines, int ls, int L, const float2* tw) {
  switch (L) {
    case 128: pow2_stages<128, INV>(buf, nlines, ls, tw); return true;
    case 256: pow2_stages<256, INV>(buf, nlines, ls, tw); return true;
    case 512: pow2_stages<512, INV>(buf, nlines, ls, tw); return true;
    case 1024: pow2_stages<1024, INV>(buf, nlines, ls, tw); return true;
    default: return false;
  }
}


// all stages of a length-n transform (radices of the plan)
template <bool INV>
__device__ __noinline__ void big_stages(float2* buf, int nlines, int ls, int n, const Radices& rr, const float2* tw) {
  int ns = 1;
  for (int s = 0; s < rr.n_st; ++s) {
    const int R = rr.r[s];
    switch (R) {
      case 2: big_stage<2, INV, 4>(buf, nlines, ls, n, ns, tw); break;
      case 3: big_stage<3, INV, 3>(buf, nlines, ls, n, ns, tw); break;
      case 4: big_stage<4, INV, 2>(buf, nlines, ls, n, ns, tw); break;
      case 5: big_stage<5, INV, 2>(buf, nlines, ls, n, ns, tw); break;
      case 7: big_stage<7, INV, 1>(buf, nlines, ls, n, ns, tw); break;
      case 8: big_stage<8, INV, 1>(buf, nlines, ls, n, ns, tw); break;
      case 16: big_stage<16, INV, 1>(buf, nlines, ls, n, ns, tw); break;
      default: break;   // host planning only makes radices 2, 3, 4, 5, 7, 8, 16
    }
    ns *= R;
  }
}

// the plan's twiddle table (length M, or n without Bluestein) copied to shared memory; no synchronisation
__device__ __forceinline__ const float2* stage_tw(float2* dst, const BigPlan& pl, const float2* tabs) {
  const int L = pl.M ? pl.M : pl.n;
  for (int t = threadIdx.x; t < L; t += NT) dst[t] = __ldg(tabs + pl.tw + t);
  return dst;
}

// tw: the plan's twiddle table (in shared memory); ends synchronised
template <bool INV>
__device__ void fcore(float2* buf, int nlines, int ls, const BigPlan& pl, const float2* tabs, const float2* tw) {
  if (pl.M == 0) {
    if (!pow2_dispatch<INV>(buf, nlines, ls, pl.n, tw)) big_stages<INV>(buf, nlines, ls, pl.n, pl.rad, tw);
    return;
  }
  const int M = pl.M;
  const float2* bh = tabs + pl.bhat;
  if (!pow2_dispatch<false>(buf, nlines, ls, M, tw)) big_stages<false>(buf, nlines, ls, M, pl.rad, tw);
  for (int line = 0; line < nlines; ++line) {
    float2* b = buf + (size_t)line * ls;
    for (int j = threadIdx.x; j < M; j += NT) b[j] = cmul(b[j], __ldg(bh + j));
  }
  __syncthreads();
  if (!pow2_dispatch<true>(buf, nlines, ls, M, tw)) big_stages<true>(buf, nlines, ls, M, pl.rad, tw);
}

// ---- column pass: item = (image, map, first column, columns) ------------------------------------
// B = 1: the inverse transform of w_hat_k = sum_j conj(d_hat_jk) lambda_hat_j; B = 0: the forward
// transform of the stored row spectra; B = 2 (one-channel items, J = 1): the forward transform, the
// product with P and the inverse transform, in shared memory (lambda_hat = P F(q), then back)
template <int B>
__global__ void __launch_bounds__(NT, kMinCtas) k_big_cols(BigArgs a) {
  constexpr bool BUILD = (B == 1);
  extern __shared__ float2 sm[];
  __shared__ BigPlan pl;
  const BigItem it = a.col_items[blockIdx.x];
  const BigImg im = a.img[it.img];
  const BigCls& bc = a.cls[im.cls];
  if (threadIdx.x == 0) pl = bc.pcol;
  __syncthreads();
  const float2* tw = stage_tw(sm + a.col_smem / sizeof(float2), pl, a.tabs);
  const int H = bc.H, Wc = bc.Wc, Om = H * Wc, nc = it.count, kw0 = it.first;
  const int ls = bc.col_ls;
  const FastDiv fnc((unsigned)nc);
  float2* Y = a.Y + (a.one ? im.xh : im.y + (size_t)it.map * Om);
  if (BUILD) {
    const float2* lam = a.lam + im.lam;
    const size_t dbase = bc.dhat + (size_t)it.map * a.J * Om;
    for (int i = threadIdx.x; i < nc * H; i += NT) {
      const int h = (int)fnc.div(i), c = i - h * nc;
      const int o = h * Wc + kw0 + c;
      float2 s = make_float2(0.f, 0.f);
      for (int j = 0; j < a.J; ++j) {
        const size_t q = dbase + (size_t)j * Om + o;
        const float2 l = lam[(size_t)j * Om + o];
        s = a.dhat16 ? cfmac(__bfloat1622float2(a.dhat16[q]), bbf16(l), s) : cfmac(a.dhat[q], l, s);
      }
      sm[(size_t)c * ls + h] = fin<true>(s, h, pl, a.tabs);
    }
  } else {
    for (int i = threadIdx.x; i < nc * H; i += NT) {
      const int h = (int)fnc.div(i), c = i - h * nc;
      sm[(size_t)c * ls + h] = fin<false>(Y[(size_t)h * Wc + kw0 + c], h, pl, a.tabs);
    }
  }
  fpad(sm, nc, ls, pl);
  __syncthreads();
  fcore<BUILD>(sm, nc, ls, pl, a.tabs, tw);
  if (B == 2) {
    // each element is read and rewritten by the same thread; the padding [n, M) is not read
    const float* pd = a.pdiag + bc.pd;
    for (int i = threadIdx.x; i < nc * H; i += NT) {
      const int h = (int)fnc.div(i), c = i - h * nc;
      const float p = pd[h * Wc + kw0 + c];
      const float2 X = fout<false>(sm[(size_t)c * ls + h], h, pl, a.tabs);
      sm[(size_t)c * ls + h] = fin<true>(make_float2(X.x * p, X.y * p), h, pl, a.tabs);
    }
    fpad(sm, nc, ls, pl);
    __syncthreads();
    fcore<true>(sm, nc, ls, pl, a.tabs, tw);
  }
  for (int i = threadIdx.x; i < nc * H; i += NT) {
    const int h = (int)fnc.div(i), c = i - h * nc;
    Y[(size_t)h * Wc + kw0 + c] = fout<(B != 0)>(sm[(size_t)c * ls + h], h, pl, a.tabs);
  }
}

// ---- row pass: item = (image, map, first row, rows) ----------------------------------------------
// Two real rows a, b share one complex transform: the inverse transforms Z = X_a + i X_b (each row
// spectrum completed by Hermitian symmetry, the imaginary parts of its DC and Nyquist bins dropped,
// as a real inverse transform does) into z = x_a + i x_b; the forward transform of u_a + i u_b gives
// U_a(k) = (Z(k) + conj Z(-k)) / 2 and U_b(k) = (Z(k) - conj Z(-k)) / 2i.
__device__ __forceinline__ float2 half_bin(const float2* row, int kw, int W, int Wc) {
  float2 v = kw < Wc ? row[kw] : row[W - kw];
  if (kw >= Wc) v.y = -v.y;
  if (kw == 0 || 2 * kw == W) v.y = 0.f;
  return v;
}

// one-channel items (the direct spatial route): the forward row transform of q (read raw from a.v),
// and the inverse row transform written to a.v as a real plane (lambda), with no state update
constexpr int kRawFwd = 4, kRawInv = 5;

template <int MODE>
__global__ void __launch_bounds__(NT, kMinCtas) k_big_rows(BigArgs a) {
  extern __shared__ float2 sm[];
  __shared__ BigPlan pl;
  __shared__ double red[NT / 32];
  const BigItem it = a.row_items[blockIdx.x];
  const BigImg im = a.img[it.img];
  const BigCls& bc = a.cls[im.cls];
  if (threadIdx.x == 0) pl = bc.prow;
  __syncthreads();
  const float2* tw = stage_tw(sm + a.row_smem / sizeof(float2), pl, a.tabs);
  const int H = bc.H, W = bc.W, Wc = bc.Wc, Om = H * Wc, nr = it.count, h0 = it.first;
  const int np = (nr + 1) / 2;
  const int ls = bc.row_ls;
  const FastDiv fW((unsigned)W), fWc((unsigned)Wc);
  const size_t moff = a.one ? (size_t)im.x : im.v + (size_t)it.map * H * W;
  float2* Y = a.Y + (a.one ? im.xh : im.y + (size_t)it.map * Om);
  const float beta = a.beta;
  const bool pair_last = !(nr & 1);   // the last transform line holds two rows
  double l1 = 0.0;
  if (MODE == kIter || MODE == kLast || MODE == kRawInv) {
    for (int i = threadIdx.x; i < np * W; i += NT) {
      const int q = (int)fW.div(i), kw = i - q * W;
      const float2 xa = half_bin(Y + (size_t)(h0 + 2 * q) * Wc, kw, W, Wc);
      const float2 xb = (2 * q + 1 < nr) ? half_bin(Y + (size_t)(h0 + 2 * q + 1) * Wc, kw, W, Wc) : make_float2(0.f, 0.f);
      sm[(size_t)q * ls + kw] = fin<true>(make_float2(xa.x - xb.y, xa.y + xb.x), kw, pl, a.tabs);
    }
    fpad(sm, np, ls, pl);
    __syncthreads();
    fcore<true>(sm, np, ls, pl, a.tabs, tw);
    for (int i = threadIdx.x; i < np * W; i += NT) {
      const int q = (int)fW.div(i), x = i - q * W;
      const bool has_b = (q < np - 1) || pair_last;
      const float2 w = fout<true>(sm[(size_t)q * ls + x], x, pl, a.tabs);
      const size_t pa = moff + (size_t)(h0 + 2 * q) * W + x, pb = pa + W;
      if (MODE == kRawInv) {
        a.v[pa] = w.x;
        if (has_b) a.v[pb] = w.y;
        continue;
      }
      const float va = a.v[pa], vb = has_b ? a.v[pb] : 0.f;
      const float na = w.x - (bclamp(va, beta) - va), nb = w.y - (bclamp(vb, beta) - vb);
      const float ca = bclamp(na, beta), cb = bclamp(nb, beta);
      a.v[pa] = na;
      if (has_b) a.v[pb] = nb;
      if (MODE == kLast) {
        if (a.z) {
          a.z[pa] = a.rho * (ca - na);
          if (has_b) a.z[pb] = a.rho * (cb - nb);
        }
      } else {
        sm[(size_t)q * ls + x] = fin<false>(make_float2(2.f * ca - na, has_b ? 2.f * cb - nb : 0.f), x, pl, a.tabs);
      }
    }
    if (MODE != kLast && MODE != kRawInv) fpad(sm, np, ls, pl);
  } else {
    const float* src = (MODE == kPrologue || MODE == kRawFwd) ? a.v : a.z;
    for (int i = threadIdx.x; i < np * W; i += NT) {
      const int q = (int)fW.div(i), x = i - q * W;
      const bool has_b = (q < np - 1) || pair_last;
      const size_t pa = moff + (size_t)(h0 + 2 * q) * W + x;
      float ta = src[pa], tb = has_b ? src[pa + W] : 0.f;
      if (MODE == kPrologue) {
        ta = 2.f * bclamp(ta, beta) - ta;
        tb = 2.f * bclamp(tb, beta) - tb;
      } else if (MODE == kObjective) {
        l1 += fabs((double)ta) + fabs((double)tb);
      }
      sm[(size_t)q * ls + x] = fin<false>(make_float2(ta, tb), x, pl, a.tabs);
    }
    fpad(sm, np, ls, pl);
  }
  if (MODE != kLast && MODE != kRawInv) {
    __syncthreads();
    fcore<false>(sm, np, ls, pl, a.tabs, tw);
    for (int i = threadIdx.x; i < nr * Wc; i += NT) {
      const int r = (int)fWc.div(i), kw = i - r * Wc;
      const float2* zq = sm + (size_t)(r >> 1) * ls;
      const int km = kw == 0 ? 0 : W - kw;
      const float2 z1 = fout<false>(zq[kw], kw, pl, a.tabs), z2 = fout<false>(zq[km], km, pl, a.tabs);
      float2 u;
      if (r & 1) u = make_float2(0.5f * (z1.y + z2.y), 0.5f * (z2.x - z1.x));
      else u = make_float2(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y));
      Y[(size_t)(h0 + r) * Wc + kw] = u;
    }
  }
  if (MODE == kObjective) {
    for (int off = 16; off > 0; off >>= 1) l1 += __shfl_down_sync(0xffffffffu, l1, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l1;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red[w];
      a.l1_items[blockIdx.x] = s;
    }
  }
}

// ---- per frequency: r_hat = sum_k d_hat_k u_hat_k - x_hat / rho; lambda_hat = P r_hat, or (objective)
// the residual energy (1/D) sum_w wt(w) |sum_k d_hat_k z_hat_k - x_hat|^2 -------------------------
template <int MODE>
__global__ void __launch_bounds__(NT) k_big_freq(BigArgs a) {
  __shared__ double red[NT / 32];
  const BigItem it = a.freq_items[blockIdx.x];
  const BigImg im = a.img[it.img];
  const BigCls& bc = a.cls[im.cls];
  const int H = bc.H, W = bc.W, Wc = bc.Wc, Om = H * Wc, J = a.J, K = a.K;
  const float irho = 1.0f / a.rho;
  double e = 0.0;
  const int o = it.first + threadIdx.x;
  if (threadIdx.x < it.count) {
    float2 r[kMaxJ];
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j) {
      if (j < J) {
        const float2 x = a.xhat[im.xh + (size_t)j * Om + o];
        r[j] = MODE == kObjective ? make_float2(-x.x, -x.y) : make_float2(-x.x * irho, -x.y * irho);
      }
    }
    const float2* Yb = a.Y + im.y;
    const float2* db = a.dhat + bc.dhat;
    // mixed precision (not the objective): both operands of every product in bfloat16
    const __nv_bfloat162* db16 = (MODE != kObjective && a.dhat16) ? a.dhat16 + bc.dhat : nullptr;
    for (int k = 0; k < K; ++k) {
      const float2 u = Yb[(size_t)k * Om + o];
      if (db16) {
        const float2 ub = bbf16(u);
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j)
          if (j < J) r[j] = cfma(__bfloat1622float2(db16[((size_t)k * J + j) * Om + o]), ub, r[j]);
      } else {
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j)
          if (j < J) r[j] = cfma(db[((size_t)k * J + j) * Om + o], u, r[j]);
      }
    }
    if (MODE == kObjective) {
      const int kw = o % Wc;
      const double wt = (kw == 0 || 2 * kw == W) ? 1.0 : 2.0;
#pragma unroll
      for (int j = 0; j < kMaxJ; ++j)
        if (j < J) e += wt * ((double)r[j].x * r[j].x + (double)r[j].y * r[j].y);
    } else if (J == 1) {
      a.lam[im.lam + o] = cscale(r[0], a.pdiag[bc.pd + o]);
    } else {
      const float2* pm = a.pmat + bc.pm + (size_t)o * J * J;
#pragma unroll
      for (int i = 0; i < kMaxJ; ++i) {
        if (i < J) {
          float2 s = make_float2(0.f, 0.f);
#pragma unroll
          for (int j = 0; j < kMaxJ; ++j)
            if (j < J) s = cfma(pm[i * J + j], r[j], s);
          a.lam[im.lam + (size_t)i * Om + o] = s;
        }
      }
    }
  }
  if (MODE == kObjective) {
    for (int off = 16; off > 0; off >>= 1) e += __shfl_down_sync(0xffffffffu, e, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red[w];
      a.e_items[blockIdx.x] = s / (double)(H * W);
    }
  }
}

// ---- spectra for the setup: the forward row transform of real maps (images, or filters placed with
// their taps centred: tap (ta, tb) at ((ta - (fh-1)/2) mod H, (tb - (fw-1)/2) mod W)) -----------------
__global__ void __launch_bounds__(NT, kMinCtas) k_big_setup_rows(BigArgs a, const BigSetupItem* items, const float* d,
                                                       const float* x, float2* dhat, float2* xhat, int fh, int fw) {
  extern __shared__ float2 sm[];
  __shared__ BigPlan pl;
  const BigSetupItem it = items[blockIdx.x];
  const BigCls& bc = a.cls[it.cls];
  if (threadIdx.x == 0) pl = bc.prow;
  __syncthreads();
  const float2* tw = stage_tw(sm + a.row_smem / sizeof(float2), pl, a.tabs);
  const int H = bc.H, W = bc.W, Wc = bc.Wc, nr = it.count, h0 = it.first;
  const int ls = bc.row_ls;
  const float* src = (it.filter ? d : x) + it.src;
  float2* dst = (it.filter ? dhat : xhat) + it.dst;
  const int ch = (fh - 1) / 2, cw = (fw - 1) / 2;
  for (int i = threadIdx.x; i < nr * W; i += NT) {
    const int r = i / W, col = i - r * W, h = h0 + r;
    float v = 0.f;
    if (it.filter) {
      const int ta = (h + ch) % H, tb = (col + cw) % W;
      if (ta < fh && tb < fw) v = src[ta * fw + tb];
    } else {
      v = src[(size_t)h * W + col];
    }
    sm[(size_t)r * ls + col] = fin<false>(make_float2(v, 0.f), col, pl, a.tabs);
  }
  fpad(sm, nr, ls, pl);
  __syncthreads();
  fcore<false>(sm, nr, ls, pl, a.tabs, tw);
  for (int i = threadIdx.x; i < nr * Wc; i += NT) {
    const int r = i / Wc, kw = i - r * Wc;
    dst[(size_t)(h0 + r) * Wc + kw] = fout<false>(sm[(size_t)r * ls + kw], kw, pl, a.tabs);
  }
}

// filter spectra by direct DFT over the taps (fh x fw nonzero entries of an H x W grid): the row DFTs of
// the tap rows, R(ta, kw) = sum_tb f(ta, tb) e^{-2 pi i kw (tb - cw) / W}, kept in shared memory (TA tap
// rows at a time), then d_hat(h, kw) = sum_ta R(ta, kw) e^{-2 pi i h (ta - ch) / H}. One CTA per
// (class, map).
__global__ void __launch_bounds__(NT) k_big_filter_spectra(BigArgs a, const float* d, float2* dhat, int fh, int fw,
                                                          int KJ, int TA) {
  extern __shared__ float2 sm[];
  const int ci = blockIdx.x / KJ, m = blockIdx.x - ci * KJ;
  const BigCls& bc = a.cls[ci];
  const int H = bc.H, W = bc.W, Wc = bc.Wc;
  const int ch = (fh - 1) / 2, cw = (fw - 1) / 2;
  const float* f = d + (size_t)m * fh * fw;
  const float2* twW = a.tabs + bc.prow.twn;
  const float2* twH = a.tabs + bc.pcol.twn;
  float2* out = dhat + bc.dhat + (size_t)m * H * Wc;
  const FastDiv fWc((unsigned)Wc);
  for (int t0 = 0; t0 < fh; t0 += TA) {
    const int tn = min(TA, fh - t0);
    __syncthreads();
    for (int i = threadIdx.x; i < tn * Wc; i += NT) {
      const int ta = (int)fWc.div(i), kw = i - ta * Wc;
      float2 s = make_float2(0.f, 0.f);
      int idx = (int)(((long long)(W - cw) * kw) % W);   // (tb - cw) kw mod W, stepped by kw
      for (int tb = 0; tb < fw; ++tb) {
        const float2 t = twW[idx];
        const float fv = f[(t0 + ta) * fw + tb];
        s.x = fmaf(fv, t.x, s.x);
        s.y = fmaf(fv, t.y, s.y);
        idx += kw;
        if (idx >= W) idx -= W;
      }
      sm[i] = s;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < H * Wc; o += NT) {
      const int h = (int)fWc.div(o), kw = o - h * Wc;
      float2 s = t0 == 0 ? make_float2(0.f, 0.f) : out[o];
      int idx = (int)(((long long)(t0 - ch + H) * h) % H);   // (ta - ch) h mod H, stepped by h
      for (int ta = 0; ta < tn; ++ta) {
        s = cfma(sm[ta * Wc + kw], twH[idx], s);
        idx += h;
        if (idx >= H) idx -= H;
      }
      out[o] = s;
    }
  }
}

// the forward column transform of the setup's row spectra, in place
__global__ void __launch_bounds__(NT, kMinCtas) k_big_setup_cols(BigArgs a, const BigSetupItem* items, float2* dhat,
                                                       float2* xhat) {
  extern __shared__ float2 sm[];
  __shared__ BigPlan pl;
  const BigSetupItem it = items[blockIdx.x];
  const BigCls& bc = a.cls[it.cls];
  if (threadIdx.x == 0) pl = bc.pcol;
  __syncthreads();
  const float2* tw = stage_tw(sm + a.col_smem / sizeof(float2), pl, a.tabs);
  const int H = bc.H, Wc = bc.Wc, nc = it.count, kw0 = it.first;
  const int ls = bc.col_ls;
  float2* dst = (it.filter ? dhat : xhat) + it.dst;
  for (int i = threadIdx.x; i < nc * H; i += NT) {
    const int c = i % nc, h = i / nc;
    sm[(size_t)c * ls + h] = fin<false>(dst[(size_t)h * Wc + kw0 + c], h, pl, a.tabs);
  }
  fpad(sm, nc, ls, pl);
  __syncthreads();
  fcore<false>(sm, nc, ls, pl, a.tabs, tw);
  for (int i = threadIdx.x; i < nc * H; i += NT) {
    const int c = i % nc, h = i / nc;
    dst[(size_t)h * Wc + kw0 + c] = fout<false>(sm[(size_t)c * ls + h], h, pl, a.tabs);
  }
}

}  // namespace big

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
static cudaError_t big_attr(const void* f, size_t smem) {
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_big_sweep(const BigArgs& a, int mode, cudaStream_t st) {
  using namespace big;
  cudaError_t e = cudaSuccess;
  const size_t tws = (size_t)a.tw_max * sizeof(float2);
  const size_t csm = a.col_smem + tws, rsm = a.row_smem + tws;
  if (mode == kIter || mode == kLast) {
    if ((e = big_attr((const void*)k_big_cols<1>, csm)) != cudaSuccess) return e;
    k_big_cols<1><<<a.n_col_items, NT, csm, st>>>(a);
  }
  switch (mode) {
    case kPrologue:
      if ((e = big_attr((const void*)k_big_rows<kPrologue>, rsm)) != cudaSuccess) return e;
      k_big_rows<kPrologue><<<a.n_row_items, NT, rsm, st>>>(a);
      break;
    case kIter:
      if ((e = big_attr((const void*)k_big_rows<kIter>, rsm)) != cudaSuccess) return e;
      k_big_rows<kIter><<<a.n_row_items, NT, rsm, st>>>(a);
      break;
    case kLast:
      if ((e = big_attr((const void*)k_big_rows<kLast>, rsm)) != cudaSuccess) return e;
      k_big_rows<kLast><<<a.n_row_items, NT, rsm, st>>>(a);
      break;
    default:
      if ((e = big_attr((const void*)k_big_rows<kObjective>, rsm)) != cudaSuccess) return e;
      k_big_rows<kObjective><<<a.n_row_items, NT, rsm, st>>>(a);
      break;
  }
  if (mode == kLast) return cudaGetLastError();
  if ((e = big_attr((const void*)k_big_cols<0>, csm)) != cudaSuccess) return e;
  k_big_cols<0><<<a.n_col_items, NT, csm, st>>>(a);
  if (mode == kObjective) k_big_freq<kObjective><<<a.n_freq_items, NT, 0, st>>>(a);
  else k_big_freq<kIter><<<a.n_freq_items, NT, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_big_lambda1(const BigArgs& a, cudaStream_t st) {
  using namespace big;
  cudaError_t e;
  const size_t tws = (size_t)a.tw_max * sizeof(float2);
  const size_t csm = a.col_smem + tws, rsm = a.row_smem + tws;
  if ((e = big_attr((const void*)k_big_rows<kRawFwd>, rsm)) != cudaSuccess) return e;
  if ((e = big_attr((const void*)k_big_cols<2>, csm)) != cudaSuccess) return e;
  if ((e = big_attr((const void*)k_big_rows<kRawInv>, rsm)) != cudaSuccess) return e;
  k_big_rows<kRawFwd><<<a.n_row_items, NT, rsm, st>>>(a);
  k_big_cols<2><<<a.n_col_items, NT, csm, st>>>(a);
  k_big_rows<kRawInv><<<a.n_row_items, NT, rsm, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_big_setup(const BigArgs& a, const BigSetupItem* row_items, int n_rows,
                             const BigSetupItem* col_items, int n_cols, const float* d, const float* x,
                             float2* dhat, float2* xhat, int fh, int fw, int n_classes, cudaStream_t st) {
  using namespace big;
  cudaError_t e;
  const size_t tws = (size_t)a.tw_max * sizeof(float2);
  if ((e = big_attr((const void*)k_big_setup_rows, a.row_smem + tws)) != cudaSuccess) return e;
  if ((e = big_attr((const void*)k_big_setup_cols, a.col_smem + tws)) != cudaSuccess) return e;
  const int wmax = kBigMaxSide / 2 + 1;
  const int TA = std::min(fh, std::max(1, (int)((64 * 1024) / (wmax * sizeof(float2)))));
  const size_t fsm = (size_t)TA * wmax * sizeof(float2);
  if ((e = big_attr((const void*)k_big_filter_spectra, fsm)) != cudaSuccess) return e;
  k_big_filter_spectra<<<n_classes * a.K * a.J, NT, fsm, st>>>(a, d, dhat, fh, fw, a.K * a.J, TA);
  if (n_rows > 0) k_big_setup_rows<<<n_rows, NT, a.row_smem + tws, st>>>(a, row_items, d, x, dhat, xhat, fh, fw);
  if (n_cols > 0) k_big_setup_cols<<<n_cols, NT, a.col_smem + tws, st>>>(a, col_items, dhat, xhat);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// host planning
// ---------------------------------------------------------------------------------------------
namespace {

bool smooth7(int n) {
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

// the DFT of x (length n, any factorisation) in double: recursive decimation in time on the smallest
// prime factor
void host_dft(const double* xr, const double* xi, int n, int stride, double* yr, double* yi) {
  if (n == 1) { yr[0] = xr[0]; yi[0] = xi[0]; return; }
  int p = 2;
  while (n % p) ++p;
  const int m = n / p;
  std::vector<double> sr(n), si(n);
  for (int r = 0; r < p; ++r) host_dft(xr + r * stride, xi + r * stride, m, stride * p, &sr[r * m], &si[r * m]);
  const double pi2 = 6.283185307179586476925286766559;
  for (int k = 0; k < n; ++k) {
    double ar = 0.0, ai = 0.0;
    for (int r = 0; r < p; ++r) {
      const double t = -pi2 * (double)(((long long)r * k) % n) / n;
      const double c = std::cos(t), s = std::sin(t);
      const double ur = sr[r * m + k % m], ui = si[r * m + k % m];
      ar += ur * c - ui * s;
      ai += ur * s + ui * c;
    }
    yr[k] = ar;
    yi[k] = ai;
  }
}

void push_twiddles(std::vector<float2>& tabs, int L) {
  const double pi2 = 6.283185307179586476925286766559;
  for (int t = 0; t < L; ++t) tabs.push_back(make_float2((float)std::cos(pi2 * t / L), (float)-std::sin(pi2 * t / L)));
}

const BigPlan& plan_of(UnevenLayout& L, int n) {
  for (const BigPlan& p : L.bplans)
    if (p.n == n) return p;
  BigPlan p{};
  p.n = n;
  if (smooth7(n)) {
    p.M = 0;
    p.rad = factorize(n);
    p.tw = p.twn = (long long)L.btabs.size();
    push_twiddles(L.btabs, n);
  } else {
    p.twn = (long long)L.btabs.size();
    push_twiddles(L.btabs, n);
    // a power of two: its transforms run with compile-time radices (pow2_stages), which pays for the
    // longer circle (measured on 256 images with sides in [64, 512])
    int M = 1;
    while (M < 2 * n - 1) M *= 2;
    p.M = M;
    p.rad = factorize(M);
    p.tw = (long long)L.btabs.size();
    push_twiddles(L.btabs, M);
    // chirp w_j = exp(-pi i j^2 / n), the phase reduced mod 2n in integers
    const double pi = 3.14159265358979323846264338328;
    std::vector<double> wr(n), wi(n);
    p.chirp = (long long)L.btabs.size();
    for (int j = 0; j < n; ++j) {
      const double t = -pi * (double)(((long long)j * j) % (2LL * n)) / n;
      wr[j] = std::cos(t);
      wi[j] = std::sin(t);
      L.btabs.push_back(make_float2((float)wr[j], (float)wi[j]));
    }
    // b_m = conj(w_|m|) on the circle of length M, its DFT divided by M
    std::vector<double> br(M, 0.0), bi(M, 0.0), hr(M), hi(M);
    for (int j = 0; j < n; ++j) {
      br[j] = wr[j]; bi[j] = -wi[j];
      if (j > 0) { br[M - j] = wr[j]; bi[M - j] = -wi[j]; }
    }
    host_dft(br.data(), bi.data(), M, 1, hr.data(), hi.data());
    p.bhat = (long long)L.btabs.size();
    for (int k = 0; k < M; ++k) L.btabs.push_back(make_float2((float)(hr[k] / M), (float)(hi[k] / M)));
  }
  L.bplans.push_back(p);
  return L.bplans.back();
}

int odd_at_least(int n) { return n | 1; }

constexpr size_t kBigLineBudget = 56 * 1024;   // shared memory of the lines of a work item (bytes)

int lines_per_item(int ls, int total) {
  const int l = (int)(kBigLineBudget / ((size_t)ls * sizeof(float2)));
  return std::max(1, std::min(l, total));
}

}  // namespace

bool big_add_class(UnevenLayout& L, int H, int W) {
  if (H < 1 || W < 1 || H > kBigMaxSide || W > kBigMaxSide) return false;
  BigCls bc{};
  bc.H = H; bc.W = W; bc.Wc = W / 2 + 1;
  bc.pcol = plan_of(L, H);
  bc.prow = plan_of(L, W);
  bc.col_ls = odd_at_least(std::max(H, bc.pcol.M));
  bc.row_ls = odd_at_least(std::max(W, bc.prow.M));
  L.bcls.push_back(bc);
  L.bcls_H.push_back(H);
  L.bcls_W.push_back(W);
  return true;
}

void big_build_one_channel(UnevenLayout& L) {
  L.scol.clear(); L.srow.clear(); L.stile.clear();
  for (int i = 0; i < (int)L.bimg.size(); ++i) {
    const BigCls& bc = L.bcls[L.bimg[i].cls];
    const int nc = lines_per_item(bc.col_ls, bc.Wc), nr = lines_per_item(bc.row_ls, bc.H);
    for (int c0 = 0; c0 < bc.Wc; c0 += nc) L.scol.push_back({i, 0, c0, std::min(nc, bc.Wc - c0)});
    for (int h0 = 0; h0 < bc.H; h0 += 2 * nr) L.srow.push_back({i, 0, h0, std::min(2 * nr, bc.H - h0)});
    for (int y0 = 0; y0 < bc.H; y0 += kUspTileH)
      for (int x0 = 0; x0 < bc.W; x0 += kUspTileW) L.stile.push_back({i, y0, x0, 0});
  }
}

void big_build_items(UnevenLayout& L, int K, int J, int fh, int fw, std::vector<BigSetupItem>& setup) {
  (void)fh; (void)fw;
  L.bcol.clear(); L.brow.clear(); L.bfreq.clear(); setup.clear();
  L.bcol_smem = L.brow_smem = 0;
  L.btw_max = 0;
  for (const BigPlan& p : L.bplans) L.btw_max = std::max(L.btw_max, p.M ? p.M : p.n);
  std::vector<int> nc(L.bcls.size()), nr(L.bcls.size());
  for (size_t ci = 0; ci < L.bcls.size(); ++ci) {
    const BigCls& bc = L.bcls[ci];
    nc[ci] = lines_per_item(bc.col_ls, bc.Wc);
    nr[ci] = lines_per_item(bc.row_ls, bc.H);   // transform lines: 2 rows each in the sweeps
    L.bcol_smem = std::max(L.bcol_smem, (size_t)nc[ci] * bc.col_ls * sizeof(float2));
    L.brow_smem = std::max(L.brow_smem, (size_t)nr[ci] * bc.row_ls * sizeof(float2));
  }
  for (int i = 0; i < (int)L.bimg.size(); ++i) {
    const int ci = L.bimg[i].cls;
    const BigCls& bc = L.bcls[ci];
    const int Om = bc.H * bc.Wc;
    for (int k = 0; k < K; ++k) {
      for (int c0 = 0; c0 < bc.Wc; c0 += nc[ci]) L.bcol.push_back({i, k, c0, std::min(nc[ci], bc.Wc - c0)});
      for (int h0 = 0; h0 < bc.H; h0 += 2 * nr[ci]) L.brow.push_back({i, k, h0, std::min(2 * nr[ci], bc.H - h0)});
    }
    for (int o0 = 0; o0 < Om; o0 += big::NT) L.bfreq.push_back({i, 0, o0, std::min(big::NT, Om - o0)});
  }
  // setup: rows of every image, then their columns (the filter spectra are direct DFTs)
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i < (int)L.bimg.size(); ++i) {
      const BigImg& im = L.bimg[i];
      const BigCls& bc = L.bcls[im.cls];
      const int Om = bc.H * bc.Wc;
      for (int j = 0; j < J; ++j) {
        const long long src = im.x + (long long)j * bc.H * bc.W, dst = im.xh + (long long)j * Om;
        if (pass == 0)
          for (int h0 = 0; h0 < bc.H; h0 += nr[im.cls])
            setup.push_back({im.cls, h0, std::min(nr[im.cls], bc.H - h0), 0, src, dst});
        else
          for (int c0 = 0; c0 < bc.Wc; c0 += nc[im.cls])
            setup.push_back({im.cls, c0, std::min(nc[im.cls], bc.Wc - c0), 0, src, dst});
      }
    }
    if (pass == 0) L.n_bsetup_rows = (int)setup.size();
  }
  L.n_bsetup_cols = (int)setup.size() - L.n_bsetup_rows;
}

}  // namespace csc
