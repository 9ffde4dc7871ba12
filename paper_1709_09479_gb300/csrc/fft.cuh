// Shared-memory 2-D real FFTs for the coding and learning kernels.
//
// The dual ADMM of Sec. 3.2 runs every product with the circulant D_k = F diag(d_hat_k) F^H in the
// Fourier domain, so each map visit is one inverse and one forward 2-D DFT of an H x W real map.
// A CTA holds one map in shared memory and transforms it in place:
//
//   * layout: spectrum bin (h, c), c < Wc = W/2+1, at complex offset h*P + c; real pixel (h, w) at
//     float offset 2*P*h + w. P is Wc rounded up to an odd number, so both the row pass
//     (consecutive threads on consecutive rows, stride P) and the column pass (consecutive threads
//     on consecutive columns) hit 16 distinct 8-byte bank pairs per half-warp;
//   * rows: a real row of W samples is read as W/2 complex values y[m] = x[2m] + i x[2m+1],
//     transformed with a W/2-point complex FFT and split into the W/2+1 bins of the real DFT;
//   * columns: W/2 complex FFTs of length H: the row DC and Nyquist bins are real, so they travel
//     together as one complex column and are separated after the transform;
//   * 1-D FFTs: mixed-radix Stockham (radices 16, 8, 4, 2, 5, 3 hand-written, 7 by direct DFT),
//     in place: every round reads its butterflies into registers, syncs, writes.
//
// Forward transforms use exp(-2 pi i / n); inverse ones exp(+2 pi i / n) and are unnormalised.
// Twiddle tables are computed on the host in double precision and staged in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace csc {

#define CSC_HD __host__ __device__ __forceinline__
#define CSC_D __device__ __forceinline__

constexpr int kMaxStages = 16;
constexpr int kMaxDirectRadix = 31;

struct Radices {
  int n_st;
  int r[kMaxStages];
};

// Factor n into Stockham stages: the power of two as radix 16/8/4 (a lone 2 only when n is 2),
// then 5s, 3s, and remaining primes (direct DFT, must be <= kMaxDirectRadix).
CSC_HD constexpr Radices factorize(int n) {
  Radices out{0, {}};
  int e = 0;
  int m = n;
  while (m > 1 && m % 2 == 0) { m /= 2; ++e; }
  // split 2^e into radices 16/8/4/2 with few stages and no radix-2 where avoidable
  while (e > 0) {
    int take = 0;
    if (e >= 7 && e != 8) take = (e % 4 == 0 || e % 4 == 3) ? 4 : 3;
    else if (e == 8) take = 4;
    else if (e == 6) take = 3;
    else if (e == 5) take = 3;
    else take = (e >= 4) ? 4 : e;   // 4,3,2,1
    out.r[out.n_st++] = 1 << take;
    e -= take;
  }
  while (m % 5 == 0) { out.r[out.n_st++] = 5; m /= 5; }
  while (m % 3 == 0) { out.r[out.n_st++] = 3; m /= 3; }
  for (int p = 7; m > 1; p += 2) {
    while (m % p == 0) { out.r[out.n_st++] = p; m /= p; }
  }
  return out;
}

CSC_HD constexpr int max_radix(const Radices& rr) {
  int m = 1;
  for (int i = 0; i < rr.n_st; ++i) m = rr.r[i] > m ? rr.r[i] : m;
  return m;
}

CSC_HD constexpr int ns_before(const Radices& rr, int s) {
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= rr.r[i];
  return ns;
}

CSC_HD constexpr int odd_pitch(int wc) { return (wc & 1) ? wc : wc + 1; }

// ---------------------------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------------------------
CSC_D float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
CSC_D float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
CSC_D float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
CSC_D float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// acc + a*b
CSC_D float2 cfma(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
// acc + conj(a)*b
CSC_D float2 cfmac(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}
CSC_D float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
template <bool INV> CSC_D float2 tw_dir(float2 w) { return INV ? make_float2(w.x, -w.y) : w; }
// multiply by -i (forward) or +i (inverse)
template <bool INV> CSC_D float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// v rounded to the nearest TF32 value (10 explicit mantissa bits, ties away from zero) and back to
// float32 (operands of the TF32 contractions); NaN and Inf pass through
CSC_D float tf32r(float v) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r & 0xFFFFE000u);
}
CSC_D float2 tf32r2(float2 v) { return make_float2(tf32r(v.x), tf32r(v.y)); }

// init + sum of the partial sums p[c * stride] over slots c = c0..c1 (the CTAs that covered an
// image), in a fixed order: four running sums over c = c0 + 4 i + r, added as (s0 + s1) + (s2 + s3),
// so that four loads are in flight at a time when an image spans many CTAs
CSC_D float2 sum_slots_at(const float2* __restrict__ p, size_t stride, int c0, int c1, float2 init) {
  float2 s0 = init, s1 = make_float2(0.f, 0.f), s2 = s1, s3 = s1;
  int c = c0;
  for (; c + 3 <= c1; c += 4) {
    const float2 v0 = p[(size_t)c * stride], v1 = p[(size_t)(c + 1) * stride];
    const float2 v2 = p[(size_t)(c + 2) * stride], v3 = p[(size_t)(c + 3) * stride];
    s0 = cadd(s0, v0);
    s1 = cadd(s1, v1);
    s2 = cadd(s2, v2);
    s3 = cadd(s3, v3);
  }
  for (; c <= c1; ++c) s0 = cadd(s0, p[(size_t)c * stride]);
  return cadd(cadd(s0, s1), cadd(s2, s3));
}

// ---------------------------------------------------------------------------------------------
// small DFTs in registers (outputs in natural order)
// ---------------------------------------------------------------------------------------------
template <bool INV> CSC_D void dft2(float2* a) {
  float2 t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}

template <bool INV> CSC_D void dft4v(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_mi<INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}
template <bool INV> CSC_D void dft4(float2* a) { dft4v<INV>(a[0], a[1], a[2], a[3]); }

constexpr float kSqrtHalf = 0.70710678118654752440f;

template <bool INV> CSC_D void dft8(float2* a) {
  float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  float2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4v<INV>(e0, e1, e2, e3);
  dft4v<INV>(o0, o1, o2, o3);
  // o_q *= w8^q, w8 = exp(-+2 pi i / 8)
  float2 w1, w3;
  if (!INV) {
    w1 = make_float2(kSqrtHalf * (o1.x + o1.y), kSqrtHalf * (o1.y - o1.x));
    w3 = make_float2(kSqrtHalf * (o3.y - o3.x), -kSqrtHalf * (o3.x + o3.y));
  } else {
    w1 = make_float2(kSqrtHalf * (o1.x - o1.y), kSqrtHalf * (o1.x + o1.y));
    w3 = make_float2(-kSqrtHalf * (o3.x + o3.y), kSqrtHalf * (o3.x - o3.y));
  }
  float2 w2 = mul_mi<INV>(o2);
  a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
  a[1] = cadd(e1, w1); a[5] = csub(e1, w1);
  a[2] = cadd(e2, w2); a[6] = csub(e2, w2);
  a[3] = cadd(e3, w3); a[7] = csub(e3, w3);
}

// 16 = 4 x 4: input n = 4 n1 + n2, output k = k1 + 4 k2 left at a[4 k1 + k2] (transposed;
// out_slot<16> gives the position of output k, resolved at compile time by the caller)
template <bool INV> CSC_D void dft16(float2* a) {
  // cos/sin(2 pi m / 16), m = 1, 3 (the twiddles w16^(n2 k1) with n2, k1 in 0..3 need m up to 9)
  constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4v<INV>(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
  // now a[4 k1 + n2] holds B[n2][k1]; multiply by w16^(n2 k1)
  auto rot = [](float2 v, float c, float s) {  // v * (c - i s) forward, (c + i s) inverse
    return INV ? make_float2(v.x * c - v.y * s, v.x * s + v.y * c)
               : make_float2(v.x * c + v.y * s, v.y * c - v.x * s);
  };
  // k1 = 1: n2 = 1,2,3 -> m = 1,2,3
  a[5] = rot(a[5], c1, s1);
  a[6] = rot(a[6], kSqrtHalf, kSqrtHalf);
  a[7] = rot(a[7], s1, c1);
  // k1 = 2: m = 2,4,6
  a[9] = rot(a[9], kSqrtHalf, kSqrtHalf);
  a[10] = mul_mi<INV>(a[10]);
  a[11] = rot(a[11], -kSqrtHalf, kSqrtHalf);
  // k1 = 3: m = 3,6,9
  a[13] = rot(a[13], s1, c1);
  a[14] = rot(a[14], -kSqrtHalf, kSqrtHalf);
  a[15] = rot(a[15], -c1, -s1);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4v<INV>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
}

// register slot holding output k of dft<R> (identity except for the transposed radix 16)
template <int R> CSC_HD constexpr int out_slot(int k) { return R == 16 ? 4 * (k % 4) + k / 4 : k; }

template <bool INV> CSC_D void dft3(float2* a) {
  constexpr float h = 0.86602540378443864676f;  // sin(2 pi / 3)
  float2 t = cadd(a[1], a[2]);
  float2 m = make_float2(a[0].x - 0.5f * t.x, a[0].y - 0.5f * t.y);
  float2 d = csub(a[1], a[2]);
  float2 r = mul_mi<INV>(make_float2(h * d.x, h * d.y));   // -+ i h (a1 - a2)
  a[0] = cadd(a[0], t);
  a[1] = cadd(m, r);
  a[2] = csub(m, r);
}

template <bool INV> CSC_D void dft5(float2* a) {
  constexpr float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
  constexpr float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
  constexpr float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
  constexpr float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
  float2 t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
  float2 t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
  float2 a0 = a[0];
  float2 p1 = make_float2(a0.x + c1 * t1.x + c2 * t2.x, a0.y + c1 * t1.y + c2 * t2.y);
  float2 p2 = make_float2(a0.x + c2 * t1.x + c1 * t2.x, a0.y + c2 * t1.y + c1 * t2.y);
  float2 q1 = make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
  float2 q2 = make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
  float2 iq1 = mul_mi<INV>(q1), iq2 = mul_mi<INV>(q2);   // -+ i q
  a[0] = cadd(a0, cadd(t1, t2));
  a[1] = cadd(p1, iq1);
  a[4] = csub(p1, iq1);
  a[2] = cadd(p2, iq2);
  a[3] = csub(p2, iq2);
}

// direct DFT of prime length R from the stage's length-n twiddle table (w_R^m = tw[m n / R])
template <int R, bool INV> CSC_D void dft_direct(float2* a, const float2* tw, int n) {
  const int st = n / R;
  float2 o[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    float2 acc = a[0];
#pragma unroll
    for (int r = 1; r < R; ++r) acc = cfma(a[r], tw_dir<INV>(tw[((r * q) % R) * st]), acc);
    o[q] = acc;
  }
#pragma unroll
  for (int q = 0; q < R; ++q) a[q] = o[q];
}

template <int R, bool INV> CSC_D void dft(float2* a, const float2* tw, int n) {
  if constexpr (R == 2) dft2<INV>(a);
  else if constexpr (R == 3) dft3<INV>(a);
  else if constexpr (R == 4) dft4<INV>(a);
  else if constexpr (R == 5) dft5<INV>(a);
  else if constexpr (R == 8) dft8<INV>(a);
  else if constexpr (R == 16) dft16<INV>(a);
  else dft_direct<R, INV>(a, tw, n);
}

// ---------------------------------------------------------------------------------------------
// one Stockham stage over a batch of lines, in place
//   line L element e at buf[L*lstride + e*es]; Ns = product of earlier radices.
// ---------------------------------------------------------------------------------------------
// butterflies a thread holds per round: a register budget of 32 complex values (16 at 1024
// threads); fixed-size plans ask for no more than one round needs (see stage_ipt)
template <int R, int NT> constexpr int items_per_thread() {
  return (NT >= 1024 ? 16 : 32) / R > 0 ? (NT >= 1024 ? 16 : 32) / R : 1;
}
CSC_HD constexpr int stage_ipt(int R, int NT, int n, int nlines, int cap) {
  const int need = (nlines * (n / R) + NT - 1) / NT;
  return need < cap ? (need > 0 ? need : 1) : cap;
}

template <int R, bool INV, int NT, int IPT = items_per_thread<R, NT>()>
CSC_D void fft_stage(float2* __restrict__ buf, int nlines, int lstride, int es, int n, int Ns,
                     const float2* __restrict__ tw) {
  const int nb = n / R;
  int lpr = (NT * IPT) / nb;
  if (lpr > nlines) lpr = nlines;
  if (lpr < 1) lpr = 1;
  const int tsu = n / (Ns * R);
  for (int L0 = 0; L0 < nlines; L0 += lpr) {
    const int nl = min(lpr, nlines - L0);
    const int items = nl * nb;
    float2 v[IPT][R];
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      const int i = threadIdx.x + it * NT;
      if (i < items) {
        const int line = L0 + i % nl, j = i / nl;
        const float2* src = buf + line * lstride + j * es;
        const int ts = (j % Ns) * tsu;
        v[it][0] = src[0];
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 x = src[r * nb * es];
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
        const int line = L0 + i % nl, j = i / nl;
        const int k = j % Ns;
        float2* dst = buf + line * lstride + ((j - k) * R + k) * es;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[r * Ns * es] = v[it][out_slot<R>(r)];
      }
    }
  }
  __syncthreads();
}

// all stages of a length-N transform over NLINES lines, radices fixed at compile time
template <int N, int S, bool INV, int NT, int NLINES>
CSC_D void stages_ct(float2* buf, int lstride, int es, const float2* tw) {
  constexpr Radices rr = factorize(N);
  if constexpr (S < rr.n_st) {
    constexpr int R = rr.r[S];
    constexpr int NS = ns_before(rr, S);
    constexpr int IPT = stage_ipt(R, NT, N, NLINES, items_per_thread<R, NT>());
    fft_stage<R, INV, NT, IPT>(buf, NLINES, lstride, es, N, NS, tw);
    stages_ct<N, S + 1, INV, NT, NLINES>(buf, lstride, es, tw);
  }
}

// one run-time stage as a call of its own: each radix gets its own register allocation (inlined
// together behind a switch they share one, and spill)
template <int R, bool INV, int NT, int IPT>
__device__ __noinline__ void fft_stage_rt(float2* buf, int nlines, int lstride, int es, int n, int Ns,
                                          const float2* tw) {
  fft_stage<R, INV, NT, IPT>(buf, nlines, lstride, es, n, Ns, tw);
}

// run-time radices (sizes without a fixed-size instantiation): dispatch each stage to its radix,
// at most 16 complex values per thread and round
template <bool INV, int NT>
__device__ __noinline__ void stages_rt(float2* buf, int nlines, int lstride, int es, int n,
                                       const Radices& rr, const float2* tw) {
  int ns = 1;
  for (int s = 0; s < rr.n_st; ++s) {
    const int R = rr.r[s];
    switch (R) {
      case 2: fft_stage_rt<2, INV, NT, 8>(buf, nlines, lstride, es, n, ns, tw); break;
      case 3: fft_stage_rt<3, INV, NT, 5>(buf, nlines, lstride, es, n, ns, tw); break;
      case 4: fft_stage_rt<4, INV, NT, 4>(buf, nlines, lstride, es, n, ns, tw); break;
      case 5: fft_stage_rt<5, INV, NT, 3>(buf, nlines, lstride, es, n, ns, tw); break;
      case 7: fft_stage_rt<7, INV, NT, 2>(buf, nlines, lstride, es, n, ns, tw); break;
      case 8: fft_stage_rt<8, INV, NT, 2>(buf, nlines, lstride, es, n, ns, tw); break;
      case 16: fft_stage_rt<16, INV, NT, 1>(buf, nlines, lstride, es, n, ns, tw); break;
      default: break;   // host planning rejects other radices
    }
    ns *= R;
  }
}

// radices the run-time path implements
CSC_HD constexpr bool radix_supported_rt(int r) {
  return r == 2 || r == 3 || r == 4 || r == 5 || r == 7 || r == 8 || r == 16;
}

// ---------------------------------------------------------------------------------------------
// 2-D geometry: compile-time (fixed sizes) or run-time
// ---------------------------------------------------------------------------------------------
template <int H_, int W_>
struct GeoCT {
  static constexpr int H = H_, W = W_, Wh = W_ / 2, Wc = W_ / 2 + 1, P = odd_pitch(W_ / 2 + 1);
  static constexpr int Omega = H_ * (W_ / 2 + 1), D = H_ * W_;
  CSC_D int h() const { return H; }
  CSC_D int w() const { return W; }
  CSC_D int wh() const { return Wh; }
  CSC_D int wc() const { return Wc; }
  CSC_D int p() const { return P; }
  CSC_D int omega() const { return Omega; }
  CSC_D int d() const { return D; }
  template <bool INV, int NT> CSC_D void rows(float2* buf, const float2* tw) const {
    stages_ct<Wh, 0, INV, NT, H>(buf, P, 1, tw);
  }
  template <bool INV, int NT> CSC_D void cols(float2* buf, const float2* tw) const {
    stages_ct<H, 0, INV, NT, Wh>(buf, 1, P, tw);
  }
};

struct GeoRT {
  int H, W, Wh, Wc, P, Omega, D;
  Radices rrow, rcol;
  CSC_D int h() const { return H; }
  CSC_D int w() const { return W; }
  CSC_D int wh() const { return Wh; }
  CSC_D int wc() const { return Wc; }
  CSC_D int p() const { return P; }
  CSC_D int omega() const { return Omega; }
  CSC_D int d() const { return D; }
  template <bool INV, int NT> CSC_D void rows(float2* buf, const float2* tw) const {
    stages_rt<INV, NT>(buf, H, P, 1, Wh, rrow, tw);
  }
  template <bool INV, int NT> CSC_D void cols(float2* buf, const float2* tw) const {
    stages_rt<INV, NT>(buf, Wh, 1, P, H, rcol, tw);
  }
};

// twiddle tables staged in shared memory: [Wh] row FFT, [H] column FFT, [Wc] real split
struct Twiddles {
  const float2* row;
  const float2* col;
  const float2* split;
};

template <class G>
CSC_HD int twiddle_count(const G& g) { return g.wh() + g.h() + g.wc(); }

// ---------------------------------------------------------------------------------------------
// real <-> half-spectrum split of each row (see file comment)
// ---------------------------------------------------------------------------------------------
template <class G, int NT>
CSC_D void split_rows_forward(const G& g, float2* buf, const float2* wsplit) {
  const int H = g.h(), Wh = g.wh(), P = g.p();
  const int pairs = Wh / 2 + 1;
  for (int i = threadIdx.x; i < H * pairs; i += NT) {
    const int h = i % H, k = i / H;
    float2* row = buf + h * P;
    if (k == 0) {
      // the real DC and Nyquist bins of the row share bin 0: X[0] + i X[Wh]
      const float2 y = row[0];
      row[0] = make_float2(y.x + y.y, y.x - y.y);
    } else {
      const int k2 = Wh - k;
      const float2 ya = row[k], yb = row[k2];
      // X[a] = (Ya + conj Yb)/2 - i w^a (Ya - conj Yb)/2,  w^a = exp(-2 pi i a / W)
      {
        const float2 s = make_float2(ya.x + yb.x, ya.y - yb.y);
        const float2 d = make_float2(ya.x - yb.x, ya.y + yb.y);
        const float2 wd = cmul(wsplit[k], d);
        row[k] = make_float2(0.5f * (s.x + wd.y), 0.5f * (s.y - wd.x));
      }
      if (k2 != k) {
        const float2 s = make_float2(yb.x + ya.x, yb.y - ya.y);
        const float2 d = make_float2(yb.x - ya.x, yb.y + ya.y);
        const float2 wd = cmul(wsplit[k2], d);
        row[k2] = make_float2(0.5f * (s.x + wd.y), 0.5f * (s.y - wd.x));
      }
    }
  }
  __syncthreads();
}

template <class G, int NT>
CSC_D void split_rows_inverse(const G& g, float2* buf, const float2* wsplit) {
  const int H = g.h(), Wh = g.wh(), P = g.p();
  const int pairs = Wh / 2 + 1;
  for (int i = threadIdx.x; i < H * pairs; i += NT) {
    const int h = i % H, k = i / H;
    float2* row = buf + h * P;
    if (k == 0) {
      // bin 0 carries the row's DC (real part) and Nyquist (imaginary part) values
      const float a = row[0].x, b = row[0].y;
      row[0] = make_float2(a + b, a - b);
    } else {
      const int k2 = Wh - k;
      const float2 xa = row[k], xb = row[k2];
      // Y[a] = (Xa + conj Xb) + i conj(w^a) (Xa - conj Xb)
      {
        const float2 s = make_float2(xa.x + xb.x, xa.y - xb.y);
        const float2 d = make_float2(xa.x - xb.x, xa.y + xb.y);
        const float2 e = cmulc(d, wsplit[k]);
        row[k] = make_float2(s.x - e.y, s.y + e.x);
      }
      if (k2 != k) {
        const float2 s = make_float2(xb.x + xa.x, xb.y - xa.y);
        const float2 d = make_float2(xb.x - xa.x, xb.y + xa.y);
        const float2 e = cmulc(d, wsplit[k2]);
        row[k2] = make_float2(s.x - e.y, s.y + e.x);
      }
    }
  }
  __syncthreads();
}

// Forward: real map (float offset 2*P*h + w) -> half spectrum (complex offset h*P + c).
// Caller syncs before (the map must be complete). Ends synced.
// the 2-D transforms are calls, not inlined: each gets its own register allocation, which
// measured faster than inlining them into the sweep (1.94 vs 2.17 ms per 128x128 sweep)
#define CSC_FFT2_ATTR __device__ __noinline__
// After the column FFT, column 0 holds Z = F(x_dc + i x_nyq) of two real columns:
// X_dc(k) = (Z(k) + conj Z(-k))/2 stays in column 0, X_nyq(k) = (Z(k) - conj Z(-k))/(2i) goes to
// column Wh. Pairs (k, H-k) are handled by one thread, so no other thread touches its bins.
template <class G, int NT>
CSC_D void unpack_dc_nyquist(const G& g, float2* buf) {
  const int H = g.h(), Wh = g.wh(), P = g.p();
  for (int k = threadIdx.x; k <= H / 2; k += NT) {
    const int k2 = (H - k) % H;
    const float2 a = buf[k * P], b = buf[k2 * P];
    // (a + conj b)/2 and (a - conj b)/(2i)
    const float2 dc = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
    const float2 ny = make_float2(0.5f * (a.y + b.y), 0.5f * (b.x - a.x));
    buf[k * P] = dc;
    buf[k * P + Wh] = ny;
    if (k2 != k) {
      buf[k2 * P] = make_float2(dc.x, -dc.y);
      buf[k2 * P + Wh] = make_float2(ny.x, -ny.y);
    }
  }
  __syncthreads();
}

// Inverse of the above before the inverse column FFT: column 0 <- X_dc + i X_nyq.
template <class G, int NT>
CSC_D void pack_dc_nyquist(const G& g, float2* buf) {
  const int H = g.h(), Wh = g.wh(), P = g.p();
  for (int k = threadIdx.x; k < H; k += NT) {
    const float2 dc = buf[k * P], ny = buf[k * P + Wh];
    buf[k * P] = make_float2(dc.x - ny.y, dc.y + ny.x);
  }
  __syncthreads();
}

template <class G, int NT>
CSC_FFT2_ATTR void rfft2(const G& g, float2* buf, const Twiddles tw) {
  g.template rows<false, NT>(buf, tw.row);
  split_rows_forward<G, NT>(g, buf, tw.split);
  g.template cols<false, NT>(buf, tw.col);
  unpack_dc_nyquist<G, NT>(g, buf);
}

// Inverse (unnormalised, result scaled by D = H*W): half spectrum -> real map.
template <class G, int NT>
CSC_FFT2_ATTR void irfft2(const G& g, float2* buf, const Twiddles tw) {
  pack_dc_nyquist<G, NT>(g, buf);
  g.template cols<true, NT>(buf, tw.col);
  split_rows_inverse<G, NT>(g, buf, tw.split);
  g.template rows<true, NT>(buf, tw.row);
}

template <class G, int NT>
CSC_D Twiddles stage_twiddles(const G& g, float2* smem, const float2* __restrict__ gtw) {
  const int n = twiddle_count(g);
  for (int i = threadIdx.x; i < n; i += NT) smem[i] = gtw[i];
  Twiddles t;
  t.row = smem;
  t.col = smem + g.wh();
  t.split = smem + g.wh() + g.h();
  return t;
}

}  // namespace csc
