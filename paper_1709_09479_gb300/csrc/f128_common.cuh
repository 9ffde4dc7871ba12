// The 128 x 128 real 2-D FFT of the fused sweeps, as per-thread passes over one map in shared memory.
//
// Layout and roles (512 threads):
//   * the spatial side is the column transform. A real map is read as 64 complex columns
//     z[h][m] = x[h][2m] + i x[h][2m+1]; thread (m = t & 63, g = t >> 6) holds the 16 rows
//     h = g + 8 j of column m (the last inverse column pass leaves w exactly there, and the first
//     forward column pass starts from there);
//   * the frequency side is the 64-point row FFT of each row of Z followed by the real split, which
//     pairs bin (kh, kw) with (-kh, 64 - kw): thread t owns two (row, residue class of kw mod 8)
//     items A and B (see items_of), i.e. 16 bins, plus the two Nyquist bins (kw = 64) of its rows
//     when t < 64. Slot s of thread t: s < 8 is value s of item A (kw = class + 8 s), 8 <= s < 16
//     value s - 8 of item B, 16 and 17 the Nyquist bins of A and B. Slot data of all threads are
//     stored thread-major: slot s at s * 512 + t (s < 16), at 8192 + (s - 16) * 64 + t (s >= 16);
//     canonical_of maps such a position to the half-spectrum index kh * 65 + kw;
//   * 128 = 16 x 8 (columns) and 64 = 8 x 8 (rows) Cooley-Tukey passes; every pass writes its outputs
//     over the shared-memory cells it read, so the callers need a block barrier between passes only.
// Forward transforms are unnormalised with exp(-2 pi i / n); the inverse is unnormalised (result
// scaled by 128 * 128). Twiddles w^m = exp(-2 pi i m / 128) come from two shared-memory tables laid
// out so that a pass reads the two twiddles of consecutive butterfly outputs in one 16-byte load.
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"

namespace csc {
namespace f128 {

constexpr int H = 128, W = 128, D = H * W, P = 65, NT = 512;
constexpr int OM = H * (W / 2 + 1);   // 8320 half-spectrum bins
constexpr int NQ = 64;                 // threads holding Nyquist bins
static_assert(16 * NT + 2 * NQ == OM, "slot layout covers the half spectrum");

// The two (row, residue class of kw mod 8) items of thread t in the row/split phase. Item B is
// the split partner of item A (row -kh, class -k mod 8), except for the four classes that are
// their own partners ((0|64, 0|4)), which threads r = 0 and r = 64 of c = 0 hold two of each.
struct Items {
  int rowA, rowB, kA, kB;
  bool self;
};
CSC_HD Items items_of(int t) {
  const int r = t & 127, c = t >> 7;
  Items it;
  if (c == 0) {
    const bool sp = (r & 63) == 0;
    it.kA = it.kB = (r < 64) ? 0 : 4;
    it.rowA = sp ? 0 : r;
    it.rowB = sp ? 64 : 128 - r;
    it.self = sp;
  } else {
    it.kA = c;
    it.kB = 8 - c;
    it.rowA = r;
    it.rowB = (128 - r) & 127;
    it.self = false;
  }
  return it;
}

// thread-major position of slot s of thread t
CSC_HD int slot_pos(int s, int t) { return s < 16 ? s * NT + t : 16 * NT + (s - 16) * NQ + t; }

// canonical half-spectrum index (kh * 65 + kw) of thread-major position p
CSC_HD int canonical_of(int p) {
  if (p < 16 * NT) {
    const int s = p / NT, t = p % NT;
    const Items it = items_of(t);
    const int j = s & 7;
    return (s < 8) ? it.rowA * 65 + it.kA + 8 * j : it.rowB * 65 + it.kB + 8 * j;
  }
  const int e = (p - 16 * NT) / NQ, t = (p - 16 * NT) % NQ;
  const Items it = items_of(t);
  return (e == 0 ? it.rowA : it.rowB) * 65 + 64;
}

struct Roles {
  int wc, g;   // column phase: column m = wc, rows g + 8 j
  int r, c;    // first row pass / second inverse row pass: row r, classes c and c + 4
  Items it;    // forward split / inverse split items
  bool nyq, cls0;
};
__device__ __forceinline__ Roles roles_of(int t) {
  Roles R;
  R.wc = t & 63;
  R.g = t >> 6;
  R.r = t & 127;
  R.c = t >> 7;
  R.it = items_of(t);
  R.nyq = t < NQ;
  R.cls0 = R.it.kA == 0;
  return R;
}

// twiddle tables: q[16 a + m] = w^(a m mod 128) (a, m < 16: the pass twiddles), s[8 k + j] = w^(k + 8 j)
// (k, j < 8: the real split of residue class k)
constexpr int kTwQ = 256, kTwS = 64, kTwEntries = kTwQ + kTwS;
struct Tw {
  const float2* q;
  const float2* s;
};
// fill the tables at tab (kTwEntries float2, 16-byte aligned) from w^m, m < 128, in global memory
template <int NTH>
__device__ __forceinline__ Tw build_tw(float2* tab, const float2* __restrict__ w128) {
  for (int i = threadIdx.x; i < kTwEntries; i += NTH) {
    const int m = i < kTwQ ? ((i >> 4) * (i & 15)) & 127 : ((i - kTwQ) >> 3) + 8 * ((i - kTwQ) & 7);
    tab[i] = w128[m];
  }
  return Tw{tab, tab + kTwQ};
}
// entries 2 i and 2 i + 1 of a table row
__device__ __forceinline__ void tw_pair(const float2* row, int i, float2& w0, float2& w1) {
  const float4 v = reinterpret_cast<const float4*>(row)[i];
  w0 = make_float2(v.x, v.y);
  w1 = make_float2(v.z, v.w);
}
// the 8 entries of a table row into registers (four 16-byte loads)
__device__ __forceinline__ void tw_row8(const float2* row, float2 (&w)[8]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) tw_pair(row, i, w[2 * i], w[2 * i + 1]);
}

__device__ __forceinline__ float clampb(float v, float b) { return fminf(fmaxf(v, -b), b); }

// pull `bytes` of the next map into L2 while this one is transformed
__device__ __forceinline__ void prefetch_l2_f128(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// forward split of one bin: X = (Za + conj Zb)/2 - i w (Za - conj Zb)/2
__device__ __forceinline__ float2 split_fwd(float2 ya, float2 yb, float2 w) {
  const float2 s = make_float2(ya.x + yb.x, ya.y - yb.y);
  const float2 d = make_float2(ya.x - yb.x, ya.y + yb.y);
  const float2 wd = cmul(w, d);
  return make_float2(0.5f * (s.x + wd.y), 0.5f * (s.y - wd.x));
}
// inverse split (unnormalised): Z = (Xa + conj Xb) + i conj(w) (Xa - conj Xb)
__device__ __forceinline__ float2 split_inv(float2 xa, float2 xb, float2 w) {
  const float2 s = make_float2(xa.x + xb.x, xa.y - xb.y);
  const float2 d = make_float2(xa.x - xb.x, xa.y + xb.y);
  const float2 e = cmulc(d, w);
  return make_float2(s.x - e.y, s.y + e.x);
}

// partner value of value j of an item of class k: the bin (-kh, 64 - kw) in the partner item
// (class 0: j = 0 pairs with the partner's Nyquist bin, j > 0 with value 8 - j; other classes
// with value 7 - j)
template <int J>
__device__ __forceinline__ float2 partner(const float2 (&p)[8], float2 pnyq, bool cls0) {
  return cls0 ? (J == 0 ? pnyq : p[(8 - J) & 7]) : p[7 - J];
}
// the partner's Y value for the forward split (Y is periodic in kw with period 64)
template <int J>
__device__ __forceinline__ float2 partner_y(const float2 (&p)[8], bool cls0) {
  return cls0 ? p[(8 - J) & 7] : p[7 - J];
}

// inverse split of the thread's bins (get(slot) -> X) and the first inverse row pass (8-point over
// kw = class + 8 n1, twiddle conj w64^(class k1)), stored over the item's cells
template <class GET>
__device__ __forceinline__ void inv_rows1(float2* buf, const Tw& T, const Roles& R, GET get) {
  const Items& it = R.it;
  float2 xa[8], xb[8], na = make_float2(0.f, 0.f), nb = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    xa[j] = get(j);
    xb[j] = get(8 + j);
  }
  if (R.nyq) {
    na = get(16);
    nb = get(17);
  }
  float2 za[8], zb[8], wa[8], wb[8];
  tw_row8(T.s + 8 * it.kA, wa);
  tw_row8(T.s + 8 * it.kB, wb);
  const bool sf = it.self, cls0 = R.cls0;
#define CSC_F128_UNSPLIT(J)                                                                       \
  {                                                                                               \
    const float2 pa = sf ? partner<J>(xa, na, cls0) : partner<J>(xb, nb, cls0);                   \
    const float2 pb = sf ? partner<J>(xb, nb, cls0) : partner<J>(xa, na, cls0);                   \
    za[J] = split_inv(xa[J], pa, wa[J]);                                                          \
    zb[J] = split_inv(xb[J], pb, wb[J]);                                                          \
  }
  CSC_F128_UNSPLIT(0) CSC_F128_UNSPLIT(1) CSC_F128_UNSPLIT(2) CSC_F128_UNSPLIT(3)
  CSC_F128_UNSPLIT(4) CSC_F128_UNSPLIT(5) CSC_F128_UNSPLIT(6) CSC_F128_UNSPLIT(7)
#undef CSC_F128_UNSPLIT
  dft8<true>(za);
  dft8<true>(zb);
  float2* ra = buf + it.rowA * P + 8 * it.kA;
  float2* rb = buf + it.rowB * P + 8 * it.kB;
  tw_row8(T.q + 16 * (2 * it.kA), wa);
  tw_row8(T.q + 16 * (2 * it.kB), wb);
  ra[0] = za[0];
  rb[0] = zb[0];
#pragma unroll
  for (int q = 1; q < 8; ++q) {
    ra[q] = cmulc(za[q], wa[q]);
    rb[q] = cmulc(zb[q], wb[q]);
  }
}

// second inverse row pass: row r, classes c and c + 4 -> canonical columns m
__device__ __forceinline__ void inv_rows2(float2* buf, const Roles& R) {
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    const int k1 = R.c + 4 * h2;
    float2* row = buf + R.r * P;
    float2 y[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = row[8 * q + k1];
    dft8<true>(y);
#pragma unroll
    for (int q = 0; q < 8; ++q) row[k1 + 8 * q] = y[q];
  }
}

// first inverse column pass: column wc, kh = 16 n1 + n2 for n2 = g, g + 8
__device__ __forceinline__ void inv_cols1(float2* buf, const Tw& T, const Roles& R) {
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    const int n2 = R.g + 8 * h2;
    float2 y[8], w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = buf[(16 * q + n2) * P + R.wc];
    tw_row8(T.q + 16 * n2, w);
    dft8<true>(y);
    buf[n2 * P + R.wc] = y[0];
#pragma unroll
    for (int q = 1; q < 8; ++q) buf[(16 * q + n2) * P + R.wc] = cmulc(y[q], w[q]);
  }
}

// second inverse column pass: afterwards zc[out_slot<16>(j)] is the map at rows g + 8 j of column wc
__device__ __forceinline__ void inv_cols2(const float2* buf, const Roles& R, float2 (&zc)[16]) {
#pragma unroll
  for (int q = 0; q < 16; ++q) zc[q] = buf[(16 * R.g + q) * P + R.wc];
  dft16<true>(zc);
}

// first forward column pass from zc[j] = the map at rows 8 j + g (natural order): 16-point, twiddle
// w128^(g k1), stored over the cells the second inverse column pass reads
__device__ __forceinline__ void fwd_cols1(float2* buf, const Tw& T, const Roles& R, float2 (&zc)[16]) {
  dft16<false>(zc);
  buf[(16 * R.g) * P + R.wc] = zc[out_slot<16>(0)];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float2 w0, w1;
    tw_pair(T.q + 16 * R.g, i, w0, w1);
    if (i > 0) buf[(16 * R.g + 2 * i) * P + R.wc] = cmul(zc[out_slot<16>(2 * i)], w0);
    buf[(16 * R.g + 2 * i + 1) * P + R.wc] = cmul(zc[out_slot<16>(2 * i + 1)], w1);
  }
}

// second forward column pass: k1 = g, g + 8 -> canonical rows kh = k1 + 16 k2
__device__ __forceinline__ void fwd_cols2(float2* buf, const Roles& R) {
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    const int k1 = R.g + 8 * h2;
    float2 y[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = buf[(16 * q + k1) * P + R.wc];
    dft8<false>(y);
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[(k1 + 16 * q) * P + R.wc] = y[q];
  }
}

// first forward row pass: row r, n2 = c, c + 4; twiddle w64^(n2 k1)
__device__ __forceinline__ void fwd_rows1(float2* buf, const Tw& T, const Roles& R) {
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    const int n2 = R.c + 4 * h2;
    float2* row = buf + R.r * P;
    float2 y[8], w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = row[8 * q + n2];
    tw_row8(T.q + 16 * (2 * n2), w);
    dft8<false>(y);
    row[n2] = y[0];
#pragma unroll
    for (int q = 1; q < 8; ++q) row[8 * q + n2] = cmul(y[q], w[q]);
  }
}

// second forward row pass of items A and B and the split: put(slot, X) for each of the thread's bins
template <class PUT>
__device__ __forceinline__ void fwd_rows2_split(const float2* buf, const Tw& T, const Roles& R, PUT put) {
  const Items& it = R.it;
  float2 ya[8], yb[8];
  const float2* ra = buf + it.rowA * P + 8 * it.kA;
  const float2* rb = buf + it.rowB * P + 8 * it.kB;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    ya[q] = ra[q];
    yb[q] = rb[q];
  }
  dft8<false>(ya);
  dft8<false>(yb);
  float2 wa[8], wb[8];
  tw_row8(T.s + 8 * it.kA, wa);
  tw_row8(T.s + 8 * it.kB, wb);
  const bool sf = it.self, cls0 = R.cls0;
#define CSC_F128_SPLIT(J)                                                                         \
  {                                                                                               \
    const float2 pa = sf ? partner_y<J>(ya, cls0) : partner_y<J>(yb, cls0);                       \
    const float2 pb = sf ? partner_y<J>(yb, cls0) : partner_y<J>(ya, cls0);                       \
    put(J, split_fwd(ya[J], pa, wa[J]));                                                          \
    put(8 + J, split_fwd(yb[J], pb, wb[J]));                                                      \
  }
  CSC_F128_SPLIT(0) CSC_F128_SPLIT(1) CSC_F128_SPLIT(2) CSC_F128_SPLIT(3)
  CSC_F128_SPLIT(4) CSC_F128_SPLIT(5) CSC_F128_SPLIT(6) CSC_F128_SPLIT(7)
#undef CSC_F128_SPLIT
  if (R.nyq) {
    // kw = 64 (w^64 = -1) of both rows, from their kw = 0 values
    const float2 pa = sf ? ya[0] : yb[0];
    const float2 pb = sf ? yb[0] : ya[0];
    const float2 m1w = make_float2(-1.f, 0.f);
    put(16, split_fwd(ya[0], pa, m1w));
    put(17, split_fwd(yb[0], pb, m1w));
  }
}

}  // namespace f128
}  // namespace csc
