// The 128 x 128 passes of f128_common.cuh with packed float32 pairs: the coding sweep's version.
//
// Same thread roles, shared-memory layout, pass order and twiddle tables as f128_common.cuh; what
// changes is how the arithmetic is issued:
//   * a complex value is a float2 (re, im) register pair, and every complex addition, subtraction and
//     multiply-add by a real constant pair is one packed instruction (fma.rn.f32x2): the butterflies
//     of the 4-, 8- and 16-point DFTs issue about half the instructions of the scalar form. A
//     multiplication by -i or +i becomes a swapped operand pair formed by two scalar subtractions;
//     twiddle products stay scalar (four fused multiply-adds);
//   * the real split pairs bin (kh, kw) with its mirror (-kh, 64 - kw), and both bins of a pair share
//     one sum, one difference and one twiddle product (w^(64 - kw) = -conj(w^kw)): for the 12 of 16
//     warps whose items are not self-paired (class c >= 1) the split costs half the scalar form.
//     The forward split's factor 1/2 is left out (the sweep stores d_hat / 2 in thread order and
//     scales lambda_hat by 2, which is exact);
//   * the twiddle tables sit in constant memory: every pass reads them at warp-uniform indices, so
//     they come through the constant cache and leave the shared-memory pipe to the spectrum.
#pragma once
#include <cuda_runtime.h>

#include "f128_common.cuh"

namespace csc {
namespace f128 {

// The tables of f128_common.cuh's build_tw in 16-byte pairs: c_twq4[8 a + i] holds q entries
// 16 a + 2 i and 16 a + 2 i + 1 (w^(a m mod 128)), c_tws4[4 k + i] holds s entries 8 k + 2 i and
// 8 k + 2 i + 1 (w^(k + 8 j)); w = exp(-2 pi i / 128). Written once per device by
// upload_f128_twiddles (sweep128.cu).
__constant__ float4 c_twq4[128];
__constant__ float4 c_tws4[32];
CSC_D void twc_split(float4 v, float2& w0, float2& w1) {
  w0 = make_float2(v.x, v.y);
  w1 = make_float2(v.z, v.w);
}
// the first 8 entries of q row a, all 8 entries of s row k, and q entries 16 a + 2 i, 16 a + 2 i + 1
CSC_D void twc_row8_q(int a, float2 (&w)[8]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) twc_split(c_twq4[8 * a + i], w[2 * i], w[2 * i + 1]);
}
CSC_D void twc_row8_s(int k, float2 (&w)[8]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) twc_split(c_tws4[4 * k + i], w[2 * i], w[2 * i + 1]);
}
CSC_D void twc_pair_q(int a, int i, float2& w0, float2& w1) { twc_split(c_twq4[8 * a + i], w0, w1); }

CSC_D float2 pk_add(float2 a, float2 b) { return __ffma2_rn(b, make_float2(1.f, 1.f), a); }
CSC_D float2 pk_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
CSC_D float2 pk_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
CSC_D float2 pk_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
CSC_D float2 pk_clamp(float2 v, float b) { return make_float2(fminf(fmaxf(v.x, -b), b), fminf(fmaxf(v.y, -b), b)); }

// 4-point DFT in place (outputs in natural order). The difference a1 - a3 is formed swapped,
// (im, re), so that t1 -+ i (a1 - a3) are two packed multiply-adds with sign pairs.
template <bool INV> CSC_D void x2_dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = pk_add(a0, a2), t1 = pk_sub(a0, a2), t2 = pk_add(a1, a3);
  const float2 ds = make_float2(a1.y - a3.y, a1.x - a3.x);
  a0 = pk_add(t0, t2);
  a2 = pk_sub(t0, t2);
  // forward: t1 - i d = (t1.re + d.im, t1.im - d.re); inverse: t1 + i d
  a1 = pk_fma(ds, INV ? make_float2(-1.f, 1.f) : make_float2(1.f, -1.f), t1);
  a3 = pk_fma(ds, INV ? make_float2(1.f, -1.f) : make_float2(-1.f, 1.f), t1);
}
// the same with output 2 returned swapped, (im, re)
template <bool INV> CSC_D void x2_dft4_s2(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = pk_add(a0, a2), t1 = pk_sub(a0, a2), t2 = pk_add(a1, a3);
  const float2 ds = make_float2(a1.y - a3.y, a1.x - a3.x);
  a0 = pk_add(t0, t2);
  a2 = make_float2(t0.y - t2.y, t0.x - t2.x);
  a1 = pk_fma(ds, INV ? make_float2(-1.f, 1.f) : make_float2(1.f, -1.f), t1);
  a3 = pk_fma(ds, INV ? make_float2(1.f, -1.f) : make_float2(-1.f, 1.f), t1);
}

// 8-point DFT in place, outputs in natural order (radix 2 x 4: two 4-point DFTs of the even and odd
// inputs, then the w8^q products fused into the output butterflies)
template <bool INV> CSC_D void x2_dft8(float2* a) {
  float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  float2 o0 = a[1], o1 = a[3], o2s = a[5], o3 = a[7];
  x2_dft4<INV>(e0, e1, e2, e3);
  x2_dft4_s2<INV>(o0, o1, o2s, o3);
  const float c = kSqrtHalf;
  // w8 o1 / c and w8^3 o3 / c: forward w8 = (1 - i)/sqrt 2, inverse its conjugate
  const float2 m1 = INV ? make_float2(o1.x - o1.y, o1.x + o1.y) : make_float2(o1.x + o1.y, o1.y - o1.x);
  const float2 m3 = INV ? make_float2(-o3.x - o3.y, o3.x - o3.y) : make_float2(o3.y - o3.x, -o3.x - o3.y);
  const float2 cp = make_float2(c, c), cm = make_float2(-c, -c);
  a[0] = pk_add(e0, o0);
  a[4] = pk_sub(e0, o0);
  a[1] = pk_fma(m1, cp, e1);
  a[5] = pk_fma(m1, cm, e1);
  // -+ i o2 from the swapped o2
  a[2] = pk_fma(o2s, INV ? make_float2(-1.f, 1.f) : make_float2(1.f, -1.f), e2);
  a[6] = pk_fma(o2s, INV ? make_float2(1.f, -1.f) : make_float2(-1.f, 1.f), e2);
  a[3] = pk_fma(m3, cp, e3);
  a[7] = pk_fma(m3, cm, e3);
}

// 16 = 4 x 4, outputs transposed exactly as dft16 of fft.cuh (out_slot<16>)
template <bool INV> CSC_D void x2_dft16(float2* a) {
  constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) x2_dft4<INV>(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
  auto rot = [](float2 v, float c, float s) {  // v * (c - i s) forward, (c + i s) inverse
    return INV ? make_float2(v.x * c - v.y * s, v.x * s + v.y * c)
               : make_float2(v.x * c + v.y * s, v.y * c - v.x * s);
  };
  a[5] = rot(a[5], c1, s1);
  a[6] = rot(a[6], kSqrtHalf, kSqrtHalf);
  a[7] = rot(a[7], s1, c1);
  a[9] = rot(a[9], kSqrtHalf, kSqrtHalf);
  a[10] = mul_mi<INV>(a[10]);
  a[11] = rot(a[11], -kSqrtHalf, kSqrtHalf);
  a[13] = rot(a[13], s1, c1);
  a[14] = rot(a[14], -kSqrtHalf, kSqrtHalf);
  a[15] = rot(a[15], -c1, -s1);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) x2_dft4<INV>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
}

// forward split of one bin without the factor 1/2: 2 X = (Za + conj Zb) - i w (Za - conj Zb)
CSC_D float2 split_fwd2(float2 ya, float2 yb, float2 w) {
  const float2 s = make_float2(ya.x + yb.x, ya.y - yb.y);
  const float2 d = make_float2(ya.x - yb.x, ya.y + yb.y);
  const float2 wd = cmul(w, d);
  return make_float2(s.x + wd.y, s.y - wd.x);
}

// inverse split of the thread's bins (get(slot) -> X) and the first inverse row pass, stored over
// the item's cells. Threads of class c >= 1 (items never self-paired) split bin pairs (A_j, B_{7-j})
// with one shared sum, difference and twiddle product:
//   s = Xa + conj Xb, d = Xa - conj Xb, f' = i conj(w) d:  Za = s + f',  Zb = conj(s - f').
template <class GET>
CSC_D void inv_rows1_x2(float2* buf, const Tw& T, const Roles& R, GET get) {
  const Items& it = R.it;
  float2 za[8], zb[8], wa[8], wb[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    za[j] = get(j);
    zb[j] = get(8 + j);
  }
  twc_row8_s(it.kA, wa);
  if (R.c != 0) {
    // pairs (A_j, B_{7-j}), j < 4, and (A_{7-j}, B_j), split in place
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int ja = h < 4 ? h : 11 - h;   // 0, 1, 2, 3, 7, 6, 5, 4
      const float2 xa = za[ja], xb = zb[7 - ja], w = wa[ja];
      const float2 sm = pk_fma(xb, make_float2(1.f, -1.f), xa);
      const float2 d = pk_fma(xb, make_float2(-1.f, 1.f), xa);
      const float2 fp = make_float2(fmaf(w.y, d.x, -w.x * d.y), fmaf(w.x, d.x, w.y * d.y));
      za[ja] = pk_add(sm, fp);
      const float2 q = pk_sub(sm, fp);
      zb[7 - ja] = make_float2(q.x, -q.y);
    }
  } else {
    float2 na = make_float2(0.f, 0.f), nb = make_float2(0.f, 0.f);
    if (R.nyq) {
      na = get(16);
      nb = get(17);
    }
    twc_row8_s(it.kB, wb);
    const bool sf = it.self, cls0 = R.cls0;
    float2 xa[8], xb[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      xa[j] = za[j];
      xb[j] = zb[j];
    }
#define CSC_F128X2_UNSPLIT(J)                                                                     \
  {                                                                                               \
    const float2 pa = sf ? partner<J>(xa, na, cls0) : partner<J>(xb, nb, cls0);                   \
    const float2 pb = sf ? partner<J>(xb, nb, cls0) : partner<J>(xa, na, cls0);                   \
    za[J] = split_inv(xa[J], pa, wa[J]);                                                          \
    zb[J] = split_inv(xb[J], pb, wb[J]);                                                          \
  }
    CSC_F128X2_UNSPLIT(0) CSC_F128X2_UNSPLIT(1) CSC_F128X2_UNSPLIT(2) CSC_F128X2_UNSPLIT(3)
    CSC_F128X2_UNSPLIT(4) CSC_F128X2_UNSPLIT(5) CSC_F128X2_UNSPLIT(6) CSC_F128X2_UNSPLIT(7)
#undef CSC_F128X2_UNSPLIT
  }
  x2_dft8<true>(za);
  x2_dft8<true>(zb);
  float2* ra = buf + it.rowA * P + 8 * it.kA;
  float2* rb = buf + it.rowB * P + 8 * it.kB;
  twc_row8_q(2 * it.kA, wa);
  twc_row8_q(2 * it.kB, wb);
  ra[0] = za[0];
  rb[0] = zb[0];
#pragma unroll
  for (int q = 1; q < 8; ++q) {
    ra[q] = cmulc(za[q], wa[q]);
    rb[q] = cmulc(zb[q], wb[q]);
  }
}

// second inverse row pass: row r, classes c and c + 4 -> canonical columns m
CSC_D void inv_rows2_x2(float2* buf, const Roles& R) {
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    const int k1 = R.c + 4 * h2;
    float2* row = buf + R.r * P;
    float2 y[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = row[8 * q + k1];
    x2_dft8<true>(y);
#pragma unroll
    for (int q = 0; q < 8; ++q) row[k1 + 8 * q] = y[q];
  }
}

// first inverse column pass: column wc, kh = 16 n1 + n2 for n2 = g, g + 8
CSC_D void inv_cols1_x2(float2* buf, const Tw& T, const Roles& R) {
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    const int n2 = R.g + 8 * h2;
    float2 y[8], w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = buf[(16 * q + n2) * P + R.wc];
    twc_row8_q(n2, w);
    x2_dft8<true>(y);
    buf[n2 * P + R.wc] = y[0];
#pragma unroll
    for (int q = 1; q < 8; ++q) buf[(16 * q + n2) * P + R.wc] = cmulc(y[q], w[q]);
  }
}

// second inverse column pass: afterwards zc[out_slot<16>(j)] is the map at rows g + 8 j of column wc
CSC_D void inv_cols2_x2(const float2* buf, const Roles& R, float2 (&zc)[16]) {
#pragma unroll
  for (int q = 0; q < 16; ++q) zc[q] = buf[(16 * R.g + q) * P + R.wc];
  x2_dft16<true>(zc);
}

// first forward column pass from zc[j] = the map at rows 8 j + g (natural order)
CSC_D void fwd_cols1_x2(float2* buf, const Tw& T, const Roles& R, float2 (&zc)[16]) {
  x2_dft16<false>(zc);
  buf[(16 * R.g) * P + R.wc] = zc[out_slot<16>(0)];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float2 w0, w1;
    twc_pair_q(R.g, i, w0, w1);
    if (i > 0) buf[(16 * R.g + 2 * i) * P + R.wc] = cmul(zc[out_slot<16>(2 * i)], w0);
    buf[(16 * R.g + 2 * i + 1) * P + R.wc] = cmul(zc[out_slot<16>(2 * i + 1)], w1);
  }
}

// second forward column pass: k1 = g, g + 8 -> canonical rows kh = k1 + 16 k2
CSC_D void fwd_cols2_x2(float2* buf, const Roles& R) {
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    const int k1 = R.g + 8 * h2;
    float2 y[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = buf[(16 * q + k1) * P + R.wc];
    x2_dft8<false>(y);
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[(k1 + 16 * q) * P + R.wc] = y[q];
  }
}

// first forward row pass: row r, n2 = c, c + 4; twiddle w64^(n2 k1)
CSC_D void fwd_rows1_x2(float2* buf, const Tw& T, const Roles& R) {
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    const int n2 = R.c + 4 * h2;
    float2* row = buf + R.r * P;
    float2 y[8], w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = row[8 * q + n2];
    twc_row8_q(2 * n2, w);
    x2_dft8<false>(y);
    row[n2] = y[0];
#pragma unroll
    for (int q = 1; q < 8; ++q) row[8 * q + n2] = cmul(y[q], w[q]);
  }
}

// second forward row pass of items A and B and the split without the factor 1/2:
// put(slot, V, conj) receives 2 X of the thread's bin `slot` as V (conj false) or as conj(V) (conj
// true). Class c >= 1 pairs (A_j, B_{7-j}) share s = Ya + conj Yb, d = Ya - conj Yb and
// e' = -i w d:  2 Xa = s + e',  2 Xb = conj(s - e').
template <class PUT>
CSC_D void fwd_rows2_split_x2(const float2* buf, const Tw& T, const Roles& R, PUT put) {
  const Items& it = R.it;
  float2 ya[8], yb[8];
  const float2* ra = buf + it.rowA * P + 8 * it.kA;
  const float2* rb = buf + it.rowB * P + 8 * it.kB;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    ya[q] = ra[q];
    yb[q] = rb[q];
  }
  x2_dft8<false>(ya);
  x2_dft8<false>(yb);
  float2 wa[8];
  twc_row8_s(it.kA, wa);
  if (R.c != 0) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float2 a = ya[j], b = yb[7 - j], w = wa[j];
      const float2 s = pk_fma(b, make_float2(1.f, -1.f), a);
      const float2 d = pk_fma(b, make_float2(-1.f, 1.f), a);
      const float2 ep = make_float2(fmaf(w.x, d.y, w.y * d.x), fmaf(w.y, d.y, -w.x * d.x));
      put(j, pk_add(s, ep), false);
      put(15 - j, pk_sub(s, ep), true);
    }
    return;
  }
  float2 wb[8];
  twc_row8_s(it.kB, wb);
  const bool sf = it.self, cls0 = R.cls0;
#define CSC_F128X2_SPLIT(J)                                                                       \
  {                                                                                               \
    const float2 pa = sf ? partner_y<J>(ya, cls0) : partner_y<J>(yb, cls0);                       \
    const float2 pb = sf ? partner_y<J>(yb, cls0) : partner_y<J>(ya, cls0);                       \
    put(J, split_fwd2(ya[J], pa, wa[J]), false);                                                  \
    put(8 + J, split_fwd2(yb[J], pb, wb[J]), false);                                              \
  }
  CSC_F128X2_SPLIT(0) CSC_F128X2_SPLIT(1) CSC_F128X2_SPLIT(2) CSC_F128X2_SPLIT(3)
  CSC_F128X2_SPLIT(4) CSC_F128X2_SPLIT(5) CSC_F128X2_SPLIT(6) CSC_F128X2_SPLIT(7)
#undef CSC_F128X2_SPLIT
  if (R.nyq) {
    const float2 pa = sf ? ya[0] : yb[0];
    const float2 pb = sf ? yb[0] : ya[0];
    const float2 m1w = make_float2(-1.f, 0.f);
    put(16, split_fwd2(ya[0], pa, m1w), false);
    put(17, split_fwd2(yb[0], pb, m1w), false);
  }
}

}  // namespace f128
}  // namespace csc
