// Double-float (two FP32 numbers, value = h + l) arithmetic for the residual of
// the mixed-precision defect correction.  GB300 executes FP64 at a small
// fraction of its FP32 rate, so the FP64-accurate residual r = b - D x is
// computed with error-free FP32 transformations instead: TwoSum (Knuth) for
// sums and FMA-based TwoProduct for products (Dekker 1971; the double-double
// algorithms of Hida, Li & Bailey 2001).  Relative accuracy about 2^-44, far
// below the 1e-10 residuals the solver needs.
#pragma once

namespace dd {

struct dfc {            // complex double-float
  float2 h, l;          // (re, im) high and low parts
};
struct df2s {           // its storage: (re_h, im_h, re_l, im_l), 16 bytes like a double2
  float4 v;
};
template <> struct StoreTraits<df2s> { typedef float T; typedef dfc C; };

// ---- real double-float primitives ---------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// Accumulation is lazy: h collects the FP32 sum exactly split by TwoSum and l
// every rounding error and low-order term, without renormalising after each
// step (h + l stays exact to ~2^-48 of the terms; |l| grows to a few ulp(h)).
// Values are renormalised once, where they are stored (stc / df_renorm).
// (h, l) += a * b for double-float a, b
__device__ __forceinline__ void df_fma(float& h, float& l, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  float s, t;
  two_sum(h, p, s, t);
  h = s;
  l += t + e;
}
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
  float s, t;
  two_sum(h, bh, s, t);
  h = s;
  l += t + bl;
}
// (h, l) -> the nearest FP32 h and the remainder l (|l| <= ulp(h) / 2)
__device__ __forceinline__ void df_renorm(float& h, float& l) {
  float s, t;
  two_sum(h, l, s, t);
  h = s;
  l = t;
}

// ---- packed pairs: two FP32 lanes in one 64-bit register --------------------------
// The f32x2 forms of add, sub, mul and fma (round to nearest on each lane) run
// the real and imaginary parts of a complex double-float through one
// instruction stream: every lane performs the same operations in the same
// order as the scalar primitives above, so the values are theirs (an exact
// zero may differ in sign where x + (-y) is written x - y).
typedef unsigned long long f2p;
__device__ __forceinline__ f2p pk(float x, float y) {
  f2p r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ f2p pk(float2 v) { return pk(v.x, v.y); }
__device__ __forceinline__ float2 upk(f2p r) {
  float x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(r));
  return make_float2(x, y);
}
__device__ __forceinline__ f2p add2(f2p a, f2p b) {
  f2p r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2p sub2(f2p a, f2p b) {
  f2p r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2p mul2(f2p a, f2p b) {
  f2p r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
  f2p r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// df_add on both lanes
__device__ __forceinline__ void df_add2(f2p& h, f2p& l, f2p bh, f2p bl) {
  const f2p s = add2(h, bh);
  const f2p bb = sub2(s, h);
  const f2p t = add2(sub2(h, sub2(s, bb)), sub2(bh, bb));
  h = s;
  l = add2(l, add2(t, bl));
}
// df_add of the negated operand on both lanes, with x + (-y) written x - y
__device__ __forceinline__ void df_sub2(f2p& h, f2p& l, f2p bh, f2p bl) {
  const f2p s = sub2(h, bh);
  const f2p bb = sub2(s, h);
  const f2p t = sub2(sub2(h, sub2(s, bb)), add2(bh, bb));
  h = s;
  l = add2(l, sub2(t, bl));
}
// df_fma on both lanes; nah = -ah, so q = -(ah bh) rounded is the negated
// product and the error terms and TwoSum follow df_fma with p = -q
__device__ __forceinline__ void df_fma2(f2p& h, f2p& l, f2p ah, f2p al, f2p nah, f2p bh, f2p bl) {
  const f2p q = mul2(nah, bh);
  f2p e = fma2(ah, bh, q);
  e = fma2(ah, bl, e);
  e = fma2(al, bh, e);
  const f2p s = sub2(h, q);
  const f2p bb = sub2(s, h);
  const f2p t = sub2(sub2(h, sub2(s, bb)), add2(q, bb));
  h = s;
  l = add2(l, add2(t, e));
}

// ---- complex helpers used by the generic stencil code -------------------------------
__device__ __forceinline__ dfc ldc(const df2s* p) {
  const float4 v = __ldg(&p->v);
  return dfc{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void stc(df2s* p, dfc v) {
  df_renorm(v.h.x, v.l.x);
  df_renorm(v.h.y, v.l.y);
  p->v = make_float4(v.h.x, v.h.y, v.l.x, v.l.y);
}
__device__ __forceinline__ void df_renorm(dfc& v) {
  df_renorm(v.h.x, v.l.x);
  df_renorm(v.h.y, v.l.y);
}
__device__ __forceinline__ void ld_pair(const df2s* p, dfc& a, dfc& b) {
  a = ldc(p);
  b = ldc(p + 1);
}
__device__ __forceinline__ void ld_pair(df2s* p, dfc& a, dfc& b) {
  const float4 x = p[0].v, y = p[1].v;
  a = dfc{make_float2(x.x, x.y), make_float2(x.z, x.w)};
  b = dfc{make_float2(y.x, y.y), make_float2(y.z, y.w)};
}
__device__ __forceinline__ void st_pair(df2s* p, dfc a, dfc b) {
  stc(p, a);
  stc(p + 1, b);
}
// (st_pair renormalises through stc)
__device__ __forceinline__ float2 split_d(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}
template <> __device__ __forceinline__ dfc cmk<dfc>(double re, double im) {
  const float2 r = split_d(re), i = split_d(im);
  return dfc{make_float2(r.x, i.x), make_float2(r.y, i.y)};
}
__device__ __forceinline__ double2 to_d2(dfc a) {
  return make_double2((double)a.h.x + (double)a.l.x, (double)a.h.y + (double)a.l.y);
}
__device__ __forceinline__ dfc cadd(dfc a, dfc b) {
  f2p h = pk(a.h), l = pk(a.l);
  df_add2(h, l, pk(b.h), pk(b.l));
  return dfc{upk(h), upk(l)};
}
__device__ __forceinline__ dfc csub(dfc a, dfc b) {
  f2p h = pk(a.h), l = pk(a.l);
  df_sub2(h, l, pk(b.h), pk(b.l));
  return dfc{upk(h), upk(l)};
}
// a + i b and a - i b
__device__ __forceinline__ dfc caddi(dfc a, dfc b) {
  df_add(a.h.x, a.l.x, -b.h.y, -b.l.y);
  df_add(a.h.y, a.l.y, b.h.x, b.l.x);
  return a;
}
__device__ __forceinline__ dfc csubi(dfc a, dfc b) {
  df_add(a.h.x, a.l.x, b.h.y, b.l.y);
  df_add(a.h.y, a.l.y, -b.h.x, -b.l.x);
  return a;
}
// acc += a b and acc += conj(a) b, as two double-float FMAs on (re, im) lane
// pairs: re += a.re b.re then -/+ a.im b.im, im += a.re b.im then +/- a.im b.re
__device__ __forceinline__ void cfma(dfc& acc, dfc a, dfc b) {
  f2p h = pk(acc.h), l = pk(acc.l);
  df_fma2(h, l, pk(a.h.x, a.h.x), pk(a.l.x, a.l.x), pk(-a.h.x, -a.h.x), pk(b.h), pk(b.l));
  df_fma2(h, l, pk(-a.h.y, a.h.y), pk(-a.l.y, a.l.y), pk(a.h.y, -a.h.y), pk(b.h.y, b.h.x), pk(b.l.y, b.l.x));
  acc = dfc{upk(h), upk(l)};
}
__device__ __forceinline__ void cfmac(dfc& acc, dfc a, dfc b) {
  f2p h = pk(acc.h), l = pk(acc.l);
  df_fma2(h, l, pk(a.h.x, a.h.x), pk(a.l.x, a.l.x), pk(-a.h.x, -a.h.x), pk(b.h), pk(b.l));
  df_fma2(h, l, pk(a.h.y, -a.h.y), pk(a.l.y, -a.l.y), pk(-a.h.y, a.h.y), pk(b.h.y, b.h.x), pk(b.l.y, b.l.x));
  acc = dfc{upk(h), upk(l)};
}

template <> struct ScalOf<dfc> { typedef float2 type; };
template <> __device__ __forceinline__ float2 mkscal<dfc>(double x) { return split_d(x); }
// a * s for a double-float real s
__device__ __forceinline__ dfc scale(dfc a, float2 s) {
  f2p h = pk(0.f, 0.f), l = pk(0.f, 0.f);
  df_fma2(h, l, pk(a.h), pk(a.l), pk(-a.h.x, -a.h.y), pk(s.x, s.x), pk(s.y, s.y));
  return dfc{upk(h), upk(l)};
}
__device__ __forceinline__ void axpy(dfc& o, float2 s, dfc v) {
  f2p h = pk(o.h), l = pk(o.l);
  df_fma2(h, l, pk(v.h), pk(v.l), pk(-v.h.x, -v.h.y), pk(s.x, s.x), pk(s.y, s.y));
  o = dfc{upk(h), upk(l)};
}
__device__ __forceinline__ float nrm2f(dfc a) { return fmaf(a.h.x, a.h.x, a.h.y * a.h.y); }

// Hermitian clover block times a double-float vector, from a double-float
// packed table: per chirality block the 6 real diagonal entries as (h, l)
// pairs (3 float4), then the 15 entries above the diagonal row by row as
// (re_h, im_h, re_l, im_l) (15 float4): 18 float4 (288 B), 36 per site.
constexpr int CLOV_HDF_F4 = 36;
__device__ __forceinline__ void clover_mul_h(const float4* __restrict__ M, dfc (&v)[12]) {
#pragma unroll
  for (int ch = 0; ch < 2; ++ch) {
    const float4* m = M + ch * 18;
    dfc w[6];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 d = __ldg(m + q);
      w[2 * q] = scale(v[ch * 6 + 2 * q], make_float2(d.x, d.y));
      w[2 * q + 1] = scale(v[ch * 6 + 2 * q + 1], make_float2(d.z, d.w));
    }
    int z = 3;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = r + 1; c < 6; ++c, ++z) {
        const float4 t = __ldg(m + z);
        const dfc e{make_float2(t.x, t.y), make_float2(t.z, t.w)};
        cfma(w[r], e, v[ch * 6 + c]);          // w_r += m v_c
        cfmac(w[c], e, v[ch * 6 + r]);         // w_c += conj(m) v_r
      }
#pragma unroll
    for (int r = 0; r < 6; ++r) v[ch * 6 + r] = w[r];
  }
}

}  // namespace dd
