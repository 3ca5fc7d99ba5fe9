// Float-float ("double-FP32") arithmetic for the D contraction of the FP64-accurate path.
//
// On B300 an FP64 operation costs 64 FP32 slots (2 DFMA vs 128 FFMA per clock and SM), and the
// FP64 stage kernel is bound by the FP64 pipe.  This path keeps the state, the fluxes and the stage
// update in FP64 but applies D in unevaluated sums of two floats, x = hi + lo (|lo| <= 2^-24 |hi|):
//   - a double is split into (hi, lo) by exponent / mantissa arithmetic on its bits (integer
//     operations, no FP64 conversion): hi keeps the leading 24 significant bits, lo the next 24
//     (rounded), so the split is exact to 2^-48 relative;
//   - a product of two such numbers is the error-free product of the high parts (Dekker's
//     two-product through an FMA) plus the two cross terms accumulated in a separate float;
//   - sums use Knuth's two-sum for the high parts and plain float sums for the low parts.
// The contraction error is about 2^-44 of sum |D||u| (FP64's is 2^-53 of it), i.e. ~1e-14
// relative per step for the configurations here, inside the 1e-12 per-step parity of the FP64
// path.  Values outside [2^-74, 2^127] in magnitude (or not finite) cannot be split into normal
// floats; a line containing one is contracted in FP64 instead, so any input stays correct.
#pragma once

#include <cuda_runtime.h>

namespace ndg {

struct ff {
  float h, l;
};

// Coefficient tables of one degree as float-float pairs (kernel parameters, constant bank).
struct BasisFF {
  float Aeh[16], Ael[16];
  float Boh[16], Bol[16];
  float Cmidh[4], Cmidl[4];
  float Dmidh[4], Dmidl[4];
};

// Split a double into hi + lo floats; false if |x| is outside [2^-74, 2^127] (zero is fine).
__device__ __forceinline__ bool ff_split(double x, float& h, float& l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const unsigned sign = (unsigned)(b >> 63) << 31;
  if (e == 0 && m == 0) {
    h = __uint_as_float(sign);
    l = 0.0f;
    return true;
  }
  if (e < 949u || e > 1150u) return false;
  // hi: same sign and exponent, the top 23 stored mantissa bits (truncation)
  h = __uint_as_float(sign | ((e - 1023u + 127u) << 23) | (unsigned)(m >> 29));
  // lo = x - hi = (remaining 29 mantissa bits) * 2^(e - 1075), rounded to 24 bits by the I2F
  const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);
  const float scale = __uint_as_float((e - 1075u + 127u) << 23);  // 2^(e - 1075), e >= 949
  const float lo = __uint2float_rn(rem) * scale;
  l = sign ? -lo : lo;
  return true;
}

// float -> double by exponent arithmetic (normal floats and zero; subnormals flush to zero).
__device__ __forceinline__ double ff_f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  const unsigned long long s = (unsigned long long)(b >> 31) << 63;
  const unsigned long long E = (unsigned long long)(e - 127u + 1023u) << 52;
  const unsigned long long M = (unsigned long long)(b & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(s | E | M));
}

__device__ __forceinline__ double ff_to_double(ff a) { return ff_f2d(a.h) + ff_f2d(a.l); }

// Knuth's two-sum: s + err == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = a + b;
  const float bb = s - a;
  err = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e += a.l + b.l;
  const float h = s + e;  // renormalise (|e| << |s| unless cancellation, then exact anyway)
  return ff{h, e - (h - s)};
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff{-b.h, -b.l}); }

// Accumulate c * x into (acc_h + acc_l): exact product of the high parts, cross terms and the
// product's rounding error into the low accumulator.
__device__ __forceinline__ void ff_fma_acc(float ch, float cl, ff x, float& acc_h, float& acc_l) {
  const float p = __fmul_rn(ch, x.h);  // rounded on its own: contracted into the sum below, the
                                       // product error pe would no longer be the sum's error
  const float pe = fmaf(ch, x.h, -p);
  float s, e;
  two_sum(acc_h, p, s, e);
  acc_h = s;
  acc_l += e + pe;
  acc_l = fmaf(ch, x.l, acc_l);
  acc_l = fmaf(cl, x.h, acc_l);
}

__device__ __forceinline__ ff ff_norm(float h, float l) {
  const float s = h + l;
  return ff{s, l - (s - h)};
}

// (scale as double, applied to a float-float value): used for the per-axis volume scale.
__device__ __forceinline__ ff ff_mul(ff a, float ch, float cl) {
  const float p = __fmul_rn(ch, a.h);
  const float pe = fmaf(ch, a.h, -p);
  const float l = fmaf(ch, a.l, fmaf(cl, a.h, pe));
  return ff_norm(p, l);
}

// out = D f along one line in float-float, by the even-odd halves of D (see contract_even_odd).
template <int N>
__device__ __forceinline__ void contract_even_odd_ff(const ff (&f)[N + 1], ff (&out)[N + 1], const BasisFF& B) {
  constexpr int n = N + 1;
  constexpr int H = n / 2;
  ff fe[H], fo[H];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    fe[m] = ff_add(f[m], f[N - m]);
    fo[m] = ff_sub(f[m], f[N - m]);
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    float eh = 0.0f, el = 0.0f, oh = 0.0f, ol = 0.0f;
#pragma unroll
    for (int m = 0; m < H; ++m) {
      ff_fma_acc(B.Aeh[i * 4 + m], B.Ael[i * 4 + m], fo[m], eh, el);
      ff_fma_acc(B.Boh[i * 4 + m], B.Bol[i * 4 + m], fe[m], oh, ol);
    }
    if (n % 2 == 1) ff_fma_acc(B.Cmidh[i], B.Cmidl[i], f[H], oh, ol);
    const ff E = ff_norm(eh, el), O = ff_norm(oh, ol);
    out[i] = ff_add(E, O);
    out[N - i] = ff_sub(E, O);
  }
  if (n % 2 == 1) {
    float mh = 0.0f, ml = 0.0f;
#pragma unroll
    for (int m = 0; m < H; ++m) ff_fma_acc(B.Dmidh[m], B.Dmidl[m], fo[m], mh, ml);
    out[H] = ff_norm(mh, ml);
  }
}

}  // namespace ndg
