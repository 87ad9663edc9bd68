// Multi-limb integer complex arithmetic for the evaluation kernel.
//
// GB300's FP64 pipe issues one warp instruction per 64 clocks per SM
// sub-partition, 30 to 60 times less than its integer multiply-add pipe.  The
// double double and quad double products that dominate evaluation are
// therefore computed here on the integer pipe, with the same accuracy contract
// (error a small multiple of 2^(-53 L) times the sum of the moduli of the
// terms):
//
//   * a floating complex number fz<W> holds re and im as W signed limbs of
//     radix 2^29 sharing one binary exponent: value = sum_k d_k 2^(29 k + f);
//     limbs 0..W-2 lie in [0, 2^29), the top limb is signed;
//   * a product of two fz<W> accumulates the 32x32 -> 64-bit limb products
//     column by column in 64-bit integers (columns below W-2 are dropped: they
//     are below the result's last limb), propagates carries, and keeps the W
//     limbs from the highest nonzero column down -- at least 29 (W - 1) + 1
//     significant bits, and the magnitude of a complex product never cancels;
//   * sums are exact integer additions in a fixed-point frame chosen per
//     polynomial and point from a rigorous bound on the terms (fixed<WA>), so
//     accumulation needs neither alignment nor normalisation;
//   * conversions from and to L-limb doubles are exact up to the last limb.
//
// Everything is host+device so the host can test the same code.
#pragma once
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define HT_HD __host__ __device__ __forceinline__
#else
#define HT_HD inline
#endif

namespace ht {
namespace mpi {

constexpr int RB = 29;
constexpr int32_t MASK = (1 << RB) - 1;

template <int W>
struct fz {
  int32_t f;  // binary exponent of limb 0's lowest bit
  int32_t r[W], i[W];
};

// fz<W> padded to a multiple of 16 bytes and aligned to 16, for scratch kept in
// local memory (the forward products of the sweep): it moves in 128-bit words.
template <int W>
struct alignas(16) fzs {
  static constexpr int NW = (2 * W + 1 + 3) / 4 * 4;
  int32_t w[NW];
  HT_HD fzs() {}
  HT_HD fzs(const fz<W>& z) {
    w[0] = z.f;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      w[1 + k] = z.r[k];
      w[1 + W + k] = z.i[k];
    }
#pragma unroll
    for (int k = 2 * W + 1; k < NW; ++k) w[k] = 0;
  }
  HT_HD operator fz<W>() const {
    fz<W> z;
    z.f = w[0];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      z.r[k] = w[1 + k];
      z.i[k] = w[1 + W + k];
    }
    return z;
  }
};

// Bit length of v (0 for 0): one count-leading-zeros instruction.
HT_HD int bitlen32(uint32_t v) {
#if defined(__CUDA_ARCH__)
  return 32 - __clz((int)v);
#else
  return v ? 32 - __builtin_clz(v) : 0;
#endif
}
HT_HD int bitlen64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return 64 - __clzll((long long)v);
#else
  return v ? 64 - __builtin_clzll(v) : 0;
#endif
}

HT_HD int64_t dbits(double d) {
  int64_t b;
  std::memcpy(&b, &d, 8);
  return b;
}
HT_HD double bitsd(int64_t b) {
  double d;
  std::memcpy(&d, &b, 8);
  return d;
}
// Decompose a finite double into (signed 53-bit integer m, exponent q): d = m 2^q.
// Zero gives m = 0.  (Subnormals are handled exactly as well.)
HT_HD void decompose(double d, int64_t& m, int& q) {
  const int64_t b = dbits(d);
  const int ex = (int)((b >> 52) & 0x7ff);
  int64_t mant = b & ((1LL << 52) - 1);
  if (ex == 0) {
    q = -1074;
  } else {
    mant |= (1LL << 52);
    q = ex - 1075;
  }
  m = (b < 0) ? -mant : mant;
}
// floor(log2 |d|) of a nonzero double (normals; subnormals treated as 2^-1023)
HT_HD int ilog2(double d) {
  const int ex = (int)((dbits(d) >> 52) & 0x7ff);
  return ex == 0 ? -1023 : ex - 1023;
}

// Add the signed integer m * 2^q into column sums acc[0..N) whose column k has
// weight 2^(29 k + f); bits below column 0 are dropped.  |m| < 2^53.
template <int N>
HT_HD void add_scaled(int64_t* acc, int64_t m, int q, int f) {
  if (m == 0) return;
  const bool neg = m < 0;
  uint64_t a = (uint64_t)(neg ? -m : m);
  int s = q - f;  // bit position of m's lowest bit in the frame
  if (s < 0) {
    if (-s >= 64) return;
    a >>= -s;
    s = 0;
  }
  int k = s / RB, r = s % RB;
  // a (< 2^53) shifted left by r (< 29) spans up to 82 bits: split in 29-bit pieces
  uint64_t lo = a & (uint64_t)MASK;      // bits 0..28
  uint64_t hi = a >> RB;                 // bits 29..52 (< 2^24)
  uint64_t p0 = lo << r;                 // < 2^57
  uint64_t p1 = hi << r;                 // < 2^52
  int64_t c0 = (int64_t)(p0 & MASK), c1 = (int64_t)((p0 >> RB) + (p1 & MASK)), c2 = (int64_t)(p1 >> RB);
  if (neg) {
    c0 = -c0;
    c1 = -c1;
    c2 = -c2;
  }
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (j == k) acc[j] += c0;
    if (j == k + 1) acc[j] += c1;
    if (j == k + 2) acc[j] += c2;
  }
}

// Carry-propagate column sums into limbs: limbs 0..N-2 in [0, 2^29), the top
// limb signed (it absorbs the final carry).
template <int N>
HT_HD void carry(int64_t* acc) {
#pragma unroll
  for (int j = 0; j + 1 < N; ++j) {
    const int64_t c = acc[j] >> RB;  // floor division (arithmetic shift)
    acc[j] -= c << RB;
    acc[j + 1] += c;
  }
}

// From L doubles per component (unevaluated sums; limb 0 leading).  The frame
// puts the leading bit of the larger component at bit 27 of the top limb.
template <int W, int L>
HT_HD fz<W> from_doubles(const double* re, const double* im) {
  fz<W> z;
  const double r0 = re[0], i0 = im[0];
  int e;
  if (r0 == 0.0 && i0 == 0.0) {
    e = 0;
  } else if (r0 == 0.0) {
    e = ilog2(i0);
  } else if (i0 == 0.0) {
    e = ilog2(r0);
  } else {
    const int a = ilog2(r0), b = ilog2(i0);
    e = a > b ? a : b;
  }
  z.f = e - 27 - RB * (W - 1);
  int64_t ar[W], ai[W];
#pragma unroll
  for (int k = 0; k < W; ++k) ar[k] = ai[k] = 0;
#pragma unroll
  for (int l = 0; l < L; ++l) {
    int64_t m;
    int q;
    decompose(re[l], m, q);
    add_scaled<W>(ar, m, q, z.f);
    decompose(im[l], m, q);
    add_scaled<W>(ai, m, q, z.f);
  }
  carry<W>(ar);
  carry<W>(ai);
#pragma unroll
  for (int k = 0; k < W; ++k) {
    z.r[k] = (int32_t)ar[k];
    z.i[k] = (int32_t)ai[k];
  }
  return z;
}

// Keep the top limbs below 2^28 in magnitude (the invariant from_doubles
// sets up): a right shift of both limb strings by 1 or 2 bits when the top
// limb of either component grew past it.  With both operands' top limbs below
// 2^28 a product's top limb stays below 2^29, so column sums never overflow
// and every consumer (products, shifts into fixed-point frames) may treat the
// top limb as a 29-bit signed value.
template <int W>
HT_HD void normalize_top(fz<W>& z) {
  const int32_t tr = z.r[W - 1] < 0 ? -z.r[W - 1] : z.r[W - 1];
  const int32_t ti = z.i[W - 1] < 0 ? -z.i[W - 1] : z.i[W - 1];
  const int32_t t = tr > ti ? tr : ti;
  const int s = t >= (1 << 29) ? 2 : (t >= (1 << 28) ? 1 : 0);
  if (s == 0) return;
#pragma unroll
  for (int k = 0; k < W - 1; ++k) {
    z.r[k] = (int32_t)((((uint32_t)z.r[k] >> s) | ((uint32_t)z.r[k + 1] << (RB - s))) & (uint32_t)MASK);
    z.i[k] = (int32_t)((((uint32_t)z.i[k] >> s) | ((uint32_t)z.i[k + 1] << (RB - s))) & (uint32_t)MASK);
  }
  z.r[W - 1] >>= s;
  z.i[W - 1] >>= s;
  z.f += s;
}

// Complex product.  Columns W-2 .. 2W-1 of the exact limb product (the lower
// ones only feed a carry below the result's last limb and are dropped).
template <int W>
HT_HD fz<W> mul(const fz<W>& a, const fz<W>& b) {
  constexpr int C0 = W - 2 > 0 ? W - 2 : 0;  // lowest column kept
  constexpr int NC = 2 * W - C0;             // columns C0 .. 2W-1
  // Three real limb products per column (Gauss): re = ar br - ai bi,
  // im = (ar + ai)(br + bi) - ar br - ai bi.  The operand sums have limbs
  // below 2^30, so a column of at most W products stays below 2^63; the
  // columns are summed modulo 2^64 (unsigned) and the exact column values,
  // which fit in int64, come out of the subtraction -- the same integers as
  // the four-product form.
  int32_t sa[W], sb[W];
#pragma unroll
  for (int x = 0; x < W; ++x) {
    sa[x] = a.r[x] + a.i[x];
    sb[x] = b.r[x] + b.i[x];
  }
  uint64_t c1[NC], c2[NC], c3[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) c1[c] = c2[c] = c3[c] = 0;
#pragma unroll
  for (int x = 0; x < W; ++x)
#pragma unroll
    for (int y = 0; y < W; ++y) {
      if (x + y < C0) continue;
      const int c = x + y - C0;
      c1[c] += (uint64_t)((int64_t)a.r[x] * b.r[y]);
      c2[c] += (uint64_t)((int64_t)a.i[x] * b.i[y]);
      c3[c] += (uint64_t)((int64_t)sa[x] * sb[y]);
    }
  int64_t cr[NC], ci[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    cr[c] = (int64_t)(c1[c] - c2[c]);
    ci[c] = (int64_t)(c3[c] - c1[c] - c2[c]);
  }
  carry<NC>(cr);
  carry<NC>(ci);
  // window: columns [W-1, 2W-2] if the top column is only a sign, else [W, 2W-1]
  const int64_t tr = cr[NC - 1], ti = ci[NC - 1];
  const bool high = !((tr == 0 || tr == -1) && (ti == 0 || ti == -1));
  fz<W> z;
  if (high) {
    z.f = a.f + b.f + RB * W;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      z.r[k] = (int32_t)cr[k + W - C0];
      z.i[k] = (int32_t)ci[k + W - C0];
    }
  } else {
    z.f = a.f + b.f + RB * (W - 1);
#pragma unroll
    for (int k = 0; k < W; ++k) {
      z.r[k] = (int32_t)cr[k + W - 1 - C0];
      z.i[k] = (int32_t)ci[k + W - 1 - C0];
    }
    z.r[W - 1] += (int32_t)(tr * (1LL << RB));  // fold a sign-only top column
    z.i[W - 1] += (int32_t)(ti * (1LL << RB));
  }
  normalize_top<W>(z);
  return z;
}

// Add e * z (e a small positive integer) into fixed-point accumulators with
// limb 0 weight 2^F: acc_r, acc_i [WA] int32 (limbs 0..WA-2 in [0, 2^29) after
// the carry, top signed).  The caller guarantees |e z| < 2^(29 (WA - 1) + 28 + F)
// (returns false, adding nothing, if z's frame lies above the accumulator's).
template <int W, int WA>
HT_HD bool acc_add(int32_t* acc_r, int32_t* acc_i, const fz<W>& z, int e, int F) {
  const int s = F - z.f;  // right shift of z into the accumulator frame
  if (s < -(RB - 1)) return false;
  int64_t ar[WA], ai[WA];
#pragma unroll
  for (int k = 0; k < WA; ++k) {
    ar[k] = acc_r[k];
    ai[k] = acc_i[k];
  }
  // z = sum_k d_k 2^(29 k + f): add each limb as a scaled integer
#pragma unroll
  for (int k = 0; k < W; ++k) {
    add_scaled<WA>(ar, (int64_t)z.r[k] * e, z.f + RB * k, F);
    add_scaled<WA>(ai, (int64_t)z.i[k] * e, z.f + RB * k, F);
  }
  carry<WA>(ar);
  carry<WA>(ai);
#pragma unroll
  for (int k = 0; k < WA; ++k) {
    acc_r[k] = (int32_t)ar[k];
    acc_i[k] = (int32_t)ai[k];
  }
  return true;
}

// One component of z as WA digits of a fixed-point frame, by one shift of the
// whole two's complement limb string: limb k of z sits at bit 29 k + (f - F)
// of the frame, F - f = 29 (q - 1) + r with 0 <= q <= W.  Bits that land
// below limb 0 are dropped (truncation: at most one unit of the last limb);
// digits 0..WA-2 come out in [0, 2^29), the top one signed.  With one zero
// digit prepended below limb 0, digit j is bits [r, r + 29) of string digits
// j + q and j + q + 1; the string is shifted down by q one bit of q at a time
// (static indices only).
template <int W, int WA>
HT_HD void shifted_digits(const int32_t* z, int q, int r, int32_t* v) {
  constexpr int N = W + WA + 4;
  constexpr int TOP = W >= 8 ? 8 : (W >= 4 ? 4 : (W >= 2 ? 2 : 1));  // highest bit of q <= W
  const int32_t ext = z[W - 1] < 0 ? MASK : 0;  // the string's sign digits
  int32_t D[N];
  D[0] = 0;
#pragma unroll
  for (int k = 0; k < W - 1; ++k) D[1 + k] = z[k];
  D[W] = z[W - 1] & MASK;
#pragma unroll
  for (int k = W + 1; k < N; ++k) D[k] = ext;
#pragma unroll
  for (int b = TOP; b >= 1; b >>= 1) {
    const bool take = (q & b) != 0;
#pragma unroll
    for (int k = 0; k < N; ++k) D[k] = take ? (k + b < N ? D[k + b] : ext) : D[k];
  }
#pragma unroll
  for (int j = 0; j < WA; ++j) {
    v[j] = (int32_t)((((uint32_t)D[j] >> r) | ((uint32_t)D[j + 1] << (RB - r))) & (uint32_t)MASK);
    if (j == WA - 1) v[j] = (v[j] << (32 - RB)) >> (32 - RB);  // the top digit carries the sign
  }
}

// Carry-propagate int32 limbs (limbs 0..N-2 to [0, 2^29), the top signed).
template <int N>
HT_HD void carry32(int32_t* a) {
#pragma unroll
  for (int j = 0; j + 1 < N; ++j) {
    const int32_t c = a[j] >> RB;  // floor division (arithmetic shift)
    a[j] &= MASK;
    a[j + 1] += c;
  }
}

// e * z into int32 accumulators acc_r, acc_i [WA] (frame F), carried.
// Returns false (adding nothing) if z's frame lies more than 28 bits above F.
// For |e| <= 3 the sums stay in 32 bits: a limb below the top holds at most
// 2^29 - 1, takes e d with |e d| <= 3 (2^29 - 1) and a carry of at most 3 in
// magnitude, so it stays inside int32 before its own carry.
template <int W, int WA>
HT_HD bool acc_add_fast(int32_t* acc_r, int32_t* acc_i, const fz<W>& z, int e, int F) {
  const int s = F - z.f;
  if (s < -(RB - 1)) return false;
  const int sp = s + RB, q = sp / RB, r = sp % RB;
  if (q > W) return true;  // below the accumulator's last limb
  int32_t dr[WA], di[WA];
  shifted_digits<W, WA>(z.r, q, r, dr);
  shifted_digits<W, WA>(z.i, q, r, di);
  if (e >= -3 && e <= 3) {
#pragma unroll
    for (int k = 0; k < WA; ++k) {
      acc_r[k] += e * dr[k];
      acc_i[k] += e * di[k];
    }
    carry32<WA>(acc_r);
    carry32<WA>(acc_i);
    return true;
  }
  int64_t ar[WA], ai[WA];
#pragma unroll
  for (int k = 0; k < WA; ++k) {
    ar[k] = acc_r[k] + (int64_t)e * dr[k];
    ai[k] = acc_i[k] + (int64_t)e * di[k];
  }
  carry<WA>(ar);
  carry<WA>(ai);
#pragma unroll
  for (int k = 0; k < WA; ++k) {
    acc_r[k] = (int32_t)ar[k];
    acc_i[k] = (int32_t)ai[k];
  }
  return true;
}

// Fixed-point value sum_k a_k 2^(29 k + F) (WA limbs, top signed) to L doubles
// whose sum equals it up to the last double's precision: the magnitude's bits
// are cut from the top into 53-bit pieces (each piece exact in a double).
template <int WA, int L>
HT_HD void fixed_to_doubles(const int32_t* a, int F, double* out) {
  int64_t m[WA];
#pragma unroll
  for (int k = 0; k < WA; ++k) m[k] = a[k];
  carry<WA>(m);
  const bool neg = m[WA - 1] < 0;
  if (neg) {
#pragma unroll
    for (int k = 0; k < WA; ++k) m[k] = -m[k];
    carry<WA>(m);  // magnitude: all limbs in [0, 2^29), top >= 0
  }
  // top nonzero limb and bit
  int top = -1;
#pragma unroll
  for (int k = 0; k < WA; ++k)
    if (m[k] != 0) top = k;
#pragma unroll
  for (int l = 0; l < L; ++l) out[l] = 0.0;
  if (top < 0) return;
  const int tb = bitlen64((uint64_t)m[top]) - 1;
  int hi_bit = RB * top + tb;  // absolute bit index of the leading bit
#pragma unroll
  for (int l = 0; l < L; ++l) {
    // extract bits [hi_bit - 52, hi_bit] as an integer (bits below 0 are zero)
    const int lo_bit = hi_bit - 52;
    uint64_t piece = 0;
#pragma unroll
    for (int k = 0; k < WA; ++k) {
      const int base = RB * k;  // limb k covers bits [base, base + 28]
      if (base + RB - 1 < lo_bit || base > hi_bit) continue;
      uint64_t v = (uint64_t)m[k];
      // keep the part of limb k inside [lo_bit, hi_bit]
      int from = lo_bit > base ? lo_bit - base : 0;
      int to = hi_bit < base + RB - 1 ? hi_bit - base : RB - 1;
      v = (v >> from) & ((1ULL << (to - from + 1)) - 1);
      const int pos = base + from - lo_bit;  // position in the piece
      piece |= pos >= 0 ? (v << pos) : (v >> -pos);
    }
    // piece * 2^(lo_bit + F), exact (piece < 2^53)
    double d = (double)(int64_t)piece;
    int ex = lo_bit + F;
    // scale by 2^ex in steps that stay in range
    while (ex > 600) {
      d *= bitsd((int64_t)(1023 + 600) << 52);
      ex -= 600;
    }
    while (ex < -600) {
      d *= bitsd((int64_t)(1023 - 600) << 52);
      ex += 600;
    }
    d *= bitsd((int64_t)(1023 + ex) << 52);
    out[l] = neg ? -d : d;
    hi_bit = lo_bit - 1;
    if (hi_bit < 0) break;
  }
}

// s a for a fixed-point value a (WA limbs, frame F) and a double s, to L
// doubles: the product is formed exactly in WA + 2 limbs (s's significand in
// a 24-bit and a 29-bit part) and converted once, as fixed_to_doubles does.
// For s = 1 the doubles are those of fixed_to_doubles.
template <int WA, int L>
HT_HD void fixed_scaled_to_doubles(const int32_t* a, int F, double s, double* out) {
  int64_t ms;
  int es;
  decompose(s, ms, es);  // s = ms 2^es, |ms| < 2^53
  const bool neg = ms < 0;
  const uint64_t u = (uint64_t)(neg ? -ms : ms);
  const int64_t lo = (int64_t)(u & (uint64_t)MASK), hi = (int64_t)(u >> RB);
  int64_t c[WA + 2];
#pragma unroll
  for (int k = 0; k < WA + 2; ++k) c[k] = 0;
#pragma unroll
  for (int k = 0; k < WA; ++k) {  // |a_k lo| < 2^58, |a_k hi| < 2^53
    c[k] += (int64_t)a[k] * lo;
    c[k + 1] += (int64_t)a[k] * hi;
  }
  if (neg) {
#pragma unroll
    for (int k = 0; k < WA + 2; ++k) c[k] = -c[k];
  }
  carry<WA + 2>(c);
  int32_t b[WA + 2];  // the top limb holds |a| |ms| / 2^(29 (WA + 1)) < 2^24
#pragma unroll
  for (int k = 0; k < WA + 2; ++k) b[k] = (int32_t)c[k];
  fixed_to_doubles<WA + 2, L>(b, F + es, out);
}

}  // namespace mpi
}  // namespace ht
