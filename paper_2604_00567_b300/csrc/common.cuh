// common.cuh — device types and the unified 6-FMA butterfly shared by the
// fused and sweep kernels of libdsfft.
//
// Packed twiddle entry (16 bytes, one per k in [0, N/2)):
//   FP32     : x = t, y = m, z = sigma*m, w = path (0 cosine, 1 sine)
//   FP16/BF16: x = (lo -t, hi t), y = (lo sigma*m, hi m), z = byte-permute
//              selector that builds the operand swap, w = -y = (lo -sigma*m,
//              hi -m)
// sigma = +1 on the cosine path, -1 on the sine path.
//
// Unified butterfly (branch-free form of the two factorizations; the
// paper's Discussion notes the per-twiddle branch can be removed by
// encoding the operand order in the table):
//   (R, S) = cosine path ? (b_r, b_i) : (b_i, b_r)
//   u = fma(-t, S, R)            cosine: b_r - t b_i  (Eq. 7 s1)
//                                sine  : b_i - t b_r  (Eq. 4 s1)
//   v = fma( t, R, S)            cosine: t b_r + b_i  (Eq. 7 s2)
//                                sine  : b_r + t b_i  (Eq. 4 s2, corrected)
//   A_r = fma( sigma m, u, a_r)  B_r = fma(-sigma m, u, a_r)   (Eqs. 5-6, 8-9)
//   A_i = fma(       m, v, a_i)  B_i = fma(-m,       v, a_i)
// With x0.5 per pass a is first replaced by RN(a/2) and m is stored halved.
// Every operation is one correctly rounded IEEE operation (fma.rn / mul.rn,
// no flush-to-zero), so the result is bit-identical to the branched forms.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "internal.h"

namespace dsfft {

constexpr double kTwoPi = 6.283185307179586476925286766559;  // 2*pi as a double: exactly 2 * M_PI

__host__ __device__ constexpr int bitrev(int v, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1) << (bits - 1 - i);
  return r;
}

// Compile-time loop: f(std::integral_constant<int, I>) for I in [BEGIN, END).
// Keeps every register-array index a constant however deep the nesting.
template <int BEGIN, int END, class F>
__device__ __forceinline__ void static_for(F &&f) {
  if constexpr (BEGIN < END) {
    f(std::integral_constant<int, BEGIN>{});
    static_for<BEGIN + 1, END>(f);
  }
}

// Streaming (evict-first) loads and stores of signal data: every element is
// touched once, so it should not displace the twiddle table in L1/L2.
__device__ __forceinline__ float2 ldcs(const float2 *p) { return __ldcs(p); }
__device__ __forceinline__ uint32_t ldcs(const uint32_t *p) { return __ldcs(reinterpret_cast<const unsigned int *>(p)); }
__device__ __forceinline__ void stcs(float2 *p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void stcs(uint32_t *p, uint32_t v) { __stcs(reinterpret_cast<unsigned int *>(p), v); }

// Where the signals of transform k live: contiguous batches (transform k at
// k N) or a gathered list of per-transform pointers (mixed batches).
template <class E>
struct ContigIO {
  const E *in;
  E *out;
  int64_t n;
  __device__ __forceinline__ const E *src(int64_t k) const { return in + k * n; }
  __device__ __forceinline__ E *dst(int64_t k) const { return out + k * n; }
};
template <class E>
struct GatherIO {
  const BatchItem *items;
  __device__ __forceinline__ const E *src(int64_t k) const { return static_cast<const E *>(items[k].in); }
  __device__ __forceinline__ E *dst(int64_t k) const { return static_cast<E *>(items[k].out); }
};

// Per-pass twiddle entries as the kernels read them: compact 8-byte
// entries, unpacked in registers to the 16-byte form above.
//   FP16/BF16: x = selector (low half) | t (high half), y = (lo sigma*m,
//              hi m); three integer operations rebuild (-t, t) (a sign flip
//              and a byte permute) and -(sigma m, m) (a sign flip), and the
//              permute that uses the selector reads only its low 16 bits.
//   FP32     : x = t, y = m with the path in bit 30 (the top exponent bit,
//              always 0 since |m| <= 1 for every factorization, halved or
//              not); sigma m = m with the sign flipped on the sine path.
// Half the bytes per entry halves the L1/L2 traffic of the later register
// stages, whose lanes each read a different entry.
template <int PREC> struct TwEntry { using T = uint2; };

template <int PREC>
__device__ __forceinline__ uint4 tw_unpack(const uint2 e) {
  uint4 r;
  if constexpr (PREC == kFP32) {
    const uint32_t path = (e.y >> 30) & 1u;
    const uint32_t m = e.y & 0xBFFFFFFFu;
    r.x = e.x;
    r.y = m;
    r.z = m ^ (path << 31);
    r.w = path;
  } else {
    r.x = __byte_perm(e.x, e.x ^ 0x80000000u, 0x3276);   // (lo -t, hi t)
    r.y = e.y;
    r.z = e.x;
    r.w = e.y ^ 0x80008000u;
  }
  return r;
}
// Entry i of a per-pass table (the table's storage is TwEntry<PREC>::T[]).
template <int PREC>
__device__ __forceinline__ uint4 tw_load(const uint4 *table, int64_t i) {
  return tw_unpack<PREC>(__ldg(reinterpret_cast<const typename TwEntry<PREC>::T *>(table) + i));
}

// Storage type of one complex element.
template <int PREC> struct Elem;
template <> struct Elem<kFP32> { using T = float2; };
template <> struct Elem<kFP16> { using T = uint32_t; };
template <> struct Elem<kBF16> { using T = uint32_t; };

// ---------------------------------------------------------------------------
// Butterfly.  a <- A, b <- B.
template <int PREC, bool SCALED> struct Bfly;

template <bool SCALED> struct Bfly<kFP32, SCALED> {
  static __device__ __forceinline__ void finish(float2 &a, float2 &b, const uint4 e, float u, float v) {
    const float m = __uint_as_float(e.y);
    const float sm = __uint_as_float(e.z);
    float ar = a.x, ai = a.y;
    if (SCALED) {
      ar = __fmul_rn(ar, 0.5f);
      ai = __fmul_rn(ai, 0.5f);
    }
    a.x = __fmaf_rn(sm, u, ar);
    b.x = __fmaf_rn(-sm, u, ar);
    a.y = __fmaf_rn(m, v, ai);
    b.y = __fmaf_rn(-m, v, ai);
  }
  static __device__ __forceinline__ void run(float2 &a, float2 &b, const uint4 e) {
    const float t = __uint_as_float(e.x);
    const bool sine = e.w != 0u;
    const float R = sine ? b.y : b.x;
    const float S = sine ? b.x : b.y;
    finish(a, b, e, __fmaf_rn(-t, S, R), __fmaf_rn(t, R, S));
  }
  // The path known at the call site (COS: cosine), for a twiddle that is
  // the same in every lane: no operand selection.
  template <bool COS>
  static __device__ __forceinline__ void run_path(float2 &a, float2 &b, const uint4 e) {
    const float t = __uint_as_float(e.x);
    const float R = COS ? b.x : b.y;
    const float S = COS ? b.y : b.x;
    finish(a, b, e, __fmaf_rn(-t, S, R), __fmaf_rn(t, R, S));
  }
};

__device__ __forceinline__ uint32_t h2_fma(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t h2_mul(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t b2_fma(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t b2_mul(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// Exchange the two halves of a packed pair.  Written as an unpack and
// repack of the 16-bit halves (not a byte permute) so that the compiler can
// fold it into the operand of the packed FMA that consumes it.
__device__ __forceinline__ uint32_t swap_halves(uint32_t x) {
  uint32_t y;
  asm("{.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\tmov.b32 %0, {h, l};}" : "=r"(y) : "r"(x));
  return y;
}

template <int PREC, bool SCALED> struct BflyPacked {
  static __device__ __forceinline__ uint32_t fma2(uint32_t a, uint32_t b, uint32_t c) {
    return PREC == kFP16 ? h2_fma(a, b, c) : b2_fma(a, b, c);
  }
  static __device__ __forceinline__ uint32_t mul2(uint32_t a, uint32_t b) {
    return PREC == kFP16 ? h2_mul(a, b) : b2_mul(a, b);
  }
  // fma(-a, b, c): the negation is exact and is written as its own
  // instruction so that the compiler can fold it into the FMA's operand.
  static __device__ __forceinline__ uint32_t nfma2(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    if (PREC == kFP16)
      asm("{.reg .b32 n;\n\tneg.f16x2 n, %1;\n\tfma.rn.f16x2 %0, n, %2, %3;}" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    else
      asm("{.reg .b32 n;\n\tneg.bf16x2 n, %1;\n\tfma.rn.bf16x2 %0, n, %2, %3;}" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
  }
  static __device__ __forceinline__ void finish(uint32_t &a, uint32_t &b, const uint4 e, uint32_t uv) {
    uint32_t ah = a;
    if (SCALED) ah = mul2(a, PREC == kFP16 ? 0x38003800u : 0x3F003F00u);  // x 0.5
    a = fma2(e.y, uv, ah);                         // (sigma m, m) (u, v) + a
    b = nfma2(e.y, uv, ah);                        // -(sigma m, m) (u, v) + a
  }
  static __device__ __forceinline__ void run(uint32_t &a, uint32_t &b, const uint4 e) {
    // X = cosine ? swap(b) : b ; Y = swap(X)
    const uint32_t X = __byte_perm(b, b, e.z);
    finish(a, b, e, fma2(e.x, X, swap_halves(X)));   // (u, v)
  }
  // The path known at the call site (COS: cosine), for a twiddle that is
  // the same in every lane: X and Y are b and its swap in a fixed order, so
  // no byte permute (the swap folds into the FMA's operand).
  template <bool COS>
  static __device__ __forceinline__ void run_path(uint32_t &a, uint32_t &b, const uint4 e) {
    const uint32_t sb = swap_halves(b);
    finish(a, b, e, COS ? fma2(e.x, sb, b) : fma2(e.x, b, sb));
  }
};

// Cosine path of an unpacked entry (FP32: path word; FP16/BF16: the byte
// permute selector, 0x1032 on the cosine path).
template <int PREC>
__device__ __forceinline__ bool tw_is_cosine(const uint4 e) {
  if constexpr (PREC == kFP32) return e.w == 0u;
  else return (e.z & 0xFFFFu) == 0x1032u;
}

template <bool SCALED> struct Bfly<kFP16, SCALED> : BflyPacked<kFP16, SCALED> {};
template <bool SCALED> struct Bfly<kBF16, SCALED> : BflyPacked<kBF16, SCALED> {};

// ---------------------------------------------------------------------------
// Radix-4 butterfly (the radix-4 extension of the Discussion: each of the
// three twiddle products takes the form of its own table entry).  Inputs
// a0..a3 = Z[q N/4 + s L + j], entries e1..e3 of W_4L^(q j); with
// (u_q, v_q) the pre-products above and W a_q = (sigma m u, m v):
//   b3 = W^3j a3 (two rounded multiplies)
//   c0 = a0 + W^2j a2, c1 = a0 - W^2j a2, c2 = W^j a1 + b3, d3 = b3 - W^j a1
//   y0 = c0 + c2, y2 = c0 - c2, y1 = c1 + s i d3, y3 = c1 - s i d3,
// s = +1 forward (y1 = c1 - i c3 with c3 = -d3), -1 inverse, every step one
// correctly rounded operation (the sums as fma(x, +-1, y), exact products).
// Scaled: a0 <- RN(a0 / 4) and the table multipliers are RN(m / 4).
// Outputs go to the registers of two consecutive radix-2 passes' results:
// a0 <- y0, a1 <- y2, a2 <- y1, a3 <- y3.
template <int PREC, bool SCALED> struct Bfly4;

template <bool SCALED> struct Bfly4<kFP32, SCALED> {
  static __device__ __forceinline__ float2 pre(const float2 b, const uint4 e) {
    const float t = __uint_as_float(e.x);
    const bool sine = e.w != 0u;
    const float R = sine ? b.y : b.x;
    const float S = sine ? b.x : b.y;
    return make_float2(__fmaf_rn(-t, S, R), __fmaf_rn(t, R, S));
  }
  // sgn: -1 forward, +1 inverse (the sign of the real part of y1's d3 term)
  static __device__ __forceinline__ void run(float2 &a0, float2 &a1, float2 &a2, float2 &a3, const uint4 e1,
                                             const uint4 e2, const uint4 e3, const float sgn) {
    const float2 p1 = pre(a1, e1), p2 = pre(a2, e2), p3 = pre(a3, e3);
    float x0r = a0.x, x0i = a0.y;
    if (SCALED) {
      x0r = __fmul_rn(x0r, 0.25f);
      x0i = __fmul_rn(x0i, 0.25f);
    }
    const float m1 = __uint_as_float(e1.y), sm1 = __uint_as_float(e1.z);
    const float m2 = __uint_as_float(e2.y), sm2 = __uint_as_float(e2.z);
    const float m3 = __uint_as_float(e3.y), sm3 = __uint_as_float(e3.z);
    const float b3r = __fmul_rn(sm3, p3.x), b3i = __fmul_rn(m3, p3.y);
    const float c0r = __fmaf_rn(sm2, p2.x, x0r), c0i = __fmaf_rn(m2, p2.y, x0i);
    const float c1r = __fmaf_rn(-sm2, p2.x, x0r), c1i = __fmaf_rn(-m2, p2.y, x0i);
    const float c2r = __fmaf_rn(sm1, p1.x, b3r), c2i = __fmaf_rn(m1, p1.y, b3i);
    const float d3r = __fmaf_rn(-sm1, p1.x, b3r), d3i = __fmaf_rn(-m1, p1.y, b3i);
    a0 = make_float2(__fmaf_rn(c2r, 1.0f, c0r), __fmaf_rn(c2i, 1.0f, c0i));
    a1 = make_float2(__fmaf_rn(c2r, -1.0f, c0r), __fmaf_rn(c2i, -1.0f, c0i));
    a2 = make_float2(__fmaf_rn(d3i, sgn, c1r), __fmaf_rn(d3r, -sgn, c1i));
    a3 = make_float2(__fmaf_rn(d3i, -sgn, c1r), __fmaf_rn(d3r, sgn, c1i));
  }
};

template <int PREC, bool SCALED> struct Bfly4Packed {
  using B = BflyPacked<PREC, SCALED>;
  static constexpr uint32_t kOne = PREC == kFP16 ? 0x3C003C00u : 0x3F803F80u;
  static constexpr uint32_t kQuarter = PREC == kFP16 ? 0x34003400u : 0x3E803E80u;
  static __device__ __forceinline__ uint32_t pre(const uint32_t b, const uint4 e) {
    const uint32_t X = __byte_perm(b, b, e.z);
    return B::fma2(e.x, X, swap_halves(X));
  }
  // sgn: the half pair (lo s, hi -s) with s = -1 forward, +1 inverse
  static __device__ __forceinline__ void run(uint32_t &a0, uint32_t &a1, uint32_t &a2, uint32_t &a3, const uint4 e1,
                                             const uint4 e2, const uint4 e3, const uint32_t sgn) {
    const uint32_t p1 = pre(a1, e1), p2 = pre(a2, e2), p3 = pre(a3, e3);
    uint32_t x0 = a0;
    if (SCALED) x0 = B::mul2(a0, kQuarter);
    const uint32_t b3 = B::mul2(e3.y, p3);
    const uint32_t c0 = B::fma2(e2.y, p2, x0), c1 = B::nfma2(e2.y, p2, x0);
    const uint32_t c2 = B::fma2(e1.y, p1, b3), d3 = B::nfma2(e1.y, p1, b3);
    const uint32_t D = swap_halves(d3);   // (d3i, d3r)
    a0 = B::fma2(c2, kOne, c0);
    a1 = B::fma2(c2, kOne ^ 0x80008000u, c0);
    a2 = B::fma2(D, sgn, c1);
    a3 = B::fma2(D, sgn ^ 0x80008000u, c1);
  }
};

template <bool SCALED> struct Bfly4<kFP16, SCALED> : Bfly4Packed<kFP16, SCALED> {};
template <bool SCALED> struct Bfly4<kBF16, SCALED> : Bfly4Packed<kBF16, SCALED> {};

}  // namespace dsfft
