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

// Storage type of one complex element.
template <int PREC> struct Elem;
template <> struct Elem<kFP32> { using T = float2; };
template <> struct Elem<kFP16> { using T = uint32_t; };
template <> struct Elem<kBF16> { using T = uint32_t; };

// ---------------------------------------------------------------------------
// Butterfly.  a <- A, b <- B.
template <int PREC, bool SCALED> struct Bfly;

template <bool SCALED> struct Bfly<kFP32, SCALED> {
  static __device__ __forceinline__ void run(float2 &a, float2 &b, const uint4 e) {
    const float t = __uint_as_float(e.x);
    const float m = __uint_as_float(e.y);
    const float sm = __uint_as_float(e.z);
    const bool sine = e.w != 0u;
    const float R = sine ? b.y : b.x;
    const float S = sine ? b.x : b.y;
    const float u = __fmaf_rn(-t, S, R);
    const float v = __fmaf_rn(t, R, S);
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

template <int PREC, bool SCALED> struct BflyPacked {
  static __device__ __forceinline__ uint32_t fma2(uint32_t a, uint32_t b, uint32_t c) {
    return PREC == kFP16 ? h2_fma(a, b, c) : b2_fma(a, b, c);
  }
  static __device__ __forceinline__ uint32_t mul2(uint32_t a, uint32_t b) {
    return PREC == kFP16 ? h2_mul(a, b) : b2_mul(a, b);
  }
  static __device__ __forceinline__ void run(uint32_t &a, uint32_t &b, const uint4 e) {
    // X = cosine ? swap(b) : b ; Y = swap(X)
    const uint32_t X = __byte_perm(b, b, e.z);
    const uint32_t Y = __byte_perm(X, X, 0x1032);
    const uint32_t uv = fma2(e.x, X, Y);           // (u, v)
    uint32_t ah = a;
    if (SCALED) ah = mul2(a, PREC == kFP16 ? 0x38003800u : 0x3F003F00u);  // x 0.5
    a = fma2(e.y, uv, ah);
    b = fma2(e.w, uv, ah);
  }
};

template <bool SCALED> struct Bfly<kFP16, SCALED> : BflyPacked<kFP16, SCALED> {};
template <bool SCALED> struct Bfly<kBF16, SCALED> : BflyPacked<kBF16, SCALED> {};

}  // namespace dsfft
