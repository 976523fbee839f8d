// table.cu — FP64 twiddle-table builder (Algorithm 1 and the two single
// factorizations of Eqs. 4-6 and 7-9), run on the GPU once per plan.
//
// For k in [0, count) (N/2 for the radix-2 table, 3N/4 for the radix-4
// table, whose W^3j products pass -pi): theta = (-2 pi k)/N in FP64 (evaluated in that order,
// so the entries of N are every (Nmax/N)-th entry of the table of Nmax),
// w_r = cos theta, w_i = sin theta.  Selection:
//   dual-select : cosine path when |w_r| >= |w_i| (Algorithm 1), else sine
//   linzer-feig : sine path; w_i := -eps where |w_i| < eps (Section I clamp)
//   cosine      : cosine path
// cosine path: m = w_r, t = w_i / w_r ; sine path: m = w_i, t = w_r / w_i.
// The inverse direction conjugates W (w_i -> -w_i) after the clamp; a scaled
// direction stores m/2 (radix-2 passes) or m/4 (radix-4 passes).  t and m
// are then rounded ONCE (cvt.rn) from FP64 to the plan precision and packed
// (layout in common.cuh).
#include "common.cuh"
#include "internal.h"

namespace dsfft {

__device__ __forceinline__ uint16_t f64_to_f16_bits(double x) {
  uint16_t h;
  asm("cvt.rn.f16.f64 %0, %1;" : "=h"(h) : "d"(x));
  return h;
}
__device__ __forceinline__ uint16_t f64_to_bf16_bits(double x) {
  uint16_t h;
  asm("cvt.rn.bf16.f64 %0, %1;" : "=h"(h) : "d"(x));
  return h;
}

struct Fp64Entry {
  double t, m;
  int sine;
};

__device__ __forceinline__ Fp64Entry fp64_entry(int64_t k, int log2n, int fac, double eps, int inverse) {
  const double th = (-kTwoPi * (double)k) / (double)(1LL << log2n);
  double wr, wi;
  sincos(th, &wi, &wr);
  int sine;
  if (fac == 2) {
    sine = !(fabs(wr) >= fabs(wi));
  } else if (fac == 0) {
    sine = 1;
    if (fabs(wi) < eps) wi = -eps;
  } else {
    sine = 0;
  }
  if (inverse) wi = -wi;
  Fp64Entry e;
  if (sine) {
    e.m = wi;
    e.t = wr / wi;
  } else {
    e.m = wr;
    e.t = wi / wr;
  }
  e.sine = sine;
  return e;
}

__global__ void build_table_kernel(int log2n, int64_t count, int fac, double eps, int prec, int inverse,
                                   double mscale, uint4 *__restrict__ out, int *__restrict__ counts) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  Fp64Entry e = fp64_entry(k, log2n, fac, eps, inverse);
  double m = e.m * mscale;   // mscale is 1, 1/2 or 1/4: exact
  uint4 w;
  if (prec == kFP32) {
    const float tf = __double2float_rn(e.t);
    const float mf = __double2float_rn(m);
    w.x = __float_as_uint(tf);
    w.y = __float_as_uint(mf);
    w.z = __float_as_uint(e.sine ? -mf : mf);
    w.w = (uint32_t)e.sine;
  } else {
    const uint32_t tb = prec == kFP16 ? f64_to_f16_bits(e.t) : f64_to_bf16_bits(e.t);
    const uint32_t mb = prec == kFP16 ? f64_to_f16_bits(m) : f64_to_bf16_bits(m);
    const uint32_t smb = e.sine ? (mb ^ 0x8000u) : mb;
    w.x = ((tb ^ 0x8000u) & 0xFFFFu) | (tb << 16);        // (lo -t, hi t)
    w.y = (smb & 0xFFFFu) | (mb << 16);                   // (lo sigma*m, hi m)
    w.z = e.sine ? 0x3210u : 0x1032u;                     // X = cosine ? swap(b) : b
    w.w = w.y ^ 0x80008000u;                              // (lo -sigma*m, hi -m)
  }
  out[k] = w;
  if (counts) atomicAdd(&counts[e.sine], 1);
}

// Store per-pass entry i: the 16-byte packed entry (form 0), or its
// compact 8-byte form (common.cuh TwEntry): form 1 for FP16/BF16
// {selector | t << 16, (sigma m, m)}, form 2 for FP32 {t, m | path << 30}
// (|m| <= 1, so bit 30 of m is free).
__device__ __forceinline__ void put_entry(void *out, int64_t i, const uint4 w, int form) {
  if (form == 1)
    static_cast<uint2 *>(out)[i] = make_uint2((w.z & 0xFFFFu) | (w.x & 0xFFFF0000u), w.y);
  else if (form == 2)
    static_cast<uint2 *>(out)[i] = make_uint2(w.x, w.y | (w.w << 30));
  else
    static_cast<uint4 *>(out)[i] = w;
}

// Per-pass copy of the packed table: pass p (half-span 2^p) uses entry
// table[j N/2^(p+1)] for j in [0, 2^p); it is stored at twp[2^p - 1 + j]
// (entries [0, count) of the N - 1).
__global__ void per_pass_table_kernel(int log2n, const uint4 *__restrict__ table, void *__restrict__ twp,
                                      int64_t count, int form) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  int p = 63 - __clzll(i + 1);            // 2^p - 1 <= i < 2^(p+1) - 1
  const int64_t j = i - ((1LL << p) - 1);
  put_entry(twp, i, table[j << (log2n - p - 1)], form);
}

cudaError_t launch_per_pass_table(int log2n, const uint4 *table, void *twp, int64_t count, int form,
                                  cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)((count + threads - 1) / threads);
  per_pass_table_kernel<<<blocks, threads, 0, stream>>>(log2n, table, twp, count, form);
  return cudaGetLastError();
}

__global__ void fp64_table_kernel(int log2n, int fac, double eps, double *t, double *m, int *path) {
  const int64_t half = 1LL << (log2n - 1);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= half) return;
  Fp64Entry e = fp64_entry(k, log2n, fac, eps, 0);
  t[k] = e.t;
  m[k] = e.m;
  path[k] = e.sine;
}

cudaError_t launch_build_table(int log2n, int64_t count, int fac, double eps, int prec, int inverse, double mscale,
                               uint4 *out, int *counts, cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)((count + threads - 1) / threads);
  build_table_kernel<<<blocks, threads, 0, stream>>>(log2n, count, fac, eps, prec, inverse, mscale, out, counts);
  return cudaGetLastError();
}

// Per-pass copy for the radix-4 passes (levels l = par, par + 2, ..., log2 N
// - 2 with par = log2 N mod 2, span L = 2^l): level l occupies
// [r4_offset(l), r4_offset(l) + 3L) as three runs of L entries, run q - 1
// holding W_4L^(q j) = table4[q j N/(4L)] for j in [0, L), q = 1, 2, 3.
__global__ void per_pass_table4_kernel(int log2n, const uint4 *__restrict__ table4, void *__restrict__ twp4,
                                       int64_t count, int form) {
  const int par = log2n & 1;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  int l = par;
  while (r4_offset(l + 2, par) <= i) l += 2;
  const int64_t L = 1LL << l;
  const int64_t rem = i - r4_offset(l, par);
  const int64_t q = rem / L + 1, j = rem % L;
  put_entry(twp4, i, table4[(q * j) << (log2n - l - 2)], form);
}

cudaError_t launch_per_pass_table4(int log2n, const uint4 *table4, void *twp4, int64_t count, int form,
                                   cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)((count + threads - 1) / threads);
  per_pass_table4_kernel<<<blocks, threads, 0, stream>>>(log2n, table4, twp4, count, form);
  return cudaGetLastError();
}

cudaError_t launch_fp64_table(int log2n, int fac, double eps, double *t, double *m, int *path,
                              cudaStream_t stream) {
  const int64_t half = 1LL << (log2n - 1);
  const int threads = 256;
  const unsigned blocks = (unsigned)((half + threads - 1) / threads);
  fp64_table_kernel<<<blocks, threads, 0, stream>>>(log2n, fac, eps, t, m, path);
  return cudaGetLastError();
}

}  // namespace dsfft
