// fused.cu — one-launch FFT for N <= 2^14: every pass of a transform runs on
// chip, so each signal is read from HBM once and written once.
//
// The m = log2 N radix-2 Stockham passes (Section IV) are grouped into
// stages of up to r = log2 R passes.  Before pass P the Stockham array is
// Z_P[s 2^P + j] (s in [0, N/2^P), j in [0, 2^P)); pass P combines
// a = Z_P[s 2^P + j], b = Z_P[N/2 + s 2^P + j] with W = table[j N/2^(P+1)]
// into Z_{P+1}[s 2^(P+1) + j] = a + W b, Z_{P+1}[s 2^(P+1) + 2^P + j] = a - W b.
// A stage of rho passes starting at P only mixes, for each (s_lo, j), the
// 2^rho values Z_P[(s_lo + q N/2^(P+rho)) 2^P + j], q in [0, 2^rho), so one
// thread keeps them in registers and runs the rho passes with the exact
// butterflies of the radix-2 algorithm (same operands, same twiddles, same
// rounding): the result is bit-identical to pass-by-pass execution.  Stages
// exchange data through shared memory.  Thread `tid` of a transform reads
// Z_P[tid + p T] (p in [0, R), T = N/R threads), which is coalesced for the
// first stage (from HBM) and bank-conflict-free for the others; the last
// stage writes X[tid + p T] (coalesced).
//
// Twiddles come from the plan's per-pass table: pass p uses entries
// twp[2^p - 1 + j] = table[j N/2^(p+1)], j in [0, 2^p) (exact copies of the
// rounded entries), so the lanes of a warp, which hold consecutive j, read
// consecutive 16-byte entries.
#include "common.cuh"
#include "internal.h"

namespace dsfft {

// Streaming (evict-first) loads and stores of signal data: every element is
// touched once, so it should not displace the twiddle table in L1/L2.
__device__ __forceinline__ float2 ldcs(const float2 *p) { return __ldcs(p); }
__device__ __forceinline__ uint32_t ldcs(const uint32_t *p) { return __ldcs(reinterpret_cast<const unsigned int *>(p)); }
__device__ __forceinline__ void stcs(float2 *p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void stcs(uint32_t *p, uint32_t v) { __stcs(reinterpret_cast<unsigned int *>(p), v); }

template <int PREC, int LOG2N, int LOG2R, bool SCALED>
struct Fused {
  using E = typename Elem<PREC>::T;
  static constexpr int N = 1 << LOG2N;
  static constexpr int R = 1 << LOG2R;
  static constexpr int T = N / R;                        // threads per transform
  static constexpr int TPC = T >= 256 ? 1 : 256 / T;     // transforms per block
  static constexpr int TPB = T * TPC;
  static constexpr int NSTAGES = (LOG2N + LOG2R - 1) / LOG2R;
  static constexpr int PADN = N + (N >> 5);              // one pad element per 32 (conflict-free
                                                         // exchanges for R = 32 (4-byte) / R = 16 (8-byte))
  static constexpr int SMEM = NSTAGES > 1 ? TPC * PADN * (int)sizeof(E) : 0;
  // Blocks per SM the register allocation must allow: 1024 threads' worth
  // (at most 64 registers per thread), so at least half the SM's warps can
  // be resident.
  static constexpr int MINB = TPB >= 1024 ? 1 : 1024 / TPB;

  static __device__ __forceinline__ int pad(int idx) { return idx + (idx >> 5); }

  // Exchange barrier of one transform's T threads: a warp barrier when they
  // share a warp, a named barrier per transform when a block holds several
  // multi-warp transforms (so transforms do not wait for each other), else
  // the block barrier.
  static __device__ __forceinline__ void sync(int lt) {
    if constexpr (T <= 32) {
      __syncwarp();
    } else if constexpr (TPC > 1) {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + lt), "r"(T) : "memory");
    } else {
      __syncthreads();
    }
  }
  static_assert(TPC <= 15 || T <= 32, "named barriers 1..15");

  // rho radix-2 passes starting at pass P on the registers of one thread.
  template <int P, int RHO>
  static __device__ __forceinline__ void compute(E (&v)[R], int tid, const uint4 *__restrict__ tw,
                                                 const Stage0Twiddles &tw0) {
    constexpr int C = R >> RHO;   // independent groups per thread
    static_for<0, C>([&](auto c_) {
      constexpr int c = decltype(c_)::value;
      const int g = tid + c * T;
      const int j = g & ((1 << P) - 1);
      static_for<0, RHO>([&](auto i_) {
        constexpr int i = decltype(i_)::value;
        constexpr int half = 1 << (RHO - 1 - i);
        static_for<0, (1 << i)>([&](auto ql_) {
          constexpr int ql = decltype(ql_)::value;
          // pass P+i, j_full = j + ql 2^P; the first stage (j = 0) reads the
          // constant bank
          uint4 e;
          if constexpr (P == 0) e = tw0.e[((1 << i) - 1) + ql];
          else e = __ldg(tw + ((1 << (P + i)) - 1) + j + (ql << P));
          constexpr int qtop = bitrev(ql, i) << (RHO - i);
          static_for<0, half>([&](auto qh_) {
            constexpr int q = qtop | decltype(qh_)::value;
            Bfly<PREC, SCALED>::run(v[c + q * C], v[c + (q + half) * C], e);
          });
        });
      });
    });
  }

  template <int S>
  static __device__ __forceinline__ void stages(E (&v)[R], E *sm, int tid, int lt, const uint4 *__restrict__ tw,
                                                const Stage0Twiddles &tw0, E *dst, bool active) {
    constexpr int P = S * LOG2R;
    constexpr int RHO = (LOG2N - P) < LOG2R ? (LOG2N - P) : LOG2R;
    constexpr int C = R >> RHO;
    if constexpr (S > 0) {
      // pad(tid + p T) = pad(tid) + p T + p T / 32 when 32 | T: one base
      // address plus compile-time offsets
      const int pt = pad(tid);
      static_for<0, R>([&](auto p_) {
        constexpr int p = decltype(p_)::value;
        if constexpr (T % 32 == 0) v[p] = sm[pt + p * T + ((p * T) >> 5)];
        else v[p] = sm[pad(tid + p * T)];
      });
    }
    compute<P, RHO>(v, tid, tw, tw0);
    if constexpr (P + RHO == LOG2N) {
      if (active) {
        static_for<0, C>([&](auto c_) {
          constexpr int c = decltype(c_)::value;
          static_for<0, (1 << RHO)>([&](auto q_) {
            constexpr int q = decltype(q_)::value;
            stcs(dst + tid + c * T + (bitrev(q, RHO) << P), v[c + q * C]);
          });
        });
      }
    } else {
      if constexpr (S > 0) sync(lt);   // previous exchange fully read
      // pad(base + off) = pad(base) + off + off / 32 when off is a multiple
      // of 32 (P >= 5) or base is and off < 32 (P = 0, RHO = 5)
      constexpr bool FOLD = P >= 5 || (P == 0 && RHO == 5);
      static_for<0, C>([&](auto c_) {
        constexpr int c = decltype(c_)::value;
        const int g = tid + c * T;
        const int base = ((g >> P) << (P + RHO)) + (g & ((1 << P) - 1));
        const int pb = pad(base);
        static_for<0, (1 << RHO)>([&](auto q_) {
          constexpr int q = decltype(q_)::value;
          constexpr int off = bitrev(q, RHO) << P;
          if constexpr (FOLD) sm[pb + off + (off >> 5)] = v[c + q * C];
          else sm[pad(base + off)] = v[c + q * C];
        });
      });
      sync(lt);
      stages<S + 1>(v, sm, tid, lt, tw, tw0, dst, active);
    }
  }
};

template <int PREC, int LOG2N, int LOG2R, bool SCALED>
__global__ void __launch_bounds__(Fused<PREC, LOG2N, LOG2R, SCALED>::TPB, Fused<PREC, LOG2N, LOG2R, SCALED>::MINB)
    fused_fft_kernel(const typename Elem<PREC>::T *in, typename Elem<PREC>::T *out, int64_t batch,
                     const uint4 *__restrict__ tw, const __grid_constant__ Stage0Twiddles tw0) {
  using K = Fused<PREC, LOG2N, LOG2R, SCALED>;
  using E = typename K::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lt = threadIdx.x / K::T;
  const int tid = threadIdx.x % K::T;
  const int64_t tr = (int64_t)blockIdx.x * K::TPC + lt;
  const bool active = tr < batch;
  E *sm = reinterpret_cast<E *>(smem_raw) + lt * K::PADN;
  E v[K::R];
  const E *src = in + tr * K::N;
  if (active) {
    static_for<0, K::R>([&](auto p_) {
      constexpr int p = decltype(p_)::value;
      v[p] = ldcs(src + tid + p * K::T);
    });
  } else {
    static_for<0, K::R>([&](auto p_) { v[decltype(p_)::value] = E{}; });
  }
  K::template stages<0>(v, sm, tid, lt, tw, tw0, out + tr * K::N, active);
}

// ---------------------------------------------------------------------------
// dispatch

// Points per thread: 32 four-byte (FP16/BF16) or 16 eight-byte (FP32)
// elements, so a thread's register block is 32 registers and every exchange
// is bank-conflict-free with the one-in-32 padding.
constexpr int fused_log2r(int prec, int log2n) {
  const int r = prec == kFP32 ? 4 : 5;
  return log2n < r ? log2n : r;
}

template <int PREC, int LOG2N, bool SCALED>
static cudaError_t launch_one(const void *in, void *out, int64_t batch, const uint4 *tw, const Stage0Twiddles &tw0,
                              cudaStream_t stream) {
  constexpr int LOG2R = fused_log2r(PREC, LOG2N);
  using K = Fused<PREC, LOG2N, LOG2R, SCALED>;
  using E = typename K::E;
  auto kern = fused_fft_kernel<PREC, LOG2N, LOG2R, SCALED>;
  const int64_t blocks = (batch + K::TPC - 1) / K::TPC;
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
  kern<<<(unsigned)blocks, K::TPB, K::SMEM, stream>>>(static_cast<const E *>(in), static_cast<E *>(out), batch, tw, tw0);
  return cudaGetLastError();
}

// Raise the dynamic shared-memory limit of both variants on the current
// device (needed above 48 KB); called once per plan creation.
template <int PREC, int LOG2N>
static cudaError_t prepare_one() {
  constexpr int LOG2R = fused_log2r(PREC, LOG2N);
  using K = Fused<PREC, LOG2N, LOG2R, false>;
  // Shared-memory carveout: enough for the blocks the register budget lets
  // reside (MINB, at least one), the rest stays L1 for the twiddle table.
  const int per_block = K::SMEM + 1024;
  int carve = (int)((100LL * per_block * (K::MINB > 0 ? K::MINB : 1) + 228 * 1024 - 1) / (228 * 1024));
  carve = carve < 1 ? 1 : carve > 100 ? 100 : carve;
  for (auto kern : {fused_fft_kernel<PREC, LOG2N, LOG2R, false>, fused_fft_kernel<PREC, LOG2N, LOG2R, true>}) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
    if (e != cudaSuccess) return e;
    if (K::SMEM > 48 * 1024) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template <int PREC, int LOG2N>
static FusedShape shape_one() {
  constexpr int LOG2R = fused_log2r(PREC, LOG2N);
  using K = Fused<PREC, LOG2N, LOG2R, false>;
  return FusedShape{LOG2R, K::T, K::TPC, K::TPB, K::SMEM};
}

using LaunchFn = cudaError_t (*)(const void *, void *, int64_t, const uint4 *, const Stage0Twiddles &,
                                 cudaStream_t);
using ShapeFn = FusedShape (*)();
using PrepareFn = cudaError_t (*)();

template <int PREC, int... L>
struct Table {
  static constexpr LaunchFn plain[] = {launch_one<PREC, L, false>...};
  static constexpr LaunchFn scaled[] = {launch_one<PREC, L, true>...};
  static constexpr ShapeFn shape[] = {shape_one<PREC, L>...};
  static constexpr PrepareFn prepare[] = {prepare_one<PREC, L>...};
};

#define DSFFT_LOG2N_LIST 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14
using T32 = Table<kFP32, DSFFT_LOG2N_LIST>;
using T16 = Table<kFP16, DSFFT_LOG2N_LIST>;
using TB16 = Table<kBF16, DSFFT_LOG2N_LIST>;

FusedShape fused_shape(int prec, int log2n) {
  if (log2n < 1 || log2n > kFusedMaxLog2N) return FusedShape{0, 0, 0, 0, 0};
  const int i = log2n - 1;
  return prec == kFP32 ? T32::shape[i]() : prec == kFP16 ? T16::shape[i]() : TB16::shape[i]();
}

cudaError_t prepare_fused(int prec, int log2n) {
  if (log2n < 1 || log2n > kFusedMaxLog2N) return cudaErrorInvalidValue;
  const int i = log2n - 1;
  return prec == kFP32 ? T32::prepare[i]() : prec == kFP16 ? T16::prepare[i]() : TB16::prepare[i]();
}

cudaError_t launch_fused(int prec, int log2n, bool scaled, const void *in, void *out, int64_t batch,
                         const uint4 *table, const Stage0Twiddles &tw0, cudaStream_t stream) {
  if (log2n < 1 || log2n > kFusedMaxLog2N) return cudaErrorInvalidValue;
  const int i = log2n - 1;
  LaunchFn f;
  if (prec == kFP32) f = scaled ? T32::scaled[i] : T32::plain[i];
  else if (prec == kFP16) f = scaled ? T16::scaled[i] : T16::plain[i];
  else f = scaled ? TB16::scaled[i] : TB16::plain[i];
  return f(in, out, batch, table, tw0, stream);
}

}  // namespace dsfft
