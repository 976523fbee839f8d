// sweep.cu — FFT for N > 2^14 in two HBM sweeps of grouped radix-2 passes.
//
// Sweep 1 runs passes [0, LS1) and sweep 2 passes [LS1, m) of the m-pass
// Stockham FFT (Section IV).  Before pass P0 the Stockham array is Z_P0; the
// LS passes starting at P0 only mix, for each group g in [0, S) (S =
// N/2^LS), the 2^LS values Z_P0[g + q S], q in [0, 2^LS), and write them to
// Z_(P0+LS)[(g >> P0) 2^(P0+LS) + (g mod 2^P0) + o 2^P0], o in [0, 2^LS).
// Inside a group the passes are the radix-2 butterflies of the whole
// transform: local pass i at local index j_loc is global pass P0 + i at
// j = (g mod 2^P0) + j_loc 2^P0, whose twiddle is per-pass entry
// 2^(P0+i) - 1 + j.  So both sweeps apply exactly the butterflies of the
// pass-by-pass algorithm and the result is bit-identical to it.
//
// A block holds G consecutive groups of one transform; lanes of a warp take
// consecutive groups, so every global load (and the stores of sweep 2) are
// runs of G consecutive elements.  Groups are exchanged between register
// stages through shared memory laid out [element][group] (conflict-free).
// Sweep 1's output of a block is one contiguous range of G 2^LS elements; it
// is transposed through shared memory so that it is stored in order.
#include "common.cuh"
#include "internal.h"

namespace dsfft {

__device__ __forceinline__ float2 sw_ldcs(const float2 *p) { return __ldcs(p); }
__device__ __forceinline__ uint32_t sw_ldcs(const uint32_t *p) { return __ldcs(reinterpret_cast<const unsigned int *>(p)); }
__device__ __forceinline__ void sw_stcs(float2 *p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void sw_stcs(uint32_t *p, uint32_t v) { __stcs(reinterpret_cast<unsigned int *>(p), v); }

template <int PREC, int LS, bool SCALED, bool LAST>
struct Sweep {
  using E = typename Elem<PREC>::T;
  static constexpr int EB = (int)sizeof(E);
  static constexpr int LOG2R = PREC == kFP32 ? 4 : 5;
  static constexpr int R = 1 << LOG2R;
  static constexpr int M = 1 << LS;                      // elements per group
  static constexpr int T = M / R;                        // threads per group
  // groups per block: at most 32, and a block's groups fill <= 128 KB
  static constexpr int LOG2G_CAP = (PREC == kFP32 ? 14 : 15) - LS;
  static constexpr int LOG2G = LOG2G_CAP < 5 ? LOG2G_CAP : 5;
  static constexpr int G = 1 << LOG2G;
  static constexpr int TPB = G * T;
  static constexpr int SMEM_X = G * M * EB;              // exchange buffer
  static constexpr int SMEM_T = LAST ? 0 : M * (G + 1) * EB;  // padded transpose buffer
  static constexpr int SMEM = SMEM_X > SMEM_T ? SMEM_X : SMEM_T;
  static constexpr int NSTAGES = (LS + LOG2R - 1) / LOG2R;

  struct Ctx {
    int tid, lg;
    int64_t g;        // group index within the transform
    int64_t jg;       // g mod 2^P0
    int P0;
  };

  template <int PL, int RHO>
  static __device__ __forceinline__ void compute(E (&v)[R], const Ctx &x, const uint4 *__restrict__ twp) {
    constexpr int C = R >> RHO;
    static_for<0, C>([&](auto c_) {
      constexpr int c = decltype(c_)::value;
      const int gl = x.tid + c * T;
      const int64_t jloc = gl & ((1 << PL) - 1);
      static_for<0, RHO>([&](auto i_) {
        constexpr int i = decltype(i_)::value;
        constexpr int half = 1 << (RHO - 1 - i);
        const int p = x.P0 + PL + i;                       // global pass
        const int64_t tp = ((1LL << p) - 1) + x.jg + (jloc << x.P0);
        static_for<0, (1 << i)>([&](auto ql_) {
          constexpr int ql = decltype(ql_)::value;
          const uint4 e = tw_load<PREC>(twp, tp + ((int64_t)ql << (PL + x.P0)));
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
  static __device__ __forceinline__ void stages(E (&v)[R], E *sm, const Ctx &x, const uint4 *__restrict__ twp,
                                                E *dst, int64_t stride, bool active) {
    constexpr int PL = S * LOG2R;
    constexpr int RHO = (LS - PL) < LOG2R ? (LS - PL) : LOG2R;
    constexpr int C = R >> RHO;
    if constexpr (S > 0) {
      static_for<0, R>([&](auto p_) {
        constexpr int p = decltype(p_)::value;
        v[p] = sm[(x.tid + p * T) * G + x.lg];
      });
    }
    compute<PL, RHO>(v, x, twp);
    if constexpr (PL + RHO == LS) {
      // local output o = tid + c T + bitrev(q) C T
      if constexpr (LAST) {
        if (active) {
          static_for<0, C>([&](auto c_) {
            constexpr int c = decltype(c_)::value;
            static_for<0, (1 << RHO)>([&](auto q_) {
              constexpr int q = decltype(q_)::value;
              const int o = x.tid + c * T + (bitrev(q, RHO) << PL);
              sw_stcs(dst + x.g + (int64_t)o * stride, v[c + q * C]);
            });
          });
        }
      } else {
        if constexpr (S > 0) __syncthreads();
        static_for<0, C>([&](auto c_) {
          constexpr int c = decltype(c_)::value;
          static_for<0, (1 << RHO)>([&](auto q_) {
            constexpr int q = decltype(q_)::value;
            const int o = x.tid + c * T + (bitrev(q, RHO) << PL);
            sm[o * (G + 1) + x.lg] = v[c + q * C];
          });
        });
        __syncthreads();
        // the block's output is the contiguous range [g0 2^LS, (g0 + G) 2^LS)
        if (active) {
          const int lin0 = threadIdx.x;
#pragma unroll 4
          for (int k = 0; k < G * M / TPB; ++k) {
            const int lin = lin0 + k * TPB;
            const int lg = lin >> LS, o = lin & (M - 1);
            sw_stcs(dst + lin, sm[o * (G + 1) + lg]);
          }
        }
      }
    } else {
      if constexpr (S > 0) __syncthreads();
      static_for<0, C>([&](auto c_) {
        constexpr int c = decltype(c_)::value;
        const int gl = x.tid + c * T;
        const int base = ((gl >> PL) << (PL + RHO)) + (gl & ((1 << PL) - 1));
        static_for<0, (1 << RHO)>([&](auto q_) {
          constexpr int q = decltype(q_)::value;
          sm[(base + (bitrev(q, RHO) << PL)) * G + x.lg] = v[c + q * C];
        });
      });
      __syncthreads();
      stages<S + 1>(v, sm, x, twp, dst, stride, active);
    }
  }
};

// Sweep 1 reads io.src and writes io.dst; sweep 2 (LAST) reads and writes
// io.dst in place.
template <int PREC, int LS, bool SCALED, bool LAST, class IO>
__global__ void __launch_bounds__(Sweep<PREC, LS, SCALED, LAST>::TPB)
    sweep_fft_kernel(const IO io, int64_t batch, int log2n, int P0, const uint4 *__restrict__ twp) {
  using K = Sweep<PREC, LS, SCALED, LAST>;
  using E = typename K::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *sm = reinterpret_cast<E *>(smem_raw);
  const int64_t n = 1LL << log2n;
  const int64_t S = n >> LS;                      // groups per transform = element stride
  const int64_t blocks_per_tr = S >> K::LOG2G;
  const int64_t tr = (int64_t)blockIdx.x / blocks_per_tr;
  const int64_t g0 = ((int64_t)blockIdx.x - tr * blocks_per_tr) << K::LOG2G;
  typename K::Ctx x;
  x.lg = threadIdx.x & (K::G - 1);
  x.tid = threadIdx.x >> K::LOG2G;
  x.g = g0 + x.lg;
  x.P0 = P0;
  x.jg = x.g & ((1LL << P0) - 1);
  const bool active = tr < batch;
  E v[K::R];
  if (active) {
    const E *src = (LAST ? io.dst(tr) : io.src(tr)) + x.g;
    static_for<0, K::R>([&](auto p_) {
      constexpr int p = decltype(p_)::value;
      v[p] = sw_ldcs(src + (int64_t)(x.tid + p * K::T) * S);
    });
  } else {
    static_for<0, K::R>([&](auto p_) { v[decltype(p_)::value] = E{}; });
  }
  // sweep 2 (LAST) writes group g's outputs at g + o S; sweep 1 writes the
  // block's contiguous range starting at g0 2^LS
  E *dst = !active ? nullptr : LAST ? io.dst(tr) : io.dst(tr) + (g0 << LS);
  K::template stages<0>(v, sm, x, twp, dst, S, active);
}

// ---------------------------------------------------------------------------
// dispatch: LS in [7, 12] (N = 2^15 .. 2^24 split as ceil(m/2) + floor(m/2))

template <int PREC, int LS, bool SCALED, bool LAST>
static cudaError_t launch_sweep_one(const void *in, void *out, const BatchItem *items, int64_t batch, int log2n,
                                    int P0, const uint4 *twp, cudaStream_t stream) {
  using K = Sweep<PREC, LS, SCALED, LAST>;
  using E = typename K::E;
  const int64_t S = 1LL << (log2n - LS);
  if (S < K::G) return cudaErrorInvalidValue;
  const int64_t blocks = batch * (S >> K::LOG2G);
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
  if (items) {
    sweep_fft_kernel<PREC, LS, SCALED, LAST, GatherIO<E>><<<(unsigned)blocks, K::TPB, K::SMEM, stream>>>(
        GatherIO<E>{items}, batch, log2n, P0, twp);
  } else {
    sweep_fft_kernel<PREC, LS, SCALED, LAST, ContigIO<E>><<<(unsigned)blocks, K::TPB, K::SMEM, stream>>>(
        ContigIO<E>{static_cast<const E *>(in), static_cast<E *>(out), 1LL << log2n}, batch, log2n, P0, twp);
  }
  return cudaGetLastError();
}

template <class F>
static cudaError_t prepare_sweep_kernel(F kern, int smem) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

template <int PREC, int LS, bool SCALED, bool LAST>
static cudaError_t prepare_sweep_one() {
  using K = Sweep<PREC, LS, SCALED, LAST>;
  using E = typename K::E;
  cudaError_t e = prepare_sweep_kernel(sweep_fft_kernel<PREC, LS, SCALED, LAST, ContigIO<E>>, K::SMEM);
  if (e != cudaSuccess) return e;
  return prepare_sweep_kernel(sweep_fft_kernel<PREC, LS, SCALED, LAST, GatherIO<E>>, K::SMEM);
}

using SweepFn = cudaError_t (*)(const void *, void *, const BatchItem *, int64_t, int, int, const uint4 *,
                                cudaStream_t);
using SweepPrepFn = cudaError_t (*)();

template <int PREC, bool SCALED, bool LAST, int... LSs>
struct SweepTable {
  static constexpr SweepFn launch[] = {launch_sweep_one<PREC, LSs, SCALED, LAST>...};
  static constexpr SweepPrepFn prepare[] = {prepare_sweep_one<PREC, LSs, SCALED, LAST>...};
};

#define DSFFT_LS_LIST 7, 8, 9, 10, 11, 12
template <int PREC>
struct SweepSet {
  using A = SweepTable<PREC, false, false, DSFFT_LS_LIST>;
  using B = SweepTable<PREC, true, false, DSFFT_LS_LIST>;
  using C = SweepTable<PREC, false, true, DSFFT_LS_LIST>;
  using D = SweepTable<PREC, true, true, DSFFT_LS_LIST>;
  static SweepFn get(bool scaled, bool last, int ls) {
    const int i = ls - 7;
    if (!last) return scaled ? B::launch[i] : A::launch[i];
    return scaled ? D::launch[i] : C::launch[i];
  }
  static cudaError_t prepare(int ls) {
    const int i = ls - 7;
    for (SweepPrepFn f : {A::prepare[i], B::prepare[i], C::prepare[i], D::prepare[i]}) {
      cudaError_t e = f();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
};

void sweep_split(int log2n, int *ls1, int *ls2) {
  *ls1 = (log2n + 1) / 2;
  *ls2 = log2n / 2;
}

cudaError_t prepare_sweeps(int prec, int log2n) {
  int ls1, ls2;
  sweep_split(log2n, &ls1, &ls2);
  for (int ls : {ls1, ls2}) {
    cudaError_t e = prec == kFP32 ? SweepSet<kFP32>::prepare(ls)
                    : prec == kFP16 ? SweepSet<kFP16>::prepare(ls) : SweepSet<kBF16>::prepare(ls);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_sweeps(int prec, int log2n, bool scaled, const void *in, void *out, const BatchItem *items,
                          int64_t batch, const uint4 *twp, cudaStream_t stream) {
  int ls1, ls2;
  sweep_split(log2n, &ls1, &ls2);
  if (ls1 < 7 || ls1 > 12 || ls2 < 7 || ls2 > 12) return cudaErrorInvalidValue;
  auto get = [&](bool last, int ls) {
    return prec == kFP32 ? SweepSet<kFP32>::get(scaled, last, ls)
           : prec == kFP16 ? SweepSet<kFP16>::get(scaled, last, ls) : SweepSet<kBF16>::get(scaled, last, ls);
  };
  cudaError_t e = get(false, ls1)(in, out, items, batch, log2n, 0, twp, stream);
  if (e != cudaSuccess) return e;
  return get(true, ls2)(out, out, items, batch, log2n, ls1, twp, stream);
}

}  // namespace dsfft
