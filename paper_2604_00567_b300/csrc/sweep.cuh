// sweep.cuh — FFT for N > 2^14 in two HBM sweeps of grouped radix-2 passes
// (kernel templates; sweep_fp32.cu / sweep_fp16.cu / sweep_bf16.cu
// instantiate them per precision, sweep.cu holds the host dispatch).
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
#pragma once

#include "fused4.cuh"
#include "internal.h"

namespace dsfft {

__device__ __forceinline__ float2 sw_ldcs(const float2 *p) { return __ldcs(p); }
__device__ __forceinline__ uint32_t sw_ldcs(const uint32_t *p) { return __ldcs(reinterpret_cast<const unsigned int *>(p)); }
__device__ __forceinline__ void sw_stcs(float2 *p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void sw_stcs(uint32_t *p, uint32_t v) { __stcs(reinterpret_cast<unsigned int *>(p), v); }

// R4: radix-4 passes (the radix-4 extension, fused4.cuh): stages of whole
// radix-4 passes with 16 points per thread; an odd LS (sweep 1 of an odd
// log2 N) starts with the radix-2 pass of span 1.
// GSHIFT: a block of 2^GSHIFT times fewer groups (at least 4) than the
// default, for launches of at most one block per two SMs (one or a few
// transforms): shorter runs per warp, more blocks.
template <int PREC, int LS, bool SCALED, bool LAST, bool R4 = false, int GSHIFT = 0>
struct Sweep {
  using E = typename Elem<PREC>::T;
  static constexpr int EB = (int)sizeof(E);
  static constexpr int LOG2R = (R4 || PREC == kFP32) ? 4 : 5;
  static constexpr int R = 1 << LOG2R;
  static constexpr int M = 1 << LS;                      // elements per group
  static constexpr int T = M / R;                        // threads per group
  // groups per block: at most 32, and at most 1024 threads (R points each)
  static constexpr int LOG2G_CAP = (LOG2R == 4 ? 14 : 15) - LS;
  static constexpr int LOG2G_DEF = LOG2G_CAP < 5 ? LOG2G_CAP : 5;
  static constexpr int LOG2G_MIN = LOG2G_DEF < 2 ? LOG2G_DEF : 2;
  static constexpr int LOG2G = LOG2G_DEF - GSHIFT > LOG2G_MIN ? LOG2G_DEF - GSHIFT : LOG2G_MIN;
  static constexpr int G = 1 << LOG2G;
  static constexpr int TPB = G * T;
  static_assert(TPB <= 1024, "one block holds at most 1024 threads");
  static constexpr int SMEM_X = G * M * EB;              // exchange buffer
  static constexpr int SMEM_T = LAST ? 0 : M * (G + 1) * EB;  // padded transpose buffer
  // Twiddle staging (sweep 2, radix-2): in a middle register stage where
  // the T threads of a group hold only 2^PL < T distinct j_loc (so T / 2^PL
  // threads load each twiddle), the block loads the stage's G 2^PL
  // (2^RHO - 1) entries once into shared memory after the exchange, and the
  // butterflies read them there.  The first stage (its columns already share
  // every twiddle, and a barrier there would hold up the arithmetic) and a
  // stage whose twiddles are all distinct per thread (the last) read the
  // table as before.
  using TE = typename TwEntry<PREC>::T;
  static __host__ __device__ constexpr bool staged(int pl, int rho) {
    return LAST && !R4 && pl > 0 && (1 << pl) < T && rho >= 4;
  }
  static __host__ __device__ constexpr int tws_entries() {
    int best = 0;
    for (int pl = 0; pl < LS;) {
      const int rho = stage_levels(pl);
      const int cnt = staged(pl, rho) ? G * (1 << pl) * ((1 << rho) - 1) : 0;
      best = cnt > best ? cnt : best;
      pl += rho;
    }
    return best;
  }
  static constexpr int TWS = tws_entries();
  static constexpr int SMEM_XT = SMEM_X + TWS * (int)sizeof(TE);
  static constexpr int SMEM = SMEM_XT > SMEM_T ? SMEM_XT : SMEM_T;
  using S4 = typename std::conditional<PREC == kFP32, float, uint32_t>::type;

  struct Ctx {
    int tid, lg;
    int64_t g;        // group index within the transform
    int64_t jg;       // g mod 2^P0
    int64_t g0;       // first group of the block
    TE *tws;          // staged twiddles (after the exchange buffer)
    int P0;
    uint4 r2e;        // radix-4 plans: radix-2 entry k = 0 (W^0)
    S4 sgn;           // radix-4 plans: sign operand of the +-i d3 terms
  };

  // levels of the register stage starting at local level PL: radix-2
  // sweeps run the remainder (LS mod LOG2R levels) first, where every
  // column of a thread has j_loc = 0 and so shares each twiddle, then
  // stages of LOG2R levels
  static __host__ __device__ constexpr int stage_levels(int pl) {
    return R4 ? r4_stage_levels(LS, LOG2R, pl)
              : (pl == 0 && LS % LOG2R != 0) ? LS % LOG2R : ((LS - pl) < LOG2R ? (LS - pl) : LOG2R);
  }

  // radix-4 passes of one stage: local levels [PL, PL + RHO), global
  // P0 + PL + ...; per-pass radix-4 entries r4_offset(lvl) + (q - 1) L + j
  template <int PL, int RHO>
  static __device__ __forceinline__ void compute4(E (&v)[R], const Ctx &x, const uint4 *__restrict__ twp) {
    constexpr int C = R >> RHO;
    constexpr bool R2 = PL == 0 && (LS & 1);
    constexpr int I0 = R2 ? 1 : 0;
    static_assert((RHO - I0) % 2 == 0, "a stage holds whole radix-4 passes");
    const int par = (x.P0 + LS) & 1;    // log2 N mod 2 (sweep 2 starts at an even or odd level)
    static_for<0, C>([&](auto c_) {
      constexpr int c = decltype(c_)::value;
      if constexpr (c > 0) asm volatile("" ::: "memory");
      const int gl = x.tid + c * T;
      const int64_t jloc = gl & ((1 << PL) - 1);
      if constexpr (R2) {
        constexpr int half = 1 << (RHO - 1);
        static_for<0, half>([&](auto qh_) {
          constexpr int q = decltype(qh_)::value;
          Bfly<PREC, SCALED>::run(v[c + q * C], v[c + (q + half) * C], x.r2e);
        });
      }
      static_for<0, (RHO - I0) / 2>([&](auto k_) {
        constexpr int i = I0 + 2 * decltype(k_)::value;
        constexpr int Q = 1 << (RHO - i - 2);
        const int lvl = x.P0 + PL + i;
        const int64_t L = 1LL << lvl;
        const int64_t tp = ((1LL << lvl) - 1 - par) + x.jg + (jloc << x.P0);
        static_for<0, (1 << i)>([&](auto ql_) {
          constexpr int ql = decltype(ql_)::value;
          const int64_t at = tp + ((int64_t)ql << (PL + x.P0));
          const uint4 e1 = tw_load<PREC>(twp, at);
          const uint4 e2 = tw_load<PREC>(twp, at + L);
          const uint4 e3 = tw_load<PREC>(twp, at + 2 * L);
          constexpr int qtop = bitrev(ql, i) << (RHO - i);
          static_for<0, Q>([&](auto qh_) {
            constexpr int q0 = qtop | decltype(qh_)::value;
            Bfly4<PREC, SCALED>::run(v[c + q0 * C], v[c + (q0 + Q) * C], v[c + (q0 + 2 * Q) * C],
                                     v[c + (q0 + 3 * Q) * C], e1, e2, e3, x.sgn);
          });
        });
      });
    });
  }

  // the staged twiddles of stage (PL, RHO): entry (i, ql, j_loc, lg) at
  // ((2^i - 1 + ql) 2^PL + j_loc) G + lg
  template <int PL, int RHO>
  static __device__ __forceinline__ void load_tws(TE *tws, const Ctx &x, const uint4 *__restrict__ twp) {
    constexpr int J = 1 << PL;
    constexpr int CNT = G * J * ((1 << RHO) - 1);
    const TE *tw = reinterpret_cast<const TE *>(twp);
    for (int e = threadIdx.x; e < CNT; e += TPB) {
      const int lg = e % G;
      const int rest = e / G;
      const int jloc = rest % J;
      const int iq = rest / J;
      const int i = 31 - __clz(iq + 1);
      const int ql = iq + 1 - (1 << i);
      const int64_t idx = ((1LL << (x.P0 + PL + i)) - 1) + (x.g0 + lg) + ((int64_t)jloc << x.P0) +
                          ((int64_t)ql << (PL + x.P0));
      tws[e] = __ldg(tw + idx);
    }
  }

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
          uint4 e;
          if constexpr (staged(PL, RHO))
            e = tw_unpack<PREC>(x.tws[((((1 << i) - 1 + ql) << PL) + (int)jloc) * G + x.lg]);
          else
            e = tw_load<PREC>(twp, tp + ((int64_t)ql << (PL + x.P0)));
          constexpr int qtop = bitrev(ql, i) << (RHO - i);
          static_for<0, half>([&](auto qh_) {
            constexpr int q = qtop | decltype(qh_)::value;
            Bfly<PREC, SCALED>::run(v[c + q * C], v[c + (q + half) * C], e);
          });
        });
      });
    });
  }

  template <int PL>
  static __device__ __forceinline__ void stages(E (&v)[R], E *sm, const Ctx &x, const uint4 *__restrict__ twp,
                                                E *dst, int64_t stride, bool active) {
    constexpr int RHO = stage_levels(PL);
    constexpr int C = R >> RHO;
    if constexpr (PL > 0) {
      static_for<0, R>([&](auto p_) {
        constexpr int p = decltype(p_)::value;
        v[p] = sm[(x.tid + p * T) * G + x.lg];
      });
    }
    if constexpr (R4) compute4<PL, RHO>(v, x, twp);
    else {
      if constexpr (staged(PL, RHO)) {
        // every thread is past the previous stage (the exchange barrier), so
        // the buffer is free
        load_tws<PL, RHO>(x.tws, x, twp);
        __syncthreads();
      }
      compute<PL, RHO>(v, x, twp);
    }
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
        if constexpr (PL > 0) __syncthreads();
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
      if constexpr (PL > 0) __syncthreads();
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
      stages<PL + RHO>(v, sm, x, twp, dst, stride, active);
    }
  }
};

// Sweep 1 reads io.src and writes io.dst; sweep 2 (LAST) reads and writes
// io.dst in place.
// Resident blocks per SM the register allocation must allow (0: the
// compiler's choice).  The unscaled FP16 first sweep in blocks of fewer
// than 1024 threads compiles to 72-84 registers when left alone, so fewer
// than 1024 threads stay resident; the floor of 1024 (64 registers, no
// spills) measured faster on B300 (FP16 inverse, unscaled: 2^18 25.3 ->
// 29.4 %, 2^19 22.1 -> 24.9 % of HBM).  Elsewhere the compiler's choice
// (at most 64 registers already) measured as fast or faster than a stated
// minimum.
template <int PREC, int LS, bool SCALED, bool LAST, bool R4, int GSHIFT>
__host__ __device__ constexpr int sweep_minb() {
  return PREC == kFP16 && !SCALED && !LAST && Sweep<PREC, LS, SCALED, LAST, R4, GSHIFT>::TPB < 1024
             ? 1024 / Sweep<PREC, LS, SCALED, LAST, R4, GSHIFT>::TPB
             : 0;
}
template <int PREC, int LS, bool SCALED, bool LAST, class IO, bool R4 = false, int GSHIFT = 0>
__global__ void __launch_bounds__(Sweep<PREC, LS, SCALED, LAST, R4, GSHIFT>::TPB,
                                  (sweep_minb<PREC, LS, SCALED, LAST, R4, GSHIFT>()))
    sweep_fft_kernel(const IO io, int64_t batch, int log2n, int P0, const uint4 *__restrict__ twp,
                     const uint4 r2e, const uint32_t sgn_bits) {
  using K = Sweep<PREC, LS, SCALED, LAST, R4, GSHIFT>;
  using E = typename K::E;
  // Sweep 2 is launched as a programmatic dependent of sweep 1 on the same
  // stream (its launch is prepared while sweep 1 runs); it waits here until
  // sweep 1 has completed and its stores are visible (a no-op for a launch
  // without that attribute).  Sweep 1 does not trigger the launch early:
  // blocks of sweep 2 placed while sweep 1 still ran measured slower for
  // small batches.
  if constexpr (LAST) asm volatile("griddepcontrol.wait;" ::: "memory");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *sm = reinterpret_cast<E *>(smem_raw);
  const int64_t n = 1LL << log2n;
  const int64_t S = n >> LS;                      // groups per transform = element stride
  // Sweep 1 (jg = 0: every group reads the same few twiddles) runs its
  // blocks transform by transform.  Sweep 2 reads per-group twiddles that
  // together span the whole per-pass table (2^24 FP16: 128 MB, more than L2),
  // so its blocks run group-major: the blocks of one group range in every
  // transform of the batch are consecutive and share each twiddle in L2.
  int64_t tr, g0;
  if constexpr (LAST) {
    const int64_t gb = (int64_t)blockIdx.x / batch;
    tr = (int64_t)blockIdx.x - gb * batch;
    g0 = gb << K::LOG2G;
  } else {
    const int64_t blocks_per_tr = S >> K::LOG2G;
    tr = (int64_t)blockIdx.x / blocks_per_tr;
    g0 = ((int64_t)blockIdx.x - tr * blocks_per_tr) << K::LOG2G;
  }
  typename K::Ctx x;
  x.lg = threadIdx.x & (K::G - 1);
  x.tid = threadIdx.x >> K::LOG2G;
  x.g = g0 + x.lg;
  x.g0 = g0;
  x.tws = reinterpret_cast<typename K::TE *>(smem_raw + K::SMEM_X);
  x.P0 = LAST ? P0 : 0;   // sweep 1 always starts at pass 0: a constant the index arithmetic folds
  x.jg = x.g & ((1LL << x.P0) - 1);
  x.r2e = r2e;
  if constexpr (PREC == kFP32) x.sgn = __uint_as_float(sgn_bits);
  else x.sgn = sgn_bits;
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

// Sweep 2 (LAST) goes out as a programmatic dependent launch of sweep 1
// (cudaLaunchKernelEx with programmatic stream serialization), which hides
// its launch latency behind sweep 1 (measured on B300, batch 1: FP16 2^20
// 7.6 -> 8.6 %, FP32 2^20 10.9 -> 12.5 % of HBM; 256 MiB batches +0.1-0.3
// points); sweep 1 is an ordinary launch.
template <bool LAST, class Kern, class... Args>
cudaError_t launch_sweep_kernel(Kern kern, int64_t blocks, int tpb, int smem, cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(tpb);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = LAST ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int PREC, int LS, bool SCALED, bool LAST, bool R4>
cudaError_t launch_sweep_one(const void *in, void *out, const BatchItem *items, int64_t batch, int log2n,
                                    int P0, const uint4 *twp, const uint4 &r2e, uint32_t sgn, cudaStream_t stream) {
  using K = Sweep<PREC, LS, SCALED, LAST, R4>;
  using E = typename K::E;
  const int64_t S = 1LL << (log2n - LS);
  if (S < K::G) return cudaErrorInvalidValue;
  const int64_t blocks = batch * (S >> K::LOG2G);
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
  if constexpr (!R4) {
    // at most one block per two SMs (one or a few transforms): the
    // narrow-group kernel, which spreads the same work over up to 4x the
    // blocks (measured on B300, batch 1: FP16 2^20 5.0 -> 7.6 %, 2^21 9.0
    // -> 11.8 %, FP32 2^18 3.3 -> 4.4 % of HBM; switching already below one
    // block per SM cost FP16 2^22 and FP32 2^21 2-4 points)
    using KS = Sweep<PREC, LS, SCALED, LAST, R4, 2>;
    if (!items && KS::LOG2G < K::LOG2G && 2 * blocks <= sweep_sm_count())
      return launch_sweep_kernel<LAST>(sweep_fft_kernel<PREC, LS, SCALED, LAST, ContigIO<E>, R4, 2>,
                                       batch * (S >> KS::LOG2G), KS::TPB, KS::SMEM, stream,
                                       ContigIO<E>{static_cast<const E *>(in), static_cast<E *>(out), 1LL << log2n},
                                       batch, log2n, P0, twp, r2e, sgn);
  }
  if (items)
    return launch_sweep_kernel<LAST>(sweep_fft_kernel<PREC, LS, SCALED, LAST, GatherIO<E>, R4>, blocks, K::TPB,
                                     K::SMEM, stream, GatherIO<E>{items}, batch, log2n, P0, twp, r2e, sgn);
  return launch_sweep_kernel<LAST>(sweep_fft_kernel<PREC, LS, SCALED, LAST, ContigIO<E>, R4>, blocks, K::TPB, K::SMEM,
                                   stream, ContigIO<E>{static_cast<const E *>(in), static_cast<E *>(out), 1LL << log2n},
                                   batch, log2n, P0, twp, r2e, sgn);
}

// Carveout: the shared memory of the blocks that can reside (registers,
// threads and shared memory decide); the rest stays L1 for the per-lane
// twiddles (measured on B300: FP16 N = 2^18 28.7 % of HBM against 26.2 %
// with the maximum carveout, FP32 2^18 30.3 against 26.6 %).
template <class F>
cudaError_t prepare_sweep_kernel(F kern, int smem, int tpb) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int nblk = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, kern, tpb, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carveout_for(smem, nblk));
}

template <int PREC, int LS, bool SCALED, bool LAST, bool R4>
cudaError_t prepare_sweep_one() {
  using K = Sweep<PREC, LS, SCALED, LAST, R4>;
  using E = typename K::E;
  cudaError_t e = prepare_sweep_kernel(sweep_fft_kernel<PREC, LS, SCALED, LAST, ContigIO<E>, R4>, K::SMEM, K::TPB);
  if (e != cudaSuccess) return e;
  if constexpr (!R4) {
    using KS = Sweep<PREC, LS, SCALED, LAST, R4, 2>;
    if constexpr (KS::LOG2G < K::LOG2G) {
      e = prepare_sweep_kernel(sweep_fft_kernel<PREC, LS, SCALED, LAST, ContigIO<E>, R4, 2>, KS::SMEM, KS::TPB);
      if (e != cudaSuccess) return e;
    }
  }
  return prepare_sweep_kernel(sweep_fft_kernel<PREC, LS, SCALED, LAST, GatherIO<E>, R4>, K::SMEM, K::TPB);
}

using SweepFn = cudaError_t (*)(const void *, void *, const BatchItem *, int64_t, int, int, const uint4 *,
                                const uint4 &, uint32_t, cudaStream_t);
using SweepPrepFn = cudaError_t (*)();

template <int PREC, bool SCALED, bool LAST, bool R4, int... LSs>
struct SweepTable {
  static constexpr SweepFn launch[] = {launch_sweep_one<PREC, LSs, SCALED, LAST, R4>...};
  static constexpr SweepPrepFn prepare[] = {prepare_sweep_one<PREC, LSs, SCALED, LAST, R4>...};
};

#define DSFFT_LS_LIST 7, 8, 9, 10, 11, 12
template <int PREC, bool R4>
struct SweepSet {
  using A = SweepTable<PREC, false, false, R4, DSFFT_LS_LIST>;
  using B = SweepTable<PREC, true, false, R4, DSFFT_LS_LIST>;
  using C = SweepTable<PREC, false, true, R4, DSFFT_LS_LIST>;
  using D = SweepTable<PREC, true, true, R4, DSFFT_LS_LIST>;
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

// Per-precision entry points (defined by explicit instantiation in
// sweep_<precision>.cu): the launcher of one sweep and the attribute set-up
// of the four kernels (scaled x last) of a sweep length.
template <int PREC>
SweepFn sweep_lookup(bool r4, bool scaled, bool last, int ls) {
  return r4 ? SweepSet<PREC, true>::get(scaled, last, ls) : SweepSet<PREC, false>::get(scaled, last, ls);
}
template <int PREC>
cudaError_t sweep_prepare_ls(bool r4, int ls) {
  return r4 ? SweepSet<PREC, true>::prepare(ls) : SweepSet<PREC, false>::prepare(ls);
}

}  // namespace dsfft
