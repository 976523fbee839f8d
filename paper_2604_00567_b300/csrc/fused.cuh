// fused.cuh — the on-chip transform of N <= 2^14 (register stages with
// shared-memory exchanges), shared by the one-size kernel (fused.cu) and the
// persistent mixed-size batch kernel (batch.cu).
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
// rounded entries; 8-byte compact entries for FP16/BF16, see common.cuh),
// so the lanes of a warp, which hold consecutive j, read consecutive
// entries.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace dsfft {

// Points per thread: 32 four-byte (FP16/BF16) or 16 eight-byte (FP32)
// elements, so a thread's register block is 32 registers and every exchange
// is bank-conflict-free with the one-in-32 padding.  The narrow variant
// halves the block (twice the threads per transform, more stages); the
// autotuner picks between them per size.
__host__ __device__ constexpr int fused_log2r(int prec, int log2n, bool narrow = false) {
  const int wide = prec == kFP32 ? 4 : 5;
  const int r = narrow && (log2n - (wide - 1)) <= 10 ? wide - 1 : wide;   // T = N / R <= 1024
  return log2n < r ? log2n : r;
}

// BT = 0: a block of T threads (one transform) when T >= 64 (FP16/BF16) or
// 128 (FP32), else of 256 threads (several transforms) per launch; BT > 0:
// the block size
// of the persistent batch kernel (T <= BT).
template <int PREC, int LOG2N, int LOG2R, bool SCALED, int BT = 0>
struct Fused {
  using E = typename Elem<PREC>::T;
  static constexpr int N = 1 << LOG2N;
  static constexpr int R = 1 << LOG2R;
  static constexpr int T = N / R;                        // threads per transform
  // one transform per block from T = 64 threads up for FP16/BF16 and from
  // T = 128 for FP32 (measured on B300 against 256-thread blocks of several
  // transforms: FP16 2^12 69.4 -> 71.2 %, 2^11 73.8 -> 75.8 % of HBM, FP32
  // 2^11 96.6 -> 99.7 %; FP32 2^10 in 64-thread blocks 102.6 -> 101.8 %,
  // FP16 2^10 in 32-thread blocks 84.3 -> 80.7 %); smaller transforms share
  // 256-thread blocks
  static constexpr int BTH = BT > 0 ? BT : (T >= (PREC == kFP32 ? 128 : 64) ? T : 256);
  static constexpr int TPC = BTH / T;                    // transforms per block (tile)
  static constexpr int TPB = T * TPC;
  static constexpr int NSTAGES = (LOG2N + LOG2R - 1) / LOG2R;
  // One pad element per 32 four-byte (FP16/BF16) or per 16 eight-byte
  // (FP32) elements: the exchanges are bank-conflict-free (a warp's 8-byte
  // accesses are served 16 lanes per 128-byte wavefront, so 8-byte elements
  // need the pad every 128 bytes).
  static constexpr int PSH = sizeof(E) == 8 ? 4 : 5;
  static constexpr int PADN = N + (N >> PSH);
  static constexpr int SMEM = NSTAGES > 1 ? TPC * PADN * (int)sizeof(E) : 0;
  // Blocks per SM the register allocation must allow: 1024 threads' worth
  // (at most 64 registers per thread), so at least half the SM's warps can
  // be resident.
  static constexpr int MINB = TPB >= 1024 ? 1 : 1024 / TPB;

  static __device__ __forceinline__ int pad(int idx) { return idx + (idx >> PSH); }

  // Exchange barrier of one transform's T threads: a warp barrier when they
  // share a warp, a named barrier per transform when a block holds several
  // multi-warp transforms (so transforms do not wait for each other), else
  // the block barrier.
  static __device__ __forceinline__ void sync(int lt) {
    if constexpr (T <= 32) {
      __syncwarp();
    } else if constexpr (TPC > 1 && TPC <= 15) {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + lt), "r"(T) : "memory");
    } else {
      __syncthreads();
    }
  }
  static_assert(BT == 0 || T <= BT, "a transform fits the block");

  // rho radix-2 passes starting at pass P on the registers of one thread,
  // in depth-first order: pass I on a block of 2^(rho - I) registers, then
  // each half of the block through the remaining passes (the halves are
  // independent after pass I).  Every butterfly keeps its operands and
  // twiddle, so the result is that of the pass-by-pass order; the order
  // keeps fewer twiddles live and lets the loads of one block overlap the
  // arithmetic of the previous one.  tw0(i) returns per-pass entry i for the
  // first stage (the same for every thread): the constant bank or the global
  // table.
  // The butterflies run on columns [CB, CB + CN) of the thread's block
  // (CN > 1 when those columns share j, hence every twiddle).
  template <int P, int RHO, int CB, int CN, int I, int QTOP, class TW0>
  static __device__ __forceinline__ void dfs(E (&v)[R], int j, const uint4 *__restrict__ tw, const TW0 &tw0) {
    constexpr int C = R >> RHO;
    constexpr int half = 1 << (RHO - 1 - I);
    constexpr int ql = bitrev(QTOP >> (RHO - I), I);   // pass P+I, j_full = j + ql 2^P
    uint4 e;
    if constexpr (P == 0) e = tw0(((1 << I) - 1) + ql);
    else e = tw_load<PREC>(tw, ((1 << (P + I)) - 1) + j + (ql << P));
    if constexpr (PREC != kFP32 && P == 0 && half * CN >= 4) {
      // first stage: e is the same in every lane, so a uniform branch on
      // its path runs the selection-free butterflies (packed precisions;
      // measured slower for FP32, whose selection is two selects)
      if (tw_is_cosine<PREC>(e)) {
        static_for<0, CN>([&](auto c_) {
          static_for<0, half>([&](auto qh_) {
            constexpr int c = CB + decltype(c_)::value, q = QTOP | decltype(qh_)::value;
            Bfly<PREC, SCALED>::template run_path<true>(v[c + q * C], v[c + (q + half) * C], e);
          });
        });
      } else {
        static_for<0, CN>([&](auto c_) {
          static_for<0, half>([&](auto qh_) {
            constexpr int c = CB + decltype(c_)::value, q = QTOP | decltype(qh_)::value;
            Bfly<PREC, SCALED>::template run_path<false>(v[c + q * C], v[c + (q + half) * C], e);
          });
        });
      }
    } else {
      static_for<0, CN>([&](auto c_) {
        static_for<0, half>([&](auto qh_) {
          constexpr int c = CB + decltype(c_)::value, q = QTOP | decltype(qh_)::value;
          Bfly<PREC, SCALED>::run(v[c + q * C], v[c + (q + half) * C], e);
        });
      });
    }
    if constexpr (I + 1 < RHO) {
      dfs<P, RHO, CB, CN, I + 1, QTOP>(v, j, tw, tw0);
      dfs<P, RHO, CB, CN, I + 1, QTOP + half>(v, j, tw, tw0);
    }
  }

  template <int P, int RHO, class TW0>
  static __device__ __forceinline__ void compute(E (&v)[R], int tid, const uint4 *__restrict__ tw, const TW0 &tw0) {
    constexpr int C = R >> RHO;   // independent groups per thread
    if constexpr (C > 1 && T % (1 << P) == 0) {
      // column c is group tid + c T, and 2^P divides T: every column has
      // j = tid mod 2^P, so each twiddle is loaded once for all of them
      dfs<P, RHO, 0, C, 0, 0>(v, tid & ((1 << P) - 1), tw, tw0);
    } else {
      static_for<0, C>([&](auto c_) {
        constexpr int c = decltype(c_)::value;
        const int g = tid + c * T;
        const int j = g & ((1 << P) - 1);
        dfs<P, RHO, c, 1, 0, 0>(v, j, tw, tw0);
      });
    }
  }

  // SIN: the first stage's values were read from `sm` (the bulk-copied
  // input), so its exchange must wait until every thread has read them.
  // Stage schedule: stages of LOG2R passes, except that the remainder
  // (LOG2N mod LOG2R passes) forms the second stage when there are three or
  // more: it then starts at pass LOG2R, where 2^LOG2R divides T, so its
  // columns share their twiddles (one load per twiddle instead of one per
  // column; the last stages, with per-thread twiddles, are full).
  static constexpr int REM = LOG2N % LOG2R;
  static constexpr bool REM_SECOND = NSTAGES >= 3 && REM != 0;
  static __host__ __device__ constexpr int stage_start(int s) {
    return REM_SECOND && s >= 2 ? (s - 1) * LOG2R + REM : s * LOG2R;
  }
  static __host__ __device__ constexpr int stage_len(int s) {
    return REM_SECOND ? (s == 1 ? REM : LOG2R)
                      : ((LOG2N - s * LOG2R) < LOG2R ? (LOG2N - s * LOG2R) : LOG2R);
  }

  template <int S, class TW0, bool SIN = false>
  static __device__ __forceinline__ void stages(E (&v)[R], E *sm, int tid, int lt, const uint4 *__restrict__ tw,
                                                const TW0 &tw0, E *dst, bool active) {
    constexpr int P = stage_start(S);
    constexpr int RHO = stage_len(S);
    constexpr int C = R >> RHO;
    if constexpr (S > 0) {
      // pad(tid + p T) = pad(tid) + p T + (p T >> PSH) when 2^PSH | T: one
      // base address plus compile-time offsets
      const int pt = pad(tid);
      static_for<0, R>([&](auto p_) {
        constexpr int p = decltype(p_)::value;
        if constexpr (T % (1 << PSH) == 0) v[p] = sm[pt + p * T + ((p * T) >> PSH)];
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
      if constexpr (S > 0 || SIN) sync(lt);   // previous exchange (or the input) fully read
      // pad(base + off) = pad(base) + off + (off >> PSH) when off is a
      // multiple of 2^PSH (P >= PSH) or base is and off < 2^RHO (P = 0,
      // RHO >= PSH)
      constexpr bool FOLD = P >= PSH || (P == 0 && RHO >= PSH);
      static_for<0, C>([&](auto c_) {
        constexpr int c = decltype(c_)::value;
        const int g = tid + c * T;
        const int base = ((g >> P) << (P + RHO)) + (g & ((1 << P) - 1));
        const int pb = pad(base);
        static_for<0, (1 << RHO)>([&](auto q_) {
          constexpr int q = decltype(q_)::value;
          constexpr int off = bitrev(q, RHO) << P;
          if constexpr (FOLD) sm[pb + off + (off >> PSH)] = v[c + q * C];
          else sm[pad(base + off)] = v[c + q * C];
        });
      });
      sync(lt);
      stages<S + 1, TW0, SIN>(v, sm, tid, lt, tw, tw0, dst, active);
    }
  }

  // One tile: transforms [0, count) of `io` (count <= TPC) by the block's
  // TPB threads; thread threadIdx.x handles transform threadIdx.x / T.
  template <class IO, class TW0>
  static __device__ __forceinline__ void run_tile(const IO &io, int count, const uint4 *__restrict__ tw,
                                                  const TW0 &tw0, E *smem) {
    const int lt = threadIdx.x / T;
    const int tid = threadIdx.x % T;
    const bool active = lt < count;
    E *sm = smem + lt * PADN;
    E v[R];
    if (active) {
      const E *src = io.src(lt);
      static_for<0, R>([&](auto p_) {
        constexpr int p = decltype(p_)::value;
        v[p] = ldcs(src + tid + p * T);
      });
    } else {
      static_for<0, R>([&](auto p_) { v[decltype(p_)::value] = E{}; });
    }
    stages<0>(v, sm, tid, lt, tw, tw0, active ? io.dst(lt) : nullptr, active);
  }
};

}  // namespace dsfft
