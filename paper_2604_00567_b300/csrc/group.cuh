// group.cuh — register-stage execution of LS consecutive radix-2 passes on
// one "group" of 2^LS values (the two phases of the cluster kernel).
//
// Before global pass P0 the Stockham array is Z_P0; the LS passes starting
// at P0 mix, for each group g, the values Z_P0[g + q S] (q in [0, 2^LS),
// S = N / 2^LS).  Local pass i at local index j_loc is global pass P0 + i at
// j = jg + j_loc 2^P0 (jg = g mod 2^P0), whose twiddle is per-pass entry
// 2^(P0+i) - 1 + j (P0 is a compile-time constant; indices fit in int for
// the sizes that use this, N <= 2^17).  A thread keeps R = 2^LOG2R values
// of its group in registers and runs up to LOG2R passes between exchanges;
// thread `tid`
// (of T = 2^LS / R per group) starts with local values tid + p T and ends
// with local outputs o = tid + c T + bitrev(q) C T.
#pragma once

#include "common.cuh"

namespace dsfft {

// TW0_ALL (P0 = 0 only): every pass's twiddles come from tw0 (the whole
// phase-1 table in the constant bank), not only the first stage's.
template <int PREC, int LS, int P0, bool SCALED, bool REM_FIRST = true, bool TW0_ALL = false>
struct GroupPasses {
  using E = typename Elem<PREC>::T;
  static constexpr int LOG2R = PREC == kFP32 ? 4 : 5;
  static constexpr int R = 1 << LOG2R;
  static constexpr int M = 1 << LS;
  static constexpr int T = M / R;

  // Stage schedule: REM_FIRST puts the remainder (LS mod LOG2R passes)
  // first, then stages of LOG2R passes: in the first stage every column of
  // a thread has j_loc = 0, so its columns share each twiddle (one load for
  // all of them), and the later stages hold one column each.  Otherwise
  // stages of LOG2R passes with the remainder last.
  static constexpr int REM = REM_FIRST ? LS % LOG2R : 0;
  static __host__ __device__ constexpr int stage_start(int s) {
    return s == 0 ? 0 : (REM ? REM : LOG2R) + (s - 1) * LOG2R;
  }
  static __host__ __device__ constexpr int stage_len(int s) {
    return s == 0 && REM ? REM : ((LS - stage_start(s)) < LOG2R ? (LS - stage_start(s)) : LOG2R);
  }
  static constexpr int NSTAGES = (LS + LOG2R - 1) / LOG2R;
  static constexpr int LAST_PL = stage_start(NSTAGES - 1);   // first local pass of the last stage

  // tw0(i): per-pass entry i for the first register stage when P0 = 0 (the
  // same for every thread: the constant bank), for every stage with TW0_ALL.  Depth-first order over the
  // stage's passes (as in fused.cuh): pass I on a block of registers, then
  // its two halves, on columns [CB, CB + CN) (CN > 1 when those columns
  // share j_loc, hence every twiddle).
  template <int PL, int RHO, int CB, int CN, int I, int QTOP, class TW0>
  static __device__ __forceinline__ void dfs(E (&v)[R], int jg, int jloc, const uint4 *__restrict__ twp,
                                             const TW0 &tw0) {
    constexpr int C = R >> RHO;
    constexpr int half = 1 << (RHO - 1 - I);
    constexpr int ql = bitrev(QTOP >> (RHO - I), I);
    constexpr int p = P0 + PL + I;                     // global pass
    static_assert(!TW0_ALL || P0 == 0, "the constant-bank table holds the passes from 0");
    uint4 e;
    if constexpr (P0 == 0 && (PL == 0 || TW0_ALL)) e = tw0(((1 << p) - 1) + jloc + (ql << PL));
    else e = tw_load<PREC>(twp, ((1 << p) - 1) + jg + (jloc << P0) + (ql << (PL + P0)));
    if constexpr (PREC != kFP32 && P0 == 0 && PL == 0 && half * CN >= 4) {
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
      dfs<PL, RHO, CB, CN, I + 1, QTOP>(v, jg, jloc, twp, tw0);
      dfs<PL, RHO, CB, CN, I + 1, QTOP + half>(v, jg, jloc, twp, tw0);
    }
  }

  template <int PL, int RHO, class TW0>
  static __device__ __forceinline__ void compute(E (&v)[R], int tid, int jg, const uint4 *__restrict__ twp,
                                                 const TW0 &tw0) {
    constexpr int C = R >> RHO;
    if constexpr (C > 1 && T % (1 << PL) == 0) {
      // column c is local group tid + c T and 2^PL divides T: every column
      // has j_loc = tid mod 2^PL, so each twiddle is loaded once for all
      dfs<PL, RHO, 0, C, 0, 0>(v, jg, tid & ((1 << PL) - 1), twp, tw0);
    } else {
      static_for<0, C>([&](auto c_) {
        constexpr int c = decltype(c_)::value;
        // keep each group's twiddle loads next to their use: hoisting all
        // C (2^RHO - 1) entries ahead would exhaust the registers
        if constexpr (c > 0) asm volatile("" ::: "memory");
        const int gl = tid + c * T;
        const int jloc = gl & ((1 << PL) - 1);
        dfs<PL, RHO, c, 1, 0, 0>(v, jg, jloc, twp, tw0);
      });
    }
  }

  // Runs all LS passes.  xw(idx, value) / xr(idx) write / read local
  // Stockham index idx of this group in the exchange buffer, sync() orders
  // the block between them, out(o, value) receives local output o.  With
  // SYNC_OUT the block synchronises before the outputs (when out() writes
  // the exchange buffer).  first_write() runs once, after the first register
  // stage and before the first write to the exchange buffer or output.
  template <bool SYNC_OUT = false, int S = 0, class TW0, class XW, class XR, class SYNC, class OUT, class FW,
            class PR, class PO>
  static __device__ __forceinline__ void run(E (&v)[R], int tid, int jg, const uint4 *__restrict__ twp,
                                             const TW0 &tw0, XW &&xw, XR &&xr, SYNC &&sync, OUT &&out,
                                             FW &&first_write, PR &&post_read, PO &&pre_out) {
    constexpr int PL = stage_start(S);
    constexpr int RHO = stage_len(S);
    constexpr int C = R >> RHO;
    constexpr bool LAST = PL + RHO == LS;
    if constexpr (S > 0) {
      static_for<0, R>([&](auto p_) {
        constexpr int p = decltype(p_)::value;
        v[p] = xr(tid + p * T);
      });
      if constexpr (LAST) post_read();
    }
    compute<PL, RHO>(v, tid, jg, twp, tw0);
    if constexpr (S == 0) first_write();
    if constexpr (LAST) {
      if constexpr (SYNC_OUT && S > 0) sync();
      pre_out();
      static_for<0, C>([&](auto c_) {
        constexpr int c = decltype(c_)::value;
        static_for<0, (1 << RHO)>([&](auto q_) {
          constexpr int q = decltype(q_)::value;
          // local output o = (tid + c T) + (bitrev(q) << PL), tid + c T < 2^PL
          out(tid + c * T, std::integral_constant<int, (bitrev(q, RHO) << PL)>{}, v[c + q * C]);
        });
      });
    } else {
      if constexpr (S > 0) sync();
      static_for<0, C>([&](auto c_) {
        constexpr int c = decltype(c_)::value;
        const int gl = tid + c * T;
        const int base = ((gl >> PL) << (PL + RHO)) + (gl & ((1 << PL) - 1));
        static_for<0, (1 << RHO)>([&](auto q_) {
          constexpr int q = decltype(q_)::value;
          xw(base + (bitrev(q, RHO) << PL), v[c + q * C]);
        });
      });
      sync();
      run<SYNC_OUT, S + 1>(v, tid, jg, twp, tw0, xw, xr, sync, out, first_write, post_read, pre_out);
    }
  }
};

}  // namespace dsfft
