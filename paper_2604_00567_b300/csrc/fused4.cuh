// fused4.cuh — the on-chip radix-4 transform of N <= 2^14 (radix-4 Stockham
// passes, plus one radix-2 pass at span 1 when log2 N is odd).
//
// A radix-4 pass at span L = 2^l turns the four values
// Z[q N/4 + s L + j] (q = 0..3) into Y[4 s L + p L + j] (p = 0..3): the same
// index map as two radix-2 passes at spans L and 2L.  The register stages of
// fused.cuh therefore carry over unchanged — a thread keeps the 2^rho values
// of a group in the positions the radix-2 passes would leave them in —
// except that a stage holds whole radix-4 passes: stage boundaries fall on
// even levels (odd log2 N: the first stage also holds the radix-2 pass).
// Within a stage, radix-4 pass i (levels i, i + 1 of the stage) combines, for
// each twiddle group ql, registers q0, q0 + Q, q0 + 2Q, q0 + 3Q (Q a quarter
// of the group's block) holding a0..a3, and leaves y0, y2, y1, y3 there.
//
// Twiddles: the per-pass radix-4 table (internal.h r4_offset): level l holds
// three runs of L entries (W^j, W^2j, W^3j of the 4L-point transform, j in
// [0, L)), so the lanes of a warp (consecutive j) read consecutive entries of
// each run.  The first stage (j = 0 for every thread) takes its entries from
// the kernel parameters (constant bank), as does the radix-2 pass (W^0).
#pragma once

#include "fused.cuh"

namespace dsfft {

// Points per thread of the radix-4 kernel: 16 for every precision.  A stage
// holds two radix-4 passes (4 levels), so a larger block (32 points) would
// only split into two independent groups and add register pressure.
__host__ __device__ constexpr int r4_log2r(int log2n) { return log2n < 4 ? log2n : 4; }

// Levels of the radix-4 register stage that starts at level p.
__host__ __device__ constexpr int r4_stage_levels(int log2n, int log2r, int p) {
  const int room = log2n - p;
  const int cap = (p == 0 && (log2n & 1)) ? 1 + 2 * ((log2r - 1) / 2) : 2 * (log2r / 2);
  return room < cap ? room : cap;
}

// First-stage twiddles of a radix-4 plan: the radix-2 entry k = 0 (W^0, for
// the radix-2 pass of odd log2 N) and the first 31 per-pass radix-4 entries.
struct Stage0R4 {
  uint4 r2;
  uint4 e[31];
};

template <int PREC, int LOG2N, int LOG2R, bool SCALED, int BT = 0>
struct Fused4 : Fused<PREC, LOG2N, LOG2R, SCALED, BT> {
  using Base = Fused<PREC, LOG2N, LOG2R, SCALED, BT>;
  using E = typename Base::E;
  using Base::N;
  using Base::R;
  using Base::T;
  using Base::pad;
  using Base::PSH;
  using Base::sync;
  static constexpr int PAR = LOG2N & 1;
  using S = typename std::conditional<PREC == kFP32, float, uint32_t>::type;   // type of the sign operand
  static constexpr bool MULTI_STAGE = r4_stage_levels(LOG2N, LOG2R, 0) < LOG2N;
  static_assert(!MULTI_STAGE || Base::SMEM > 0, "an exchange buffer whenever there are several stages");

  // Radix-4 pass at stage-local level I on the block of registers starting
  // at QTOP (2^(RHO - I) registers), then its four quarter blocks through the
  // remaining passes (they are independent after it): depth-first, as in
  // fused.cuh.
  template <int P, int RHO, int CI, int I, int QTOP>
  static __device__ __forceinline__ void dfs4(E (&v)[R], int j, const uint4 *__restrict__ tw, const Stage0R4 &tw0,
                                              S sgn) {
    constexpr int C = R >> RHO;
    constexpr int lvl = P + I;
    constexpr int L = 1 << lvl;
    constexpr int Q = 1 << (RHO - I - 2);
    constexpr int ql = bitrev(QTOP >> (RHO - I), I);
    uint4 e1, e2, e3;
    if constexpr (P == 0) {
      constexpr int o = (int)r4_offset(lvl, PAR) + ql;
      e1 = tw0.e[o];
      e2 = tw0.e[o + L];
      e3 = tw0.e[o + 2 * L];
    } else {
      const int at = (int)r4_offset(lvl, PAR) + j + (ql << P);
      e1 = tw_load<PREC>(tw, at);
      e2 = tw_load<PREC>(tw, at + L);
      e3 = tw_load<PREC>(tw, at + 2 * L);
    }
    static_for<0, Q>([&](auto qh_) {
      constexpr int q0 = QTOP | decltype(qh_)::value;
      Bfly4<PREC, SCALED>::run(v[CI + q0 * C], v[CI + (q0 + Q) * C], v[CI + (q0 + 2 * Q) * C],
                               v[CI + (q0 + 3 * Q) * C], e1, e2, e3, sgn);
    });
    if constexpr (I + 2 < RHO) {
      dfs4<P, RHO, CI, I + 2, QTOP>(v, j, tw, tw0, sgn);
      dfs4<P, RHO, CI, I + 2, QTOP + Q>(v, j, tw, tw0, sgn);
      dfs4<P, RHO, CI, I + 2, QTOP + 2 * Q>(v, j, tw, tw0, sgn);
      dfs4<P, RHO, CI, I + 2, QTOP + 3 * Q>(v, j, tw, tw0, sgn);
    }
  }

  template <int P, int RHO>
  static __device__ __forceinline__ void compute(E (&v)[R], int tid, const uint4 *__restrict__ tw,
                                                 const Stage0R4 &tw0, S sgn) {
    constexpr bool R2 = P == 0 && PAR == 1;
    constexpr int I0 = R2 ? 1 : 0;
    constexpr int C = R >> RHO;
    static_assert((RHO - I0) % 2 == 0, "a stage holds whole radix-4 passes");
    static_for<0, C>([&](auto c_) {
      constexpr int c = decltype(c_)::value;
      const int g = tid + c * T;
      const int j = g & ((1 << P) - 1);
      if constexpr (R2) {
        constexpr int half = 1 << (RHO - 1);
        static_for<0, half>([&](auto qh_) {
          constexpr int q = decltype(qh_)::value;
          Bfly<PREC, SCALED>::run(v[c + q * C], v[c + (q + half) * C], tw0.r2);
        });
        if constexpr (RHO > 1) {
          dfs4<P, RHO, c, 1, 0>(v, j, tw, tw0, sgn);
          dfs4<P, RHO, c, 1, half>(v, j, tw, tw0, sgn);
        }
      } else {
        dfs4<P, RHO, c, 0, 0>(v, j, tw, tw0, sgn);
      }
    });
  }

  template <int P>
  static __device__ __forceinline__ void stages(E (&v)[R], E *sm, int tid, int lt, const uint4 *__restrict__ tw,
                                                const Stage0R4 &tw0, S sgn, E *dst, bool active) {
    constexpr int RHO = r4_stage_levels(LOG2N, LOG2R, P);
    constexpr int C = R >> RHO;
    if constexpr (P > 0) {
      const int pt = pad(tid);
      static_for<0, R>([&](auto p_) {
        constexpr int p = decltype(p_)::value;
        if constexpr (T % (1 << PSH) == 0) v[p] = sm[pt + p * T + ((p * T) >> PSH)];
        else v[p] = sm[pad(tid + p * T)];
      });
    }
    compute<P, RHO>(v, tid, tw, tw0, sgn);
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
      if constexpr (P > 0) sync(lt);
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
      stages<P + RHO>(v, sm, tid, lt, tw, tw0, sgn, dst, active);
    }
  }

  template <class IO>
  static __device__ __forceinline__ void run_tile(const IO &io, int count, const uint4 *__restrict__ tw,
                                                  const Stage0R4 &tw0, S sgn, E *smem) {
    const int lt = threadIdx.x / T;
    const int tid = threadIdx.x % T;
    const bool active = lt < count;
    E *sm = smem + lt * Base::PADN;
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
    stages<0>(v, sm, tid, lt, tw, tw0, sgn, active ? io.dst(lt) : nullptr, active);
  }
};

}  // namespace dsfft
