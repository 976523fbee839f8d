// cluster.cu — one-launch FFT for N = 2^15 .. 2^17 on a thread-block
// cluster: the transform stays on chip across K = 2..8 SMs.
//
// The m passes are split as in the two-sweep path (passes [0, LS1), then
// [LS1, m)), but the intermediate Stockham array Z_LS1 lives in the
// cluster's distributed shared memory instead of HBM:
//   phase 1: CTA `rank` runs passes [0, LS1) on groups g = rank GC1 + lg
//            (values x[g + q M2], q in [0, M1)); its last register stage
//            stores each output Z_LS1[g M1 + o] straight into the shared
//            memory of the CTA that needs it in phase 2 (DSMEM stores:
//            value g of phase-2 group o, owner o / GC2);
//   phase 2: CTA `rank` reads, for groups g' = rank GC2 + lg, the values
//            Z_LS1[g' + q M1] (q in [0, M2)) from its own shared memory,
//            runs passes [LS1, m) and stores X[g' + o M1] to HBM.
// Cluster barrier (A): no CTA writes into another before that CTA has read
// its last phase-1 exchange (split: each thread arrives once it has read,
// computes its last phase-1 stage, and waits just before its remote
// stores).  Then (B), every remote store has landed before phase 2 reads:
// for 4-byte elements (FP16, BF16) the stores are st.async and each
// CTA waits (bounded) on its own mbarrier until its phase-2 bytes have
// arrived, with a relaxed cluster arrive after the stores and the matching
// wait at exit so that no CTA leaves while another may still send to it;
// otherwise plain remote stores and a second cluster barrier.  Every radix-2 butterfly of the pass-by-pass algorithm is executed
// with its own operands and twiddle, so the output is bit-identical to it;
// HBM sees one read and one write.
//
// Shared layout: value o of local group lg at lg (M + 1) + o, M the group
// length (one pad element per group).  Lanes of a warp are consecutive
// groups: their local accesses (same o) fall in distinct banks, every access
// is a per-thread base plus a compile-time offset, and the remote stores of
// a warp (same output o, consecutive g) fill 32 consecutive elements of one
// owner's group.  The first register stage of phase 1 (passes 0..4, the
// same twiddles for every thread) reads its twiddles from the kernel
// parameters (constant bank); for FP32 every phase-1 stage does (the lanes
// of a warp, consecutive groups of one thread index, share each twiddle).
#include <cooperative_groups.h>

#include "group.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace dsfft {

__device__ __forceinline__ float2 cl_ldcs(const float2 *p) { return __ldcs(p); }
__device__ __forceinline__ uint32_t cl_ldcs(const uint32_t *p) { return __ldcs(reinterpret_cast<const unsigned int *>(p)); }
__device__ __forceinline__ void cl_stcs(float2 *p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void cl_stcs(uint32_t *p, uint32_t v) { __stcs(reinterpret_cast<unsigned int *>(p), v); }

// Distributed shared memory: map a local shared address into CTA `rank`'s
// window.
__device__ __forceinline__ uint32_t dsmem_map(uint32_t local_addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
  return r;
}

template <int PREC, int LOG2N, int LOG2K, bool SCALED>
struct Clus {
  using E = typename Elem<PREC>::T;
  static constexpr int N = 1 << LOG2N;
  static constexpr int K = 1 << LOG2K;
  static constexpr int LS1 = (LOG2N + 1) / 2;
  static constexpr int LS2 = LOG2N / 2;
  static constexpr int M1 = 1 << LS1;
  static constexpr int M2 = 1 << LS2;
  static constexpr int GC1 = M2 / K;     // phase-1 groups per CTA
  static constexpr int GC2 = M1 / K;     // phase-2 groups per CTA
  // remainder stage first where measured faster: phase 2 always (its first
  // stage then shares twiddles across columns), phase 1 for FP32 only
  // FP32: every phase-1 twiddle from the kernel parameters (Phase1Twiddles;
  // measured faster, FP32 2^16 39.6 -> 41.9 % of HBM); FP16/BF16: only the
  // first stage's (reading the later ones from the constant bank measured
  // slower there, 41.9 -> 38.7 %)
  static constexpr bool TW0_ALL = PREC == kFP32;
  using TwParams = typename std::conditional<TW0_ALL, Phase1Twiddles, Stage0Twiddles>::type;
  using P1 = GroupPasses<PREC, LS1, 0, SCALED, PREC == kFP32, TW0_ALL>;
  using P2 = GroupPasses<PREC, LS2, LS1, SCALED, true>;
  static constexpr int R = P1::R;
  static constexpr int TPB = GC1 * P1::T;
  static constexpr int S1 = M1 + 1;      // padded group strides
  static constexpr int S2 = M2 + 1;
  static constexpr int SMEM = (GC1 * S1 > GC2 * S2 ? GC1 * S1 : GC2 * S2) * (int)sizeof(E);
  static constexpr int MINB = TPB >= 1024 ? 1 : 1024 / TPB;   // 1024 resident threads: <= 64 registers
  // Phase-1 outputs by st.async counted on the owner's mbarrier (measured
  // faster on B300 for 4-byte elements), else by plain remote stores and a
  // second cluster barrier (FP32: 8-byte st.async measured slower).
  static constexpr bool ASYNC = PREC != kFP32;
  static_assert(GC2 * P2::T == TPB, "both phases use the same threads");
  static_assert(GC1 >= 32 && GC2 >= 32, "a warp must span 32 groups");
  static_assert(K <= 8, "portable cluster size");
  static_assert(LS1 > P1::LOG2R, "phase 1 has an exchange before its last stage");
  static_assert(GC2 >= (1 << P1::LAST_PL), "a phase-1 output's owner depends only on its compile-time part");
  static_assert(!TW0_ALL || (1 << LS1) - 1 <= (int)(sizeof(Phase1Twiddles) / sizeof(uint4)),
                "the phase-1 table fits the parameters");
};

// Asynchronous remote stores whose arrival the destination CTA counts on
// its own mbarrier (complete_tx, in bytes), and the bounded wait on it.
__device__ __forceinline__ void st_async(uint32_t addr, uint32_t v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr), "r"(v),
               "r"(bar)
               : "memory");
}
__device__ __forceinline__ void st_async(uint32_t addr, float2 v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
               "f"(v.x), "f"(v.y), "r"(bar)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// false after about one second (%globaltimer)
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) return false;
  }
}

// Remote stores (volatile: they must stay between the two cluster barriers).
__device__ __forceinline__ void dsmem_st(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void dsmem_st(uint32_t addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}

template <int PREC, int LOG2N, int LOG2K, bool SCALED, class IO>
__global__ void __cluster_dims__(1 << LOG2K, 1, 1)
    __launch_bounds__(Clus<PREC, LOG2N, LOG2K, SCALED>::TPB, Clus<PREC, LOG2N, LOG2K, SCALED>::MINB)
    cluster_fft_kernel(const IO io, int64_t batch, const uint4 *__restrict__ twp,
                       const __grid_constant__ typename Clus<PREC, LOG2N, LOG2K, SCALED>::TwParams tw0, int *status,
                       uint32_t tx_extra) {
  using K = Clus<PREC, LOG2N, LOG2K, SCALED>;
  using E = typename K::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *sm = reinterpret_cast<E *>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int64_t tr = (int64_t)blockIdx.x / K::K;
  (void)batch;
  auto tw0f = [&](int i) { return tw0.e[i]; };
  constexpr int ES = (int)sizeof(E);

  // ASYNC: completes when this CTA's phase-2 input has arrived (armed with
  // its byte count; initialised before cluster barrier A, which every
  // sender passes before its first store)
  __shared__ __align__(8) uint64_t recv_bar;
  const uint32_t bar_local = (uint32_t)__cvta_generic_to_shared(&recv_bar);
  if (K::ASYNC && threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_local) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_local),
                 "r"((uint32_t)(K::GC2 * K::M2 * ES) + tx_extra)
                 : "memory");
  }

  E v[K::R];
  // ---- phase 1: passes [0, LS1); outputs pushed into the owners' phase-2 layout ----
  {
    const int lg = threadIdx.x % K::GC1;
    const int tid = threadIdx.x / K::GC1;
    const int g = rank * K::GC1 + lg;
    const E *src = io.src(tr) + g;
    static_for<0, K::R>([&](auto p_) {
      constexpr int p = decltype(p_)::value;
      v[p] = cl_ldcs(src + (int64_t)(tid + p * K::P1::T) * K::M2);
    });
    // output o = a + b (a = tid + c T1 runtime, b compile-time) is Z_LS1[g M1 + o]:
    // value g of phase-2 group o, held by CTA o / GC2 at local group o mod GC2
    const uint32_t pbase = (uint32_t)__cvta_generic_to_shared(sm) + (uint32_t)((tid * K::S2 + g) * ES);
    uint32_t rbase[K::K], rbar[K::K];
    static_for<0, K::K>([&](auto r_) {
      rbase[decltype(r_)::value] = dsmem_map(pbase, decltype(r_)::value);
      if constexpr (K::ASYNC) rbar[decltype(r_)::value] = dsmem_map(bar_local, decltype(r_)::value);
    });
    E *grp = sm + lg * K::S1;
    K::P1::template run<false>(
        v, tid, 0, twp, tw0f, [&](int idx, E val) { grp[idx] = val; }, [&](int idx) { return grp[idx]; },
        [] { __syncthreads(); },
        [&](int a, auto b_, E val) {
          constexpr int b = decltype(b_)::value;
          constexpr int owner = b / K::GC2;
          constexpr int lgo = b % K::GC2;
          // a = tid + c T1: the c T1 part is folded by the caller into `a`; recover it
          const uint32_t addr = rbase[owner] + (uint32_t)(((a - tid) + lgo) * K::S2 * ES);
          if constexpr (K::ASYNC) st_async(addr, val, rbar[owner]);
          else dsmem_st(addr, val);
        },
        [] {}, [] { cluster_arrive(); }, [] { cluster_wait(); });
  }
  bool ok = true;
  if constexpr (K::ASYNC) {
    cluster_arrive_relaxed();   // lifetime only: no CTA exits before every CTA has sent
    ok = mbar_wait_cluster(bar_local, 0);
  } else {
    cluster_arrive();   // every remote store done (release) ...
    cluster_wait();     // ... and visible before phase 2 reads them
  }
  // ---- phase 2: passes [LS1, m) from local shared memory ----
  if (!K::ASYNC || !__syncthreads_or(!ok)) {
    unsigned tx;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tx));
    const int lg = tx % K::GC2;
    const int tid = tx / K::GC2;
    const int gp = rank * K::GC2 + lg;          // g' in [0, M1)
    E *grp = sm + lg * K::S2;
    static_for<0, K::R>([&](auto p_) {
      constexpr int p = decltype(p_)::value;
      v[p] = grp[tid + p * K::P2::T];
    });
    E *dst = io.dst(tr) + gp;
    K::P2::template run<false>(
        v, tid, gp, twp, tw0f, [&](int idx, E val) { grp[idx] = val; }, [&](int idx) { return grp[idx]; },
        [] { __syncthreads(); },
        [&](int a, auto b_, E val) {
          constexpr int b = decltype(b_)::value;
          cl_stcs(dst + (int64_t)(a + b) * K::M1, val);
        },
        [] { __syncthreads(); }, [] {}, [] {});
  } else if (threadIdx.x == 0) {
    atomicOr(status, 2);   // the input did not arrive in time: this CTA's outputs are not written
  }
  if constexpr (K::ASYNC) cluster_wait();
}

// ---------------------------------------------------------------------------
// dispatch: (prec, log2n) -> cluster size K; -1 when the size is not handled.
// The largest portable cluster whose CTAs still span 32 groups: smaller CTAs
// (more of them per SM) wait less at the cluster barriers (measured on B300:
// FP16 N = 2^16 K = 2 / 4 / 8 -> 26 / 28 / 31 % of HBM).

int cluster_log2k(int prec, int log2n) {
  if (prec == kFP32) return log2n == 15 ? 2 : log2n == 16 ? 3 : -1;
  return log2n == 15 ? 2 : log2n == 16 ? 3 : log2n == 17 ? 3 : -1;
}

// Launched with the load-balancing cluster scheduling policy (the hardware
// may place a cluster's CTAs by SM load rather than spreading them): measured
// on B300, FP16 N = 2^16 41.0 -> 41.8 % of HBM, 2^15 45.5 -> 46.8 %, FP32
// 2^15 49.3 -> 50.1 %, against the default policy.
template <int PREC, int LOG2N, int LOG2K, bool SCALED, class IO>
static cudaError_t launch_cluster_io(const IO &io, int64_t blocks, int64_t batch, const uint4 *twp,
                                     const typename Clus<PREC, LOG2N, LOG2K, SCALED>::TwParams &tw0, int *status,
                                     uint32_t tx_extra, cudaStream_t stream) {
  using K = Clus<PREC, LOG2N, LOG2K, SCALED>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(K::TPB);
  cfg.dynamicSmemBytes = K::SMEM;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
  attr[0].val.clusterSchedulingPolicyPreference = cudaClusterSchedulingPolicyLoadBalancing;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cluster_fft_kernel<PREC, LOG2N, LOG2K, SCALED, IO>, io, batch, twp, tw0, status,
                            tx_extra);
}

template <int PREC, int LOG2N, int LOG2K, bool SCALED>
static cudaError_t launch_cluster_one(const void *in, void *out, const BatchItem *items, int64_t batch,
                                      const uint4 *twp, const Stage0Twiddles &tw0s, const Phase1Twiddles *tw1,
                                      int *status, uint32_t tx_extra, cudaStream_t stream) {
  using K = Clus<PREC, LOG2N, LOG2K, SCALED>;
  using E = typename K::E;
  const int64_t blocks = batch * K::K;
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
  const typename K::TwParams *tw0p;
  if constexpr (K::TW0_ALL) {
    if (!tw1) return cudaErrorInvalidValue;
    tw0p = tw1;
  } else {
    (void)tw1;
    tw0p = &tw0s;
  }
  const typename K::TwParams &tw0 = *tw0p;
  if (items)
    return launch_cluster_io<PREC, LOG2N, LOG2K, SCALED>(GatherIO<E>{items}, blocks, batch, twp, tw0, status,
                                                         tx_extra, stream);
  return launch_cluster_io<PREC, LOG2N, LOG2K, SCALED>(
      ContigIO<E>{static_cast<const E *>(in), static_cast<E *>(out), K::N}, blocks, batch, twp, tw0, status,
      tx_extra, stream);
}

// Carveout: the shared memory of the CTAs the register budget lets reside
// (MINB); the rest of the SM's L1/shared array stays L1 (measured on B300,
// FP16 N = 2^16: 41.1 % of HBM against 37.7 % with the maximum carveout,
// with fewer MIO-throttle and barrier stalls; one CTA fewer per SM for a
// larger L1: 34.3 %).
template <class F>
static cudaError_t prepare_cluster_kernel(F kern, int smem, int nblk) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                              carveout_for(smem, nblk));
}

template <int PREC, int LOG2N, int LOG2K>
static cudaError_t prepare_cluster_one() {
  using K = Clus<PREC, LOG2N, LOG2K, false>;
  using E = typename K::E;
  cudaError_t e;
  if ((e = prepare_cluster_kernel(cluster_fft_kernel<PREC, LOG2N, LOG2K, false, ContigIO<E>>, K::SMEM, K::MINB)) != cudaSuccess) return e;
  if ((e = prepare_cluster_kernel(cluster_fft_kernel<PREC, LOG2N, LOG2K, true, ContigIO<E>>, K::SMEM, K::MINB)) != cudaSuccess) return e;
  if ((e = prepare_cluster_kernel(cluster_fft_kernel<PREC, LOG2N, LOG2K, false, GatherIO<E>>, K::SMEM, K::MINB)) != cudaSuccess) return e;
  return prepare_cluster_kernel(cluster_fft_kernel<PREC, LOG2N, LOG2K, true, GatherIO<E>>, K::SMEM, K::MINB);
}

cudaError_t prepare_cluster(int prec, int log2n) {
  switch (prec * 100 + log2n) {
    case kFP32 * 100 + 15: return prepare_cluster_one<kFP32, 15, 2>();
    case kFP32 * 100 + 16: return prepare_cluster_one<kFP32, 16, 3>();
    case kFP16 * 100 + 15: return prepare_cluster_one<kFP16, 15, 2>();
    case kFP16 * 100 + 16: return prepare_cluster_one<kFP16, 16, 3>();
    case kFP16 * 100 + 17: return prepare_cluster_one<kFP16, 17, 3>();
    case kBF16 * 100 + 15: return prepare_cluster_one<kBF16, 15, 2>();
    case kBF16 * 100 + 16: return prepare_cluster_one<kBF16, 16, 3>();
    case kBF16 * 100 + 17: return prepare_cluster_one<kBF16, 17, 3>();
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_cluster(int prec, int log2n, bool scaled, const void *in, void *out, const BatchItem *items,
                           int64_t batch, const uint4 *twp, const Stage0Twiddles &tw0, const Phase1Twiddles *tw1,
                           int *status, uint32_t tx_extra, cudaStream_t stream) {
  if (!status) return cudaErrorInvalidValue;
#define DSFFT_CL(P, L, LK)                                                                                          \
  case P * 100 + L:                                                                                                 \
    return scaled ? launch_cluster_one<P, L, LK, true>(in, out, items, batch, twp, tw0, tw1, status, tx_extra, stream) \
                  : launch_cluster_one<P, L, LK, false>(in, out, items, batch, twp, tw0, tw1, status, tx_extra, stream);
  switch (prec * 100 + log2n) {
    DSFFT_CL(kFP32, 15, 2)
    DSFFT_CL(kFP32, 16, 3)
    DSFFT_CL(kFP16, 15, 2)
    DSFFT_CL(kFP16, 16, 3)
    DSFFT_CL(kFP16, 17, 3)
    DSFFT_CL(kBF16, 15, 2)
    DSFFT_CL(kBF16, 16, 3)
    DSFFT_CL(kBF16, 17, 3)
  }
#undef DSFFT_CL
  return cudaErrorInvalidValue;
}

}  // namespace dsfft
