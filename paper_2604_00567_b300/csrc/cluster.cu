// cluster.cu — one-launch FFT for N = 2^15 .. 2^17 on a thread-block
// cluster: the transform stays on chip across K = 2..8 SMs.
//
// The m passes are split as in the two-sweep path (passes [0, LS1), then
// [LS1, m)), but the intermediate Stockham array Z_LS1 lives in the
// cluster's distributed shared memory instead of HBM:
//   phase 1: CTA `rank` runs passes [0, LS1) on groups g = rank GC1 + lg
//            (values x[g + q M2], q in [0, M1)) and keeps Z_LS1[g M1 + o]
//            in its own shared memory;
//   cluster barrier;
//   phase 2: CTA `rank` reads, for groups g' = rank GC2 + lg, the values
//            Z_LS1[g' + q M1] (q in [0, M2)) from the shared memory of CTA
//            q / GC1 (DSMEM loads), runs passes [LS1, m) and stores
//            X[g' + o M1] to HBM.
// A second cluster barrier separates the remote reads from the reuse of the
// buffer for phase 2's own exchanges (and from the owner's exit); it is
// split: each thread arrives once its remote reads are done and waits only
// before its first write to the buffer, so the first register stage of
// phase 2 runs while the other CTAs finish their reads.  Every radix-2 butterfly of the
// pass-by-pass algorithm is executed with its own operands and twiddle, so
// the output is bit-identical to it; HBM sees one read and one write.
//
// Shared layout (both phases): value o of local group lg at lg (M + 1) + o,
// M the group length (one pad element per group).  Lanes of a warp are
// consecutive groups: their local accesses (same o) fall in distinct banks,
// every access is a per-thread base plus a compile-time offset, and the
// phase-2 remote reads (same phase-1 group q, consecutive o = g') cover 32
// consecutive elements of the owner's memory.  The first register stage of
// phase 1 (passes 0..4, the same twiddles for every thread) reads its
// twiddles from the kernel parameters (constant bank).
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
// window and load from it.  Volatile: the loads must stay between the two
// cluster barriers.
__device__ __forceinline__ uint32_t dsmem_map(uint32_t local_addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void dsmem_ld(uint32_t addr, uint32_t &v) {
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
}
__device__ __forceinline__ void dsmem_ld(uint32_t addr, float2 &v) {
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
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
  using P1 = GroupPasses<PREC, LS1, 0, SCALED>;
  using P2 = GroupPasses<PREC, LS2, LS1, SCALED>;
  static constexpr int R = P1::R;
  static constexpr int TPB = GC1 * P1::T;
  static constexpr int S1 = M1 + 1;      // padded group strides
  static constexpr int S2 = M2 + 1;
  static constexpr int SMEM = (GC1 * S1 > GC2 * S2 ? GC1 * S1 : GC2 * S2) * (int)sizeof(E);
  static constexpr int MINB = TPB >= 1024 ? 1 : 1024 / TPB;   // 1024 resident threads: <= 64 registers
  static_assert(GC2 * P2::T == TPB, "both phases use the same threads");
  static_assert(GC1 >= 32 && GC2 >= 32, "a warp must span 32 groups");
  static_assert(K <= 8, "portable cluster size");
  static_assert(GC1 % P2::T == 0, "a thread's phase-2 reads never straddle two owners");
};

template <int PREC, int LOG2N, int LOG2K, bool SCALED, class IO>
__global__ void __cluster_dims__(1 << LOG2K, 1, 1)
    __launch_bounds__(Clus<PREC, LOG2N, LOG2K, SCALED>::TPB, Clus<PREC, LOG2N, LOG2K, SCALED>::MINB)
    cluster_fft_kernel(const IO io, int64_t batch, const uint4 *__restrict__ twp,
                       const __grid_constant__ Stage0Twiddles tw0) {
  using K = Clus<PREC, LOG2N, LOG2K, SCALED>;
  using E = typename K::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *sm = reinterpret_cast<E *>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int64_t tr = (int64_t)blockIdx.x / K::K;
  // the grid is exactly batch * K blocks, so every cluster is active
  (void)batch;
  auto tw0f = [&](int i) { return tw0.e[i]; };

  E v[K::R];
  // ---- phase 1: passes [0, LS1) ----
  {
    const int lg = threadIdx.x % K::GC1;
    const int tid = threadIdx.x / K::GC1;
    const int64_t g = (int64_t)rank * K::GC1 + lg;
    const E *src = io.src(tr) + g;
    static_for<0, K::R>([&](auto p_) {
      constexpr int p = decltype(p_)::value;
      v[p] = cl_ldcs(src + (int64_t)(tid + p * K::P1::T) * K::M2);
    });
    E *grp = sm + lg * K::S1;
    K::P1::template run<true>(
        v, tid, 0, twp, tw0f, [&](int idx, E val) { grp[idx] = val; }, [&](int idx) { return grp[idx]; },
        [] { __syncthreads(); }, [&](int o, E val) { grp[o] = val; }, [] {});
  }
  cluster.sync();   // Z_LS1 complete in every CTA of the cluster
  // ---- phase 2: passes [LS1, m) ----
  {
    // opaque copy of the thread index: stops the compiler from sharing
    // phase 1's address arithmetic (and keeping it live) when GC1 == GC2
    unsigned tx;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tx));
    const int lg = tx % K::GC2;
    const int tid = tx / K::GC2;
    const int gp = rank * K::GC2 + lg;          // g' in [0, M1)
    // Z_LS1[g' + q M1] is value o = g' of phase-1 group q, held by CTA
    // q / GC1 at local group q mod GC1; with q = tid + p T2 and T2 | GC1 the
    // owner and the group's offset are compile-time for each p
    const uint32_t local_base =
        (uint32_t)__cvta_generic_to_shared(sm) + (uint32_t)((tid * K::S1 + gp) * (int)sizeof(E));
    uint32_t rbase[K::K];
    static_for<0, K::K>([&](auto r_) { rbase[decltype(r_)::value] = dsmem_map(local_base, decltype(r_)::value); });
    static_for<0, K::R>([&](auto p_) {
      constexpr int p = decltype(p_)::value;
      constexpr int owner = (p * K::P2::T) / K::GC1;
      constexpr int gl0 = (p * K::P2::T) % K::GC1;
      dsmem_ld(rbase[owner] + (uint32_t)(gl0 * K::S1 * (int)sizeof(E)), v[p]);
    });
    // arrive: this thread's remote reads are done (release orders them
    // first); wait: every CTA's reads of this buffer are done
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    E *grp = sm + lg * K::S2;
    E *dst = io.dst(tr) + gp;
    K::P2::template run<false>(
        v, tid, gp, twp, tw0f, [&](int idx, E val) { grp[idx] = val; }, [&](int idx) { return grp[idx]; },
        [] { __syncthreads(); }, [&](int o, E val) { cl_stcs(dst + (int64_t)o * K::M1, val); },
        [] { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); });
  }
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

template <int PREC, int LOG2N, int LOG2K, bool SCALED>
static cudaError_t launch_cluster_one(const void *in, void *out, const BatchItem *items, int64_t batch,
                                      const uint4 *twp, const Stage0Twiddles &tw0, cudaStream_t stream) {
  using K = Clus<PREC, LOG2N, LOG2K, SCALED>;
  using E = typename K::E;
  const int64_t blocks = batch * K::K;
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
  if (items) {
    cluster_fft_kernel<PREC, LOG2N, LOG2K, SCALED, GatherIO<E>><<<(unsigned)blocks, K::TPB, K::SMEM, stream>>>(
        GatherIO<E>{items}, batch, twp, tw0);
  } else {
    cluster_fft_kernel<PREC, LOG2N, LOG2K, SCALED, ContigIO<E>><<<(unsigned)blocks, K::TPB, K::SMEM, stream>>>(
        ContigIO<E>{static_cast<const E *>(in), static_cast<E *>(out), K::N}, batch, twp, tw0);
  }
  return cudaGetLastError();
}

template <class F>
static cudaError_t prepare_cluster_kernel(F kern, int smem) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

template <int PREC, int LOG2N, int LOG2K>
static cudaError_t prepare_cluster_one() {
  using K = Clus<PREC, LOG2N, LOG2K, false>;
  using E = typename K::E;
  cudaError_t e;
  if ((e = prepare_cluster_kernel(cluster_fft_kernel<PREC, LOG2N, LOG2K, false, ContigIO<E>>, K::SMEM)) != cudaSuccess) return e;
  if ((e = prepare_cluster_kernel(cluster_fft_kernel<PREC, LOG2N, LOG2K, true, ContigIO<E>>, K::SMEM)) != cudaSuccess) return e;
  if ((e = prepare_cluster_kernel(cluster_fft_kernel<PREC, LOG2N, LOG2K, false, GatherIO<E>>, K::SMEM)) != cudaSuccess) return e;
  return prepare_cluster_kernel(cluster_fft_kernel<PREC, LOG2N, LOG2K, true, GatherIO<E>>, K::SMEM);
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
                           int64_t batch, const uint4 *twp, const Stage0Twiddles &tw0, cudaStream_t stream) {
#define DSFFT_CL(P, L, LK)                                                                                 \
  case P * 100 + L:                                                                                        \
    return scaled ? launch_cluster_one<P, L, LK, true>(in, out, items, batch, twp, tw0, stream)   \
                  : launch_cluster_one<P, L, LK, false>(in, out, items, batch, twp, tw0, stream);
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
