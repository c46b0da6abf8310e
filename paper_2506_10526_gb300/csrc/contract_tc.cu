// Triple contraction of Eq. (estimator_t) on the 5th-generation tensor cores
// (tcgen05, sm_103a):
//
//   S(l nu3; i nu1, j nu2) = sum_x F_{l,nu3}(x) * P_{nu1 nu2}(x),
//   P(x) = F_{i,nu1}(x) F_{j,nu2}(x)      (pair product, FP32)
//
// Each FP32 operand is split into hi + lo (hi = round(v), lo = round(v - hi));
// three products hi.hi + hi.lo + lo.hi accumulate in FP32 in tensor memory
// (the lo.lo term is below the split's own error).  Two operand formats
// (template parameter F16):
//  * split BF16: 2 x 8 significant bits, FP32 range;
//  * split FP16: 2 x 11 significant bits.  The fields arrive scaled by 2^k_l
//    (|.| < 2^7) as FP16 hi + lo; the producers scale the pair product by
//    2^(k_i + k_j) (|.| < 2^14) before the split.  The FP64 sums multiply by
//    2^-(k_i + k_j + k_l), which is exact.  Per term the error is about
//    3 x 2^-22 of its magnitude, against 3 x 2^-16 for split BF16.
//
// Work unit: a CTA pair (thread-block cluster of 2 on neighbouring SMs) runs
// the two-SM MMA (tcgen05.mma.cta_group::2, M256 N256 K16) on one tile,
// persistent over a static tile list:
//   A = 256 fields (l, nu3) of the third ring: 128 per CTA  -> TMEM lanes
//   B = 512 channel pairs: nu1 in 32 x nu2 in 16, as two N = 256 halves;
//       each CTA makes and holds 128 pairs of each half      -> 2 x 256 TMEM columns
//   K = image pixels in chunks of 32 (64-byte rows, 64B swizzle, K-major)
// Each CTA's tensor memory receives its own 128 fields x all 512 pairs.  Per
// stage a CTA supplies half of the A and half of the B operand, so it reads
// 8 KB of shared memory per MMA (12 KB in the one-SM form) and makes half as
// many pair operands for the same tensor work.
//
// Roles per CTA (352 threads):
//   warp 0      TMA of the A hi/lo fields (boxes of 8, 32 or 128 rows; runs of
//               consecutive field rows take the larger boxes), 3-stage ring
//   warp 1      leader CTA: TMEM allocation and the MMA thread;
//               peer CTA: TMEM allocation and a relay that tells the leader
//               when the peer's stage is loaded (remote mbarrier arrive)
//   warps 2-9   pair producers (FP32 product, hi/lo split, swizzled stores;
//               3-stage ring) and, after the last stage of a tile, epilogue
//   warp 10     TMA of the producers' FP32 rows of F_i and F_j, 3-stage ring
// MMA completions are committed to the mbarriers of both CTAs (multicast).
//
// Epilogue (the producer warps): tcgen05.ld of the CTA's 128 x 512 FP32 tile,
// shared-memory pre-reduction keyed by (ring triple segment, nu1-nu2,
// nu2-nu3) into the idle B buffers, then FP64 global atomics into the
// collapse sums (and, when asked, FP64 atomics into the FULL cube).
//
// Channel-symmetric accumulation (cube blocks S x S x S): a ring triple with a
// repeated ring is symmetric under exchanging the channels of the repeated ring,
// so only one ordering is contracted.  Ring pairs (i, i) keep pairs nu1 <= nu2
// (rectangles wholly below the diagonal are not in the tile list; tiles that
// straddle it carry `diag` and the epilogue drops pairs with nu1 > nu2).  Ring
// triples (i, j, j), i < j, are contracted on the ring pair (j, j) with rows
// (i, nu1) ("swapped" rows, pairs (nu2, nu3) with nu2 <= nu3), so the same
// pair-level cut applies to them; their reduction key and flush map (pa, pb,
// nu1) to the separations (nu1 - nu3, nu2 - nu3) accordingly.  The other
// ordering is filled in from the computed one before the sums are read.
//
// Every mbarrier wait is bounded by %globaltimer.  A wait that gives up sets
// the abort flag of both CTAs of the pair and the plan's error word; all roles
// then run their loops to the end without waiting or issuing work, the TMA
// threads wait (bounded) for their own copies in flight, the MMA thread for
// its last commit, and the pair frees TMEM after a cluster barrier.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "bs_internal.h"

namespace bsi {

namespace {

constexpr int KC = 32;                    // BF16 elements per K chunk = 64 bytes
constexpr int MROWS = 128;                // fields per CTA (256 per pair)
constexpr int P1 = 32, P2 = 16;           // pair rectangle of a tile
constexpr int PHALF = 128;                // pairs per CTA per N-half
constexpr int ASTAGES = 3;                // field-operand ring depth
constexpr int STAGES = 3;                 // pair-operand ring depth
constexpr int RSTAGES = 3;                // FP32 row ring depth
// (three-deep rings measured faster than four-deep ones on the MWA-like
// workload, 291-297 vs 305-308 ms: less shared memory, more L1 per SM)
constexpr int NPROD = 8;                  // producer / epilogue warps
constexpr int NTHREADS = 32 * (3 + NPROD);  // TMA (A), MMA/relay, producers, TMA (rows)
constexpr int GROUP = 8;                  // fields per 8-row box
constexpr int NGROUP = MROWS / GROUP;
constexpr int A_BYTES = MROWS * KC * 2;   // 8 KB (hi or lo)
constexpr int B_BYTES = 2 * PHALF * KC * 2;  // 16 KB (hi or lo): both halves
constexpr int RAW_ROWS = 16 + P2;         // 16 rows of F_i (8 per half), 16 of F_j
constexpr int RAW_BYTES = RAW_ROWS * KC * 4;  // 4 KB: 128-byte rows, 128B swizzle
constexpr int RAW_BOX_BYTES = 8 * KC * 4;     // one TMA box: 8 rows
constexpr int MAX_SEG = 16;
// tensor maps per level: hi/lo with boxes of 8, 32 and 128 field rows, FP32 rows
constexpr int NMAPS = 7;
// a_full, a_empty, pfull per field stage; b_full, b_empty per pair stage; raw_full,
// raw_empty per row stage; acc_full, acc_empty, stall
constexpr int NBAR = 3 * ASTAGES + 2 * STAGES + 2 * RSTAGES + 3;

// Shared-memory layout (the same for both operand formats) and the MMA
// instruction descriptor.
template <bool F16>
struct Lay {
  static constexpr int BP = 2;  // pair operand parts: hi, lo
  static constexpr int RED_CAP = STAGES * BP * B_BYTES / 4;  // floats in the B buffers
  static constexpr int OFF_A = 0;
  static constexpr int OFF_B = OFF_A + ASTAGES * 2 * A_BYTES;
  static constexpr int OFF_RAW = OFF_B + STAGES * BP * B_BYTES;
  static constexpr int OFF_ROW = OFF_RAW + RSTAGES * RAW_BYTES;
  static constexpr int OFF_COL = OFF_ROW + MROWS * 16;  // the tile's column entries (epilogue)
  static constexpr int OFF_SEG = OFF_COL + MROWS * 16;
  static constexpr int OFF_SSC = OFF_SEG + MAX_SEG * 16;  // per-segment FP64 unscale (FP16)
  static constexpr int OFF_RSC = OFF_SSC + MAX_SEG * 8;   // per-row FP64 unscale (FP16)
  static constexpr int OFF_BAR = OFF_RSC + MROWS * 8;
  static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
  static constexpr int SMEM_BYTES = OFF_MISC + 64 + 1024;  // + alignment slack
  static_assert(OFF_RAW % 1024 == 0 && RAW_BYTES % 1024 == 0,
                "128B-swizzled TMA needs 1 KB alignment");
  // instruction descriptor, kind::f16: D f32, A and B bf16 (1) or f16 (0), both
  // K-major, N = 256, M = 256
  static constexpr uint32_t IDESC = (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) |
                                    ((256u >> 3) << 17) | ((256u >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// Shared-memory address of the same variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Arrive on an mbarrier of any CTA of the cluster (address from map_rank).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
template <bool CLUSTER>
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  if (CLUSTER)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
  return ok != 0;
}
// Bounded wait; false on timeout or when the CTA is aborting.  CLUSTER: the
// phase was completed by arrivals from the other CTA of the pair.
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit_ns,
                                          volatile int *abort_flag) {
  if (mbar_try<CLUSTER>(bar, parity)) return true;
  const uint64_t t0 = gtime();
  while (true) {
    if (mbar_try<CLUSTER>(bar, parity)) return true;
    if (*abort_flag) return false;
    if ((long long)(gtime() - t0) > limit_ns) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
template <bool F16>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(Lay<F16>::IDESC), "r"(acc));
}
// Arrive (once) on the mbarrier at this shared offset in both CTAs of the pair
// when every MMA issued so far has completed.
__device__ __forceinline__ void tc_commit_pair(uint32_t bar) {
  const uint16_t mask = 3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
// Shared-memory float reduction (no return value) at a shared-space address.
__device__ __forceinline__ void red_add_shared(uint32_t addr, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
// Byte offset of 16-byte chunk c (0..3) of row r in a 64B-swizzled K-major tile.
__device__ __forceinline__ uint32_t sw64_off(int r, int c) {
  return (uint32_t)(r * 64 + ((c ^ ((r >> 1) & 3)) << 4));
}
// Byte offset of 16-byte chunk c (0..7) of row r in a 128B-swizzled tile of
// 128-byte rows (TMA SWIZZLE_128B on a 1024-byte aligned buffer).
__device__ __forceinline__ uint32_t sw128_off(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}
// BF16 hi/lo split of two FP32 values, packed (element 0 in the low half).
__device__ __forceinline__ void split2(float v0, float v1, uint32_t &hi, uint32_t &lo) {
  __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
  hi = *reinterpret_cast<uint32_t *>(&h);
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
  __nv_bfloat162 l = __floats2bfloat162_rn(v0 - h0, v1 - h1);
  lo = *reinterpret_cast<uint32_t *>(&l);
}
// FP16 hi/lo split of two FP32 values, packed (element 0 in the low half).
__device__ __forceinline__ void split2_f16(float v0, float v1, uint32_t &hi, uint32_t &lo) {
  const __half2 h = __floats2half2_rn(v0, v1);
  hi = *reinterpret_cast<const uint32_t *>(&h);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
  lo = *reinterpret_cast<const uint32_t *>(&l);
}
// 2^k as FP32 (|k| <= 126) and as FP64 (|k| <= 1022), built from the exponent field.
__device__ __forceinline__ float exp2i_f32(int k) { return __uint_as_float((uint32_t)(k + 127) << 23); }
__device__ __forceinline__ double exp2i_f64(int k) {
  return __longlong_as_double((long long)(k + 1023) << 52);
}

template <bool F16>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
    k_contract_tc(const __grid_constant__ TcArgs a) {
  using Ly = Lay<F16>;
  constexpr int OFF_A = Ly::OFF_A, OFF_B = Ly::OFF_B, OFF_RAW = Ly::OFF_RAW, OFF_ROW = Ly::OFF_ROW,
                OFF_COL = Ly::OFF_COL, OFF_SEG = Ly::OFF_SEG, OFF_BAR = Ly::OFF_BAR,
                OFF_MISC = Ly::OFF_MISC, RED_CAP = Ly::RED_CAP, BP = Ly::BP;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();  // 0: leader (issues the MMAs), 1: peer
  const uint32_t sA = smem_u32(sm + OFF_A), sB = smem_u32(sm + OFF_B);
  const uint32_t sBar = smem_u32(sm + OFF_BAR);
  auto a_full = [&](int s) { return sBar + 8 * s; };
  auto a_empty = [&](int s) { return sBar + 8 * (ASTAGES + s); };
  auto pfull = [&](int s) { return sBar + 8 * (2 * ASTAGES + s); };  // peer stage loaded
  auto b_full = [&](int s) { return sBar + 8 * (3 * ASTAGES + s); };
  auto empty = [&](int s) { return sBar + 8 * (3 * ASTAGES + STAGES + s); };  // pair stage free
  auto raw_full = [&](int r) { return sBar + 8 * (3 * ASTAGES + 2 * STAGES + r); };
  auto raw_empty = [&](int r) { return sBar + 8 * (3 * ASTAGES + 2 * STAGES + RSTAGES + r); };
  const uint32_t acc_full = sBar + 8 * (3 * ASTAGES + 2 * STAGES + 2 * RSTAGES),
                 acc_empty = acc_full + 8, stall_bar = acc_full + 16;
  const uint32_t sRaw = smem_u32(sm + OFF_RAW);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + OFF_MISC);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + OFF_MISC + 4);
  const uint32_t peer_abort = map_rank(smem_u32(sm + OFF_MISC + 4), rank ^ 1u);
  const uint32_t acc_empty_lead = map_rank(acc_empty, 0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < ASTAGES; ++s) {
      mbar_init(a_full(s), 1);
      mbar_init(a_empty(s), 1);
      mbar_init(pfull(s), 1);
    }
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(b_full(s), NPROD);
      mbar_init(empty(s), 1);
    }
    for (int r = 0; r < RSTAGES; ++r) {
      mbar_init(raw_full(r), 1);
      mbar_init(raw_empty(r), NPROD);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 2 * NPROD);  // the producer warps of both CTAs (leader's copy is used)
    mbar_init(stall_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  tc_fence_before();
  cluster_sync_all();  // barriers of both CTAs initialised, TMEM allocated
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const long long limit = a.wait_limit_ns;
  const int ntot = a.ntiles;
  const int cid = (int)cluster_id(), ncl = (int)cluster_count();
  const CUtensorMap *maps = reinterpret_cast<const CUtensorMap *>(a.maps);

  auto fail = [&]() {
    *abort_flag = 1;
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(peer_abort), "r"(1) : "memory");
    atomicExch(a.err, 1);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer (A)
    if (lane == 0) {
      uint32_t it = 0;
      int armed[ASTAGES] = {};
      for (int gt = cid; gt < ntot; gt += ncl) {
        const TcTile t = a.tiles[gt];
        const TcGroup &G = a.groups[t.group];
        const CUtensorMap *mg = maps + NMAPS * t.group;
        const int cbase = t.col0 + MROWS * (int)rank;
        int rowc[NGROUP];
#pragma unroll
        for (int g = 0; g < NGROUP; ++g) {
          const int e = cbase + g * GROUP;
          int f = -1;
          if (e < t.ncol) f = G.cols[t.col_off + e].field;
          rowc[g] = f >= 0 ? t.b * G.nf + f : G.batch * G.nf;  // out of range: TMA fills zeros
        }
        // runs of consecutive field rows go in one box of 128 or 32 rows (the same
        // bytes land at the same places as with 8-row boxes)
        int boxk[NGROUP];  // 3: 128 rows, 2: 32 rows, 1: 8 rows, 0: covered
#pragma unroll
        for (int g = 0; g < NGROUP; ++g) boxk[g] = 1;
        bool run128 = true;
#pragma unroll
        for (int g = 1; g < NGROUP; ++g) run128 = run128 && rowc[g] == rowc[0] + 8 * g;
        if (run128) {
          boxk[0] = 3;
#pragma unroll
          for (int g = 1; g < NGROUP; ++g) boxk[g] = 0;
        } else {
#pragma unroll
          for (int g = 0; g < NGROUP; g += 4) {
            const bool r32 = rowc[g + 1] == rowc[g] + 8 && rowc[g + 2] == rowc[g] + 16 &&
                             rowc[g + 3] == rowc[g] + 24;
            if (r32) {
              boxk[g] = 2;
              boxk[g + 1] = boxk[g + 2] = boxk[g + 3] = 0;
            }
          }
        }
        const int k0 = t.kseg * G.kseg_len, k1 = min(G.Kpad, k0 + G.kseg_len);
        for (int kc = k0; kc < k1; kc += KC, ++it) {
          const int s = it % ASTAGES;
          const uint32_t ph = (it / ASTAGES) & 1;
          if (*abort_flag) continue;
          if (!mbar_wait(a_empty(s), ph ^ 1, limit, abort_flag)) {
            fail();
            continue;
          }
          mbar_expect_tx(a_full(s), 2 * A_BYTES);
          ++armed[s];
          const uint32_t dh = sA + s * 2 * A_BYTES, dl = dh + A_BYTES;
#pragma unroll
          for (int g = 0; g < NGROUP; ++g) {
            if (boxk[g] == 0) continue;
            const CUtensorMap *mh = mg + 2 * (boxk[g] - 1);
            tma_load_2d(dh + g * GROUP * 64, mh, kc, rowc[g], a_full(s));
            tma_load_2d(dl + g * GROUP * 64, mh + 1, kc, rowc[g], a_full(s));
          }
        }
      }
      // copies in flight land before the CTA can exit
      for (int s = 0; s < ASTAGES; ++s)
        if (armed[s]) {
          volatile int never = 0;
          if (!mbar_wait(a_full(s), (armed[s] - 1) & 1, limit, &never)) atomicExch(a.err, 1);
        }
    }
  } else if (warp == 1) {
    if (rank == 0 && lane == 0) {
      // ---------------------------------------------------------- MMA issuer (leader)
      uint32_t it = 0, tc = 0;
      uint32_t last_bar = 0, last_par = 0;
      bool committed = false;
      if (a.stall_test) {  // failure-injection test: a barrier nothing arrives at
        if (!mbar_wait(stall_bar, 0, limit, abort_flag)) fail();
      }
      for (int gt = cid; gt < ntot; gt += ncl, ++tc) {
        const TcTile t = a.tiles[gt];
        const TcGroup &G = a.groups[t.group];
        const int k0 = t.kseg * G.kseg_len, k1 = min(G.Kpad, k0 + G.kseg_len);
        const int nst = (k1 - k0) / KC;
        bool ok = !*abort_flag;
        if (ok && !mbar_wait<true>(acc_empty, (tc & 1) ^ 1, limit, abort_flag)) {
          fail();
          ok = false;
        }
        tc_fence_after();
        for (int st = 0; st < nst; ++st, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          const int sa = it % ASTAGES;
          const uint32_t pha = (it / ASTAGES) & 1;
          if (!ok || *abort_flag) {
            ok = false;
            continue;
          }
          if (!mbar_wait(a_full(sa), pha, limit, abort_flag) ||
              !mbar_wait(b_full(s), ph, limit, abort_flag) ||
              !mbar_wait<true>(pfull(sa), pha, limit, abort_flag)) {
            fail();
            ok = false;
            continue;
          }
          tc_fence_after();
          const uint32_t ah = sA + sa * 2 * A_BYTES, al = ah + A_BYTES;
          const uint32_t bh = sB + s * BP * B_BYTES, bl = bh + B_BYTES;
#pragma unroll
          for (int kk = 0; kk < KC / 16; ++kk) {
            const uint64_t dah = sw64_desc(ah + kk * 32), dal = sw64_desc(al + kk * 32);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const uint64_t dbh = sw64_desc(bh + h * PHALF * 64 + kk * 32);
              const uint32_t d = tmem + h * 256;
              tc_mma<F16>(d, dah, dbh, (st == 0 && kk == 0) ? 0u : 1u);
              tc_mma<F16>(d, dah, sw64_desc(bl + h * PHALF * 64 + kk * 32), 1u);
              tc_mma<F16>(d, dal, dbh, 1u);
            }
          }
          tc_commit_pair(a_empty(sa));
          tc_commit_pair(empty(s));
          last_bar = empty(s);
          last_par = ph;
          committed = true;
        }
        if (ok && !*abort_flag) {
          tc_commit_pair(acc_full);
          last_bar = acc_full;
          last_par = tc & 1;
          committed = true;
        }
      }
      if (committed) {  // every MMA issued has finished before TMEM is freed
        volatile int never = 0;
        if (!mbar_wait(last_bar, last_par, limit, &never)) atomicExch(a.err, 1);
      }
    } else if (rank == 1 && lane == 0) {
      // ---------------------------------------------------------- relay (peer)
      // Stage `it` of this CTA is in shared memory (fields by TMA, pairs by the
      // producers): tell the leader's MMA thread.
      const uint32_t pfull_lead0 = map_rank(pfull(0), 0);
      uint32_t it = 0;
      for (int gt = cid; gt < ntot; gt += ncl) {
        const TcTile t = a.tiles[gt];
        const TcGroup &G = a.groups[t.group];
        const int k0 = t.kseg * G.kseg_len, k1 = min(G.Kpad, k0 + G.kseg_len);
        for (int kc = k0; kc < k1; kc += KC, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          const int sa = it % ASTAGES;
          const uint32_t pha = (it / ASTAGES) & 1;
          if (*abort_flag) continue;
          if (!mbar_wait(a_full(sa), pha, limit, abort_flag) ||
              !mbar_wait(b_full(s), ph, limit, abort_flag)) {
            fail();
            continue;
          }
          mbar_arrive_cluster(pfull_lead0 + 8 * sa);
        }
      }
    }
  } else if (warp == 2 + NPROD) {
    // ------------------------------------------------------------ TMA producer (FP32 rows)
    if (lane == 0) {
      uint32_t rit = 0;
      int armed[RSTAGES] = {};
      for (int gt = cid; gt < ntot; gt += ncl) {
        const TcTile t = a.tiles[gt];
        const TcGroup &G = a.groups[t.group];
        const CUtensorMap *map_f = maps + NMAPS * t.group + 6;
        // this CTA's nu1 rows: nu1_0 + 8 rank + [0, 8) and nu1_0 + 16 + 8 rank + [0, 8);
        // rows past the channel block hold other fields (or zeros past the array):
        // their pair columns are dropped in the epilogue
        const int rowi = t.b * G.nf + t.ri * G.nc + t.nu1_0 + 8 * (int)rank;
        const int rowj = t.b * G.nf + t.rj * G.nc + t.nu2_0;
        const int k0 = t.kseg * G.kseg_len, k1 = min(G.Kpad, k0 + G.kseg_len);
        for (int kc = k0; kc < k1; kc += KC, ++rit) {
          const int r = rit % RSTAGES;
          const uint32_t ph = (rit / RSTAGES) & 1;
          if (*abort_flag) continue;
          if (!mbar_wait(raw_empty(r), ph ^ 1, limit, abort_flag)) {
            fail();
            continue;
          }
          mbar_expect_tx(raw_full(r), RAW_BYTES);
          ++armed[r];
          const uint32_t d = sRaw + r * RAW_BYTES;
          tma_load_2d(d, map_f, kc, rowi, raw_full(r));
          tma_load_2d(d + RAW_BOX_BYTES, map_f, kc, rowi + 16, raw_full(r));
          tma_load_2d(d + 2 * RAW_BOX_BYTES, map_f, kc, rowj, raw_full(r));
          tma_load_2d(d + 3 * RAW_BOX_BYTES, map_f, kc, rowj + 8, raw_full(r));
        }
      }
      for (int r = 0; r < RSTAGES; ++r)
        if (armed[r]) {
          volatile int never = 0;
          if (!mbar_wait(raw_full(r), (armed[r] - 1) & 1, limit, &never)) atomicExch(a.err, 1);
        }
    }
  } else {
    // ------------------------------------------------------------ producers + epilogue
    const int pw = warp - 2;  // 0..7
    const int ptid = threadIdx.x - 64;
    const unsigned char *rawb = sm + OFF_RAW;
    int4 *rowinfo = reinterpret_cast<int4 *>(sm + OFF_ROW);  // (C_m, E_m, trip, nu3 | -1)
    int4 *seginfo = reinterpret_cast<int4 *>(sm + OFF_SEG);  // (base, E, trip, hi)
    double *segscale = reinterpret_cast<double *>(sm + Ly::OFF_SSC);  // 2^-(k_i+k_j+k_l)
    double *rowscale = reinterpret_cast<double *>(sm + Ly::OFF_RSC);
    ColEntry *colbuf = reinterpret_cast<ColEntry *>(sm + OFF_COL);
    int *nseg_s = reinterpret_cast<int *>(sm + OFF_MISC + 8);
    int *total_s = reinterpret_cast<int *>(sm + OFF_MISC + 12);
    float *red = reinterpret_cast<float *>(sm + OFF_B);
    // lane -> (row ap, b-offset bq, k-chunk kcq).  Warp pw makes the pairs of this
    // CTA's nu1 rows q = 2pw + ap (q < 8: half 0, nu1 = nu1_0 + 8 rank + q; q >= 8:
    // half 1, nu1 = nu1_0 + 16 + 8 rank + q - 8) with nu2 = bq + 4y (y = 0..3): pair
    // row (q >> 3) 128 + (q & 7) 16 + nu2 of the B operand.  With the 128-byte
    // swizzle the 16 distinct F_j chunks of a load fall on 8 distinct bank groups
    // (two wavefronts, the minimum for 256 bytes); the swizzled operand stores of
    // a warp spread evenly over the banks.
    const int kcq = lane & 3, bq = (lane >> 2) & 3, ap = lane >> 4;
    const int qrow = 2 * pw + ap;
    const int prow0 = (qrow >> 3) * PHALF + (qrow & 7) * P2;
    uint32_t it = 0, rit = 0, tc = 0;
    for (int gt = cid; gt < ntot; gt += ncl, ++tc) {
      const TcTile t = a.tiles[gt];
      const TcGroup &G = a.groups[t.group];
      const int b = t.b;
      const int cbase = t.col0 + MROWS * (int)rank;
      const int k0 = t.kseg * G.kseg_len, k1 = min(G.Kpad, k0 + G.kseg_len);
      // split FP16: the pair product is scaled by 2^(k_i + k_j) — one factor on
      // F_i when it is a finite FP32 power of two, else 2^k_i on F_i and 2^k_j
      // on the product (|k| <= 100 each)
      float sc_i = 1.f, sc_p = 1.f;
      if constexpr (F16) {
        const int ki = G.kexp[b * G.nslot + t.ri], kj = G.kexp[b * G.nslot + t.rj];
        const int kij = ki + kj;
        if (kij >= -120 && kij <= 120) {
          sc_i = exp2i_f32(kij);
        } else {
          sc_i = exp2i_f32(ki);
          sc_p = exp2i_f32(kj);
        }
      }

      for (int kc = k0; kc < k1; kc += KC, ++it, ++rit) {
        const int s = it % STAGES;
        const uint32_t ph = (it / STAGES) & 1;
        const int r = rit % RSTAGES;
        const uint32_t rph = (rit / RSTAGES) & 1;
        bool ok = !*abort_flag;
        if (ok && !mbar_wait(raw_full(r), rph, limit, abort_flag)) {
          fail();
          ok = false;
        }
        // 1 nu1 x 4 nu2 pairs x 8 pixels per lane
        float fi[8], fj[4][8];
        if (ok) {
          const unsigned char *rb = rawb + r * RAW_BYTES;
          {
            const float4 u = *reinterpret_cast<const float4 *>(rb + sw128_off(qrow, 2 * kcq));
            const float4 v = *reinterpret_cast<const float4 *>(rb + sw128_off(qrow, 2 * kcq + 1));
            fi[0] = u.x; fi[1] = u.y; fi[2] = u.z; fi[3] = u.w;
            fi[4] = v.x; fi[5] = v.y; fi[6] = v.z; fi[7] = v.w;
          }
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const int row = 16 + bq + 4 * y;
            const float4 u = *reinterpret_cast<const float4 *>(rb + sw128_off(row, 2 * kcq));
            const float4 v = *reinterpret_cast<const float4 *>(rb + sw128_off(row, 2 * kcq + 1));
            fj[y][0] = u.x; fj[y][1] = u.y; fj[y][2] = u.z; fj[y][3] = u.w;
            fj[y][4] = v.x; fj[y][5] = v.y; fj[y][6] = v.z; fj[y][7] = v.w;
          }
        }
        __syncwarp();
        if (lane == 0 && ok) mbar_arrive(raw_empty(r));
        if (ok && !mbar_wait(empty(s), ph ^ 1, limit, abort_flag)) {
          fail();
          ok = false;
        }
        if (ok) {
          unsigned char *bh = sm + OFF_B + s * BP * B_BYTES;
          unsigned char *bl = bh + B_BYTES;
          if constexpr (F16) {
#pragma unroll
            for (int k = 0; k < 8; ++k) fi[k] *= sc_i;
            if (sc_p != 1.f) {  // tile-uniform: only for extreme field scales
#pragma unroll
              for (int y = 0; y < 4; ++y)
#pragma unroll
                for (int k = 0; k < 8; ++k) fj[y][k] *= sc_p;
            }
          }
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const int p = prow0 + bq + 4 * y;  // pair row
            uint4 H, L;
            if constexpr (F16) {
              split2_f16(fi[0] * fj[y][0], fi[1] * fj[y][1], H.x, L.x);
              split2_f16(fi[2] * fj[y][2], fi[3] * fj[y][3], H.y, L.y);
              split2_f16(fi[4] * fj[y][4], fi[5] * fj[y][5], H.z, L.z);
              split2_f16(fi[6] * fj[y][6], fi[7] * fj[y][7], H.w, L.w);
            } else {
              split2(fi[0] * fj[y][0], fi[1] * fj[y][1], H.x, L.x);
              split2(fi[2] * fj[y][2], fi[3] * fj[y][3], H.y, L.y);
              split2(fi[4] * fj[y][4], fi[5] * fj[y][5], H.z, L.z);
              split2(fi[6] * fj[y][6], fi[7] * fj[y][7], H.w, L.w);
            }
            const uint32_t o = sw64_off(p, kcq);
            *reinterpret_cast<uint4 *>(bh + o) = H;
            *reinterpret_cast<uint4 *>(bl + o) = L;
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncwarp();
        if (lane == 0 && ok) mbar_arrive(b_full(s));
      }

      // ---------------------------------------------------------- epilogue
      bool ok = !*abort_flag;
      if (ok && !mbar_wait(acc_full, tc & 1, limit, abort_flag)) {
        fail();
        ok = false;
      }
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      tc_fence_after();
      if (ptid < MROWS) {  // the tile's column entries (field -2: past the end of the list)
        ColEntry ce{-2, 0, 0, 0};
        if (cbase + ptid < t.ncol) ce = G.cols[t.col_off + cbase + ptid];
        colbuf[ptid] = ce;
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (ptid == 0) {
        // segments of consecutive rows with one ring triple
        int ns = 0, base = 0, m = 0;
        while (m < MROWS) {
          const ColEntry c0 = colbuf[m];
          if (c0.field == -2) break;
          if (c0.field < 0) {
            ++m;
            continue;
          }
          int lo = c0.nu3, hi = c0.nu3, q = m;
          while (q + 1 < MROWS && colbuf[q + 1].field != -2) {
            const ColEntry cn = colbuf[q + 1];
            if (cn.field >= 0 && (cn.trip != c0.trip || cn.swapped != c0.swapped)) break;
            ++q;
            if (cn.field >= 0) {
              lo = min(lo, cn.nu3);
              hi = max(hi, cn.nu3);
            }
          }
          const int E = (P2 - 1) + (hi - lo) + 1;
          const int sw = c0.swapped ? 1 << 16 : 0;  // E < 2^16 (hi - lo < MROWS)
          double usc = 1.0;  // undoes the split-FP16 operand scales of this ring triple
          if constexpr (F16)
            usc = exp2i_f64(-(G.kexp[b * G.nslot + t.ri] + G.kexp[b * G.nslot + t.rj] +
                              G.kexp[b * G.nslot + c0.field / G.nc]));
          if (ns < MAX_SEG) {
            seginfo[ns] = make_int4(base, E | sw, c0.trip, hi);
            segscale[ns] = usc;
          }
          // reduction key of pair (pa, pb) on row r: (dd, e2) with dd = pa - pb + P2 - 1
          // and e2 = hi - nu3 + pb (ordinary row) or e2 = nu1 - lo + P2 - 1 - pb
          // (swapped row); the entry is dd * E + e2 = rowinfo.x + pa E - pb (E -+ 1)
          for (int r = m; r <= q; ++r) {
            const ColEntry cr = colbuf[r];
            rowscale[r] = usc;
            if (cr.field < 0)
              rowinfo[r] = make_int4(0, 0, cr.trip, -1);
            else if (ns >= MAX_SEG)  // no reduction slot: direct atomics (total > RED_CAP)
              rowinfo[r] = make_int4(0, sw, cr.trip, cr.nu3);
            else if (sw)
              rowinfo[r] = make_int4(base + (P2 - 1) * E + (cr.nu3 - lo) + P2 - 1, E | sw, cr.trip,
                                     cr.nu3);
            else
              rowinfo[r] = make_int4(base + (P2 - 1) * E + hi - cr.nu3, E, cr.trip, cr.nu3);
          }
          base += (P1 + P2 - 1) * E;
          ++ns;
          m = q + 1;
        }
        for (int r = m; r < MROWS; ++r) rowinfo[r] = make_int4(0, 0, 0, -1);
        *nseg_s = ns;
        *total_s = (ns <= MAX_SEG) ? base : RED_CAP + 1;
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      const int total = *total_s;
      const bool use_red = G.dsum != nullptr && total <= RED_CAP;
      if (use_red)
        for (int q = ptid; q < total; q += 256) red[q] = 0.f;
      asm volatile("bar.sync 1, 256;" ::: "memory");
      // TMEM: warp -> lane quadrant (warp % 4) and column half
      const int quad = warp & 3, half = pw >> 2;
      const int m = 32 * quad + lane;
      const int4 ri = rowinfo[m];
      const bool row_ok = ri.w >= 0;
      const bool swr = (ri.y >> 16) != 0;  // row (i, nu1) against pairs (nu2, nu3)
      const int Er = ri.y & 0xffff, Fr = swr ? Er + 1 : Er - 1;
      const double rsc = F16 && row_ok ? rowscale[m] : 1.0;
      // the group's fields in registers: the loop below writes memory through
      // atomics, which would otherwise make every field a reload.  Kept pairs:
      // inside the block, and nu1 <= nu2 (pa - pb <= dmax) on a rectangle that
      // straddles the diagonal of a one-ring pair operand
      const int pa_hi = G.nu1_hi - t.nu1_0, pb_hi = G.nu2_hi - t.nu2_0;
      const int dmax = t.diag ? t.nu2_0 - t.nu1_0 : P1;
      const bool fast = use_red && G.out_full == nullptr;  // collapse only: shared reduction
      const double tn = (G.out_full && row_ok) ? G.tnorm[ri.z] * rsc : 0.0;
      const int n2 = 2 * G.nc - 1;
      const uint32_t red_row = smem_u32(red) + 4u * (uint32_t)ri.x;
      for (int ch = 0; ch < 256 / 32; ++ch) {
        uint32_t v[32];
        if (ok) tc_ld32(tmem + ((uint32_t)(32 * quad) << 16) + half * 256 + ch * 32, v);
        if (!ok || !row_ok) continue;
        if (fast) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int p = half * 256 + ch * 32 + j;
            const int pa = p >> 4, pb = p & 15;
            if (pa >= pa_hi || pb >= pb_hi || pa - pb > dmax) continue;
            red_add_shared(red_row + 4u * (uint32_t)(pa * Er - pb * Fr), __uint_as_float(v[j]));
          }
          continue;
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int p = half * 256 + ch * 32 + j;
          const int pa = p >> 4, pb = p & 15;
          const int nu1 = t.nu1_0 + pa, nu2 = t.nu2_0 + pb;
          if (pa >= pa_hi || pb >= pb_hi || pa - pb > dmax) continue;
          const float sv = __uint_as_float(v[j]);
          if (use_red) {
            red_add_shared(red_row + 4u * (uint32_t)(pa * Er - pb * Fr), sv);
          } else if (G.dsum) {
            // separations (nu1 - nu3, nu2 - nu3); a swapped row holds nu1 and the
            // pair (nu2, nu3)
            const int e1 = swr ? ri.w - nu2 : nu1 - ri.w, e2 = swr ? nu1 - nu2 : nu2 - ri.w;
            const long long o = (long long)b * G.dsum_bstride +
                                ((long long)ri.z * n2 + (e1 + G.nc - 1)) * n2 + (e2 + G.nc - 1);
            if (BS_CHK(o, (long long)G.batch * G.dsum_bstride, 31))
              atomicAdd(G.dsum + o, (double)sv * rsc);
          }
          if (G.out_full && !swr) {
            const long long o = (long long)b * G.full_bstride +
                                (((long long)ri.z * G.nc + nu1) * G.nc + nu2) * G.nc + ri.w;
            if (BS_CHK(o, (long long)G.batch * G.full_bstride, 34))
              atomicAdd(G.out_full + o, (double)sv * tn);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0 && ok) mbar_arrive_cluster(acc_empty_lead);
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (use_red && ok) {
        // in the order of the (d1, d2) plane: entry (dd, e2) of a segment sits at
        // d1 = dd + e2 + const, d2 = e2 + const, so plane row r = dd + e2 holds the
        // contiguous run e2 in [max(0, r - (P1 + P2 - 2)), min(E - 1, r)].  One warp
        // per row: coalesced FP64 atomics, a few sectors per row instead of one per
        // entry (walking the buffer linearly would step along a diagonal of the plane)
        const int ns = *nseg_s;
        for (int sg = 0; sg < ns; ++sg) {
          const int4 si = seginfo[sg];  // (base, E | swapped << 16, trip, hi)
          const int E = si.y & 0xffff;
          const double sc = F16 ? segscale[sg] : 1.0;
          if (si.y >> 16) {
            // swapped rows: entry (dd, e2) sits at d1 = nu1 - nu3 = e2 + c1 and
            // d2 = nu2 - nu3 = dd + c2, so plane row e2 holds the contiguous run dd
            const int lo = si.w - (E - P2);
            const int c1 = lo - (P2 - 1) - t.nu2_0 + G.nc - 1;
            const int c2 = t.nu1_0 - t.nu2_0 - (P2 - 1) + G.nc - 1;
            double *plane = G.dsum + (long long)b * G.dsum_bstride + (long long)si.z * n2 * n2;
            const float *rs = red + si.x;
            for (int e2 = pw; e2 < E; e2 += NPROD) {
              const long long row = (long long)(e2 + c1) * n2;
              for (int dd = lane; dd < P1 + P2 - 1; dd += 32) {
                const float v = rs[dd * E + e2];
                if (v == 0.f) continue;
                if (BS_CHK(e2 + c1, n2, 35) && BS_CHK(dd + c2, n2, 36))
                  atomicAdd(plane + row + (dd + c2), F16 ? (double)v * sc : (double)v);
              }
            }
            continue;
          }
          const int d1base = t.nu1_0 - (P2 - 1) - si.w + G.nc - 1;  // d1 index = dd + e2 + d1base
          const int d2base = t.nu2_0 - si.w + G.nc - 1;             // d2 index = e2 + d2base
          double *plane = G.dsum + (long long)b * G.dsum_bstride + (long long)si.z * n2 * n2;
          const float *rs = red + si.x;
          const int nrow = (P1 + P2 - 1) + E - 1;
          for (int r = pw; r < nrow; r += NPROD) {
            const int e2lo = max(0, r - (P1 + P2 - 2)), e2hi = min(E - 1, r);
            const long long row = (long long)(r + d1base) * n2;
            for (int e2 = e2lo + lane; e2 <= e2hi; e2 += 32) {
              const float v = rs[(r - e2) * E + e2];
              if (v == 0.f) continue;
              if (BS_CHK(r + d1base, n2, 32) && BS_CHK(e2 + d2base, n2, 33))
                atomicAdd(plane + row + (e2 + d2base), F16 ? (double)v * sc : (double)v);
            }
          }
        }
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
    }
  }
  tc_fence_before();
  cluster_sync_all();  // all MMAs of the pair have completed (the leader waited for them)
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

template <bool F16>
cudaError_t launch_tc(const TcArgs &a, int nsm, cudaStream_t s) {
  constexpr int SMEM = Lay<F16>::SMEM_BYTES;
  cudaError_t e = smem_optin_once<k_contract_tc<F16>>();
  if (e != cudaSuccess) return e;
  // one CTA pair per two SMs, as many pairs as can be resident at once
  static int max_pairs = 0;
  if (max_pairs == 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * (nsm / 2), 1, 1);
    cfg.blockDim = dim3(NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = SMEM;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, k_contract_tc<F16>, &cfg);
    if (e != cudaSuccess) return e;
    max_pairs = n > 0 ? n : 1;
  }
  const int pairs = std::max(1, std::min({a.ntiles, max_pairs, nsm / 2}));
  k_contract_tc<F16><<<2 * pairs, NTHREADS, SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

int tc_smem_bytes(int f16) { return f16 ? Lay<true>::SMEM_BYTES : Lay<false>::SMEM_BYTES; }

cudaError_t launch_contract_tc(const TcArgs &a, int nsm, cudaStream_t s) {
  if (a.ntiles == 0) return cudaSuccess;
  return a.f16 ? launch_tc<true>(a, nsm, s) : launch_tc<false>(a, nsm, s);
}

}  // namespace bsi
