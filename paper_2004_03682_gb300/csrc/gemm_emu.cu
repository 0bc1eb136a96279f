// Split-precision emulation of complex-FP64 GEMM on the 5th-generation tensor
// cores (tcgen05, BF16 in, FP32 accumulate in TMEM), for the large contractions
// of step 3 of the TTGT list (Sec. II.B).
//
// Method: error-free splitting in the manner of Ozaki, Ogita, Oishi and Rump
// ("Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 59, 2012).
// Every row of A (column of B) gets a power-of-two exponent E with |x| < 2^E;
// x 2^-E is cut into S integer slices of BETA bits,
//     x 2^-E = sum_s a_s 2^(-BETA s),  a_1 in [-2^BETA, 2^BETA], a_s in [-2^(BETA-1), 2^(BETA-1)],
// each exact in BF16.  The products a_s b_t with s + t <= S + 1 ("diagonals" d =
// s + t) are summed on the tensor cores; every diagonal has its own FP32 TMEM
// accumulator and stays an exact integer over a chunk of KC real K terms, so
// the chunk sums are folded exactly into an int64 per output element:
//     R += sum_d acc_d 2^(BETA (S + 1 - d)),   C = 2^(E_i + F_j - BETA (S + 1)) R.
// Complex operands use the real embedding C' = A' B'' with A' = [Re A | Im A]
// (K' = 2K) and B'' columns (2j, 2j+1) = ([Re B_j; -Im B_j], [Im B_j; Re B_j]).
//
// Kernel: one CTA per 128 x (BN/2 complex) output tile; warp 0 issues 1-D TMA
// bulk copies of pre-tiled slice tiles (the split kernels write them in the
// canonical no-swizzle K-major UMMA layout), warp 1 issues tcgen05.mma (one
// MMA per A slice s covers all diagonals s+1..S+1 by stacking the B slices
// along N), the other 12 (six slices: 16) warps drain the double-buffered TMEM accumulators.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "emu.h"
#include "fpbits.h"

namespace {

constexpr int BM = 128;        // rows per tile (tcgen05 M)
constexpr int KB = 32;         // real K per smem k-block (4 core matrices of 8 bf16)
constexpr int BETA = 7;        // bits per slice
constexpr int KC_BLOCKS = 16;  // k-blocks per exact chunk: KC = 512 real terms
constexpr int EMU_GM = 8;      // default row tiles per group of the GEMM work order (tuned per plan)
#define EXP_ZERO (-1100)       // exponent of an all-zero row / column (any x 2^-EXP_ZERO stays 0)
// alpha encodings for the GEMM epilogue: alpha = +2^k -> k + ALPHA_POS_BIAS,
// alpha = -2^k -> -(k + ALPHA_NEG_BIAS), anything else -> ALPHA_GENERAL
#define ALPHA_GENERAL 0
#define ALPHA_POS_BIAS 64
#define ALPHA_NEG_BIAS 64

template <int S>
struct Shape {
  static constexpr int BN = S <= 5 ? 48 : 32;  // real output columns per tile
  // epilogue: WPQ warps on each TMEM lane quarter, each HW = BN / WPQ real columns of
  // every diagonal (more warps per tile shorten the per-warp chain of TMEM loads and
  // integer folds that bounds short-K products); warps 0 and 1 load and issue MMAs
  static constexpr int WPQ = BN == 32 ? 4 : 3;
  static constexpr int EPI = 4 * WPQ;
  static constexpr int HW = BN / WPQ;
  static constexpr int THREADS = 64 + 32 * EPI;
  static constexpr int A_TILE = BM * KB;       // bf16 elements per slice tile
  static constexpr int B_TILE = BN * KB;
  static constexpr int A_STAGE = S * A_TILE * 2;  // bytes
  static constexpr int B_STAGE = S * B_TILE * 2;
  static constexpr int STAGE = A_STAGE + B_STAGE;
  static constexpr int ACC = S * BN;             // TMEM columns per accumulator buffer
  static constexpr int STAGES = S <= 5 ? 4 : 3;  // as many stages as 227 KB of shared memory holds
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256 + 4096;  // + barriers + a copy of the problem list
  static_assert(SMEM <= 232448, "shared memory");
  static_assert(2 * ACC <= 512, "TMEM");
  static_assert(S * BN <= 256, "MMA N");
  static_assert(BN % 16 == 0, "N multiple of 16");
  static_assert(HW % 8 == 0 && HW * WPQ == BN, "epilogue columns per warp");
};

struct EmuProb {
  int64_t a_src, b_src, c_off;  // complex offsets in the per-instance A, B, C tensors
  int64_t a_sl, b_sl;           // bf16 offsets of the slice tiles (per instance)
  int64_t a_ex, b_ex;           // offsets of the exponent arrays (per instance)
  int64_t ws;                   // split-K partials offset (complex, per instance)
  int32_t M, N, K, Kp;          // Kp = 2 Kh, Kh = K rounded up to 16
  int32_t tiles_m, tiles_n, tile0, nh;    // tile0: first GEMM work item; nh: halves of the K' axis
                                         // (2: complex operands, A' = [Re A | Im A]; 1: real operands,
                                         // A' = Re A and one B row per output column)
  int32_t ksplit, kcb, arows, brows;     // K splits, k-blocks per split (multiple of KC_BLOCKS),
                                         // rows stored per A / B slice tile (a problem with a
                                         // single row / column tile keeps only its 8-row groups
                                         // in use: a prefix of the canonical tile)
  int64_t au0, bu0;  // first split-A / split-B unit of this problem (units: 8-groups of one row / column)
  int64_t red0;      // first output of this problem in the split-K reduction order
  // segmented products (operand sets): k-blocks [0, nkb0) read the slice tiles at
  // a_sl / b_sl, [nkb0, nkb0 + nkb1) those at a_sl1 / b_sl1, the rest those at a_sl2 /
  // b_sl2, each member tiled over its own k-blocks; nkb1 = 0: one segment
  int64_t a_sl1, b_sl1, a_sl2, b_sl2;
  int32_t nkb0, nkb1;
  int64_t rx0, cx0;  // first row- / column-exponent scan item of this problem
};

// Limit of every bounded wait inside k_emu_gemm, and the timeout test hook (see
// exp_test_emu_wait in the header): normally 2 s and off.
struct EmuWaitTest {
  unsigned long long wait_ns;
  int skip_kblock;
  int pad_;
};

// ---------------------------------------------------------------------------
// PTX helpers
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after wait_ns (2 s unless a test shortens it) or when
// another role already gave up, recording the failure; never spins forever.
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort, int* gerr,
                          unsigned long long wait_ns) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 255) == 0) {
      if (*abort) return false;
      if (gtimer() - t0 > wait_ns) {
        *abort = 1;
        atomicExch(gerr, 1);
        return false;
      }
    }
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// canonical K-major, no swizzle: core matrix = 8 rows x 16 B; LBO = step between
// core matrices along K, SBO = step between 8-row groups.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// kind::f16 instruction descriptor: D F32, A/B BF16, both K-major, M = 128.
__device__ __forceinline__ uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(BM >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// offset (in elements) of element (r, k) inside a tile of `rows` x KB, core-matrix order
__device__ __forceinline__ int core_off(int r, int k) { return ((r >> 3) * (KB / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

// ---------------------------------------------------------------------------
// GEMM kernel
// the same for a 128-bit integer: above 63 bits the value is shifted down to 63
// bits with the dropped bits folded into the lowest (sticky) bit, which leaves the
// round-to-nearest-even decision of scaled_i64 unchanged
__device__ __forceinline__ double scaled_i128(__int128 R, int e) {
  const long long lo = (long long)R;
  if ((__int128)lo == R) return scaled_i64(lo, e);
  const bool neg = R < 0;
  unsigned __int128 m = neg ? (unsigned __int128)(-R) : (unsigned __int128)R;
  const unsigned long long hi = (unsigned long long)(m >> 64);
  const int len = 128 - __clzll((long long)hi);  // bit length, > 63
  const int sft = len - 63;
  unsigned long long v = (unsigned long long)(m >> sft);
  if ((m << (128 - sft)) != 0) v |= 1ull;
  const long long sv = (long long)v;
  return scaled_i64(neg ? -sv : sv, e + sft);
}

// K half of the real embedding (each half padded to 16) and the number of
// 32-wide k ranges a half spans (the split kernels' CTA count per tile)
__host__ __device__ __forceinline__ int kh_of(const EmuProb& P) { return P.Kp / P.nh; }
__host__ __device__ __forceinline__ int nkh_of(const EmuProb& P) { return (P.Kp / P.nh + KB - 1) / KB; }
// split-A units (8-groups) per row of a work item: 2 when a half is 16 wide, else 4
__host__ __device__ __forceinline__ int gpr_of(const EmuProb& P) { return kh_of(P) == 16 ? 2 : 4; }
// output columns per tile: BN / 2 complex columns (real embedding), or BN real ones
__host__ __device__ __forceinline__ int ocols_of(const EmuProb& P, int BN) { return P.nh == 2 ? BN / 2 : BN; }

// Index of the last problem whose first unit (tile, split-A or split-B unit) is <= x.
// Those first units do not decrease along the list (a problem with no units shares
// its successor's), so this is the problem that owns unit x.
enum UnitKind { UNIT_TILE, UNIT_A, UNIT_B, UNIT_RX, UNIT_CX };
template <UnitKind U>
__device__ __forceinline__ int64_t first_unit(const EmuProb& q) {
  return U == UNIT_TILE ? int64_t(q.tile0) : U == UNIT_A ? q.au0 : U == UNIT_B ? q.bu0 : U == UNIT_RX ? q.rx0 : q.cx0;
}
template <UnitKind U>
__device__ __forceinline__ int prob_of_unit(const EmuProb* probs, int nprobs, int64_t x) {
  int lo = 0, hi = nprobs - 1;
#pragma unroll 1
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first_unit<U>(probs[mid]) <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One work item of the persistent GEMM: (instance, K split, row tile, column tile).
struct EmuWork {
  int pi, inst, ks, mt, nt, kb0, nkb, nkb_all;
};
// t2p (nullable): the problem of every work item of one instance, for launches whose
// problem list is too long for shared memory (one load instead of a binary search).
__device__ __forceinline__ EmuWork emu_work(const EmuProb* probs, int nprobs, int n_tiles, int w, int GMr,
                                            const int* __restrict__ t2p) {
  EmuWork W;
  W.inst = w / n_tiles;
  const int tile = w - W.inst * n_tiles;
  const int pi = t2p ? t2p[tile] : prob_of_unit<UNIT_TILE>(probs, nprobs, tile);
  const EmuProb& P = probs[pi];
  W.pi = pi;
  int lt = tile - P.tile0;
  const int tmn = P.tiles_m * P.tiles_n;
  W.ks = lt / tmn;
  lt -= W.ks * tmn;
  // grouped order: consecutive items (one wave of CTAs) walk GMr row tiles
  // column by column, so their A and B slice tiles are reused from L2
  const int grp = lt / (GMr * P.tiles_n);
  const int m0 = grp * GMr;
  const int gm = min(GMr, P.tiles_m - m0);
  const int r = lt - m0 * P.tiles_n;
  W.mt = m0 + r % gm;
  W.nt = r / gm;
  W.nkb_all = P.Kp / KB;
  W.kb0 = W.ks * P.kcb;
  W.nkb = min(W.nkb_all, W.kb0 + P.kcb) - W.kb0;
  return W;
}

// Persistent: each CTA walks the work items blockIdx.x, blockIdx.x + gridDim.x, ...
// The stage ring and the two TMEM accumulator buffers run on across items, so
// the epilogue of one tile overlaps the MMAs of the next and the producer
// prefetches across tile boundaries.
template <int S>
__global__ void __launch_bounds__(Shape<S>::THREADS, 1)
    k_emu_gemm(const EmuProb* probs, int nprobs, int n_tiles, int n_work, int gm,
               const __nv_bfloat16* __restrict__ Asl, const __nv_bfloat16* __restrict__ Bsl,
               const int* __restrict__ Aex, const int* __restrict__ Bex, cplx* __restrict__ C, int64_t asl_is,
               int64_t bsl_is, int64_t aex_is, int64_t bex_is, int64_t c_is, cplx alpha, int alpha_e, int beta,
               int* __restrict__ gerr, cplx* __restrict__ ws, int64_t ws_is, EmuWaitTest wt,
               const int* __restrict__ t2p) {
  using SH = Shape<S>;
  constexpr int STAGES = SH::STAGES;
  const unsigned long long wns = wt.wait_ns;
  // test hook (-1 = off): CTA 0 never issues the copies of its k-block skip_g, so the
  // MMA issuer's wait on that stage runs out; nothing is in flight for that stage
  const int skip_g = blockIdx.x == 0 ? wt.skip_kblock : -1;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)((uintptr_t(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = (uint64_t*)(smem + STAGES * SH::STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;
  uint64_t* acce = accf + 2;
  uint64_t* drain = acce + 2;
  uint32_t* tslot = (uint32_t*)(drain + 1);
  volatile int* abort = (volatile int*)(tslot + 1);
  // the problem list, read by every role for every work item, kept in shared memory
  EmuProb* sprobs = (EmuProb*)(smem + STAGES * SH::STAGE + 256);
  constexpr int MAXP = 4096 / int(sizeof(EmuProb));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (nprobs <= MAXP) {
    const long long* src = reinterpret_cast<const long long*>(probs);
    long long* dst = reinterpret_cast<long long*>(sprobs);
    for (int i = threadIdx.x; i < nprobs * int(sizeof(EmuProb) / 8); i += blockDim.x) dst[i] = src[i];
    probs = sprobs;
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&accf[b], 1); mbar_init(&acce[b], SH::EPI); }
    mbar_init(drain, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ---- producer: 1-D TMA bulk copies of the pre-tiled slice tiles
    if (lane == 0) {
      uint32_t g = 0;  // k-blocks issued by this CTA
      bool stop = false;
      for (int w = blockIdx.x; w < n_work && !stop; w += gridDim.x) {
        const EmuWork W = emu_work(probs, nprobs, n_tiles, w, gm, t2p);
        const EmuProb& P = probs[W.pi];
        const int at = P.arows * KB, bt = P.brows * KB;  // stored slice tile sizes (elements)
        const __nv_bfloat16* Ai = Asl + W.inst * asl_is;
        const __nv_bfloat16* Bi = Bsl + W.inst * bsl_is;
        for (int kb = 0; kb < W.nkb; ++kb, ++g) {
          const int st = g % STAGES;
          if (g >= STAGES && !mbar_wait(&empty[st], ((g / STAGES) & 1) ^ 1, abort, gerr, wns)) { stop = true; break; }
          if (int(g) == skip_g) continue;
          // this k-block's slice tiles: its segment's members, tiled over their own k-blocks
          const int kg = W.kb0 + kb;
          int64_t as = P.a_sl, bs = P.b_sl;
          int nk = W.nkb_all, kl = kg;
          if (P.nkb1 > 0) {
            if (kg < P.nkb0) {
              nk = P.nkb0;
            } else if (kg < P.nkb0 + P.nkb1) {
              as = P.a_sl1, bs = P.b_sl1, nk = P.nkb1, kl = kg - P.nkb0;
            } else {
              as = P.a_sl2, bs = P.b_sl2, nk = W.nkb_all - P.nkb0 - P.nkb1, kl = kg - P.nkb0 - P.nkb1;
            }
          }
          const __nv_bfloat16* Ak = Ai + as + (int64_t(W.mt) * nk + kl) * (S * at);
          const __nv_bfloat16* Bk = Bi + bs + (int64_t(W.nt) * nk + kl) * (S * bt);
          uint8_t* sA = smem + st * SH::STAGE;
          uint8_t* sB = sA + SH::A_STAGE;
          mbar_expect_tx(&full[st], uint32_t(S * (at + bt) * 2));
          // rows past the stored prefix keep stale data: they only feed output rows /
          // columns beyond M / N, which the epilogue never stores
          if (P.arows == BM) {
            bulk_g2s(sA, Ak, SH::A_STAGE, &full[st]);
          } else {
            for (int s2 = 0; s2 < S; ++s2) bulk_g2s(sA + s2 * SH::A_TILE * 2, Ak + int64_t(s2) * at, at * 2, &full[st]);
          }
          if (P.brows == SH::BN) {
            bulk_g2s(sB, Bk, SH::B_STAGE, &full[st]);
          } else {
            for (int s2 = 0; s2 < S; ++s2) bulk_g2s(sB + s2 * SH::B_TILE * 2, Bk + int64_t(s2) * bt, bt * 2, &full[st]);
          }
        }
      }
      if (*abort) {
        // let the copies already issued land before the CTA exits
        for (uint32_t k = g > STAGES ? g - STAGES : 0; k < g; ++k) {
          if (int(k) == skip_g) continue;  // never issued
          volatile int dummy = 0;
          mbar_wait(&full[k % STAGES], (k / STAGES) & 1, &dummy, gerr, wns);
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      uint32_t g = 0, gc = 0;  // k-blocks consumed, accumulator chunks started
      bool stop = false;
      for (int w = blockIdx.x; w < n_work && !stop; w += gridDim.x) {
        const EmuWork W = emu_work(probs, nprobs, n_tiles, w, gm, t2p);
        for (int kb = 0; kb < W.nkb; ++kb, ++g) {
          const int st = g % STAGES;
          const bool first = (kb % KC_BLOCKS) == 0;
          const int buf = gc & 1;
          if (first && gc >= 2) {
            if (!mbar_wait(&acce[buf], ((gc >> 1) - 1) & 1, abort, gerr, wns)) { stop = true; break; }
            fence_after();
          }
          if (!mbar_wait(&full[st], (g / STAGES) & 1, abort, gerr, wns)) { stop = true; break; }
          fence_after();
          const uint32_t aA = su32(smem + st * SH::STAGE);
          const uint32_t aB = aA + SH::A_STAGE;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            const uint32_t id = idesc_bf16((S - s) * SH::BN);
            const uint32_t d = tmem + buf * 256 + s * SH::BN;
#pragma unroll
            for (int k16 = 0; k16 < 2; ++k16) {
              const uint64_t ad = sdesc(aA + s * SH::A_TILE * 2 + k16 * 256, 128, 512);
              const uint64_t bd = sdesc(aB + k16 * 256, 128, 512);
              mma_bf16(d, ad, bd, id, (first && s == 0 && k16 == 0) ? 0u : 1u);
            }
          }
          mma_commit(&empty[st]);
          if ((kb % KC_BLOCKS) == KC_BLOCKS - 1 || kb == W.nkb - 1) {
            mma_commit(&accf[buf]);
            ++gc;
          }
        }
      }
    }
  } else {
    // ---- epilogue: SH::EPI warps, one TMEM lane (= output row) per thread.  A warp
    // may only read its own lane quarter (warp % 4); the WPQ warps of a quarter take
    // one HW-column share of the BN columns of every diagonal each.
    constexpr int HW = SH::HW;  // real columns per epilogue warp
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    uint32_t gc = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < n_work && ok; w += gridDim.x) {
      const EmuWork W = emu_work(probs, nprobs, n_tiles, w, gm, t2p);
      const EmuProb& P = probs[W.pi];
      const int nchunks = (W.nkb + KC_BLOCKS - 1) / KC_BLOCKS;
      long long R[HW];
#pragma unroll
      for (int j = 0; j < HW; ++j) R[j] = 0;
      // 8-column groups of this warp that hold outputs (warp-uniform): none when the
      // warp's 32 rows are all past M
      const bool cpx = P.nh == 2;  // complex: output column pairs (Re, Im); real: one per column
      const int ncv = cpx ? 2 * min(P.N - W.nt * (SH::BN / 2), SH::BN / 2) : min(P.N - W.nt * SH::BN, SH::BN);
      int nv8 = min(max((ncv - h * HW + 7) / 8, 0), HW / 8);
      if (W.mt * BM + q * 32 >= P.M) nv8 = 0;
      // the tile's row / column exponents, loaded before the accumulators are ready
      const int gi = W.mt * BM + row;
      // first output column of this warp
      const int j0 = cpx ? W.nt * (SH::BN / 2) + h * (HW / 2) : W.nt * SH::BN + h * HW;
      const int ei = gi < P.M ? Aex[W.inst * aex_is + P.a_ex + gi] : 0;
      int fj[HW / 2];  // complex columns' exponents (real columns load theirs at the store)
#pragma unroll
      for (int jj = 0; jj < HW / 2; ++jj)
        fj[jj] = (cpx && gi < P.M && j0 + jj < P.N) ? Bex[W.inst * bex_is + P.b_ex + j0 + jj] : 0;
      for (int ch = 0; ch < nchunks; ++ch, ++gc) {
        const int buf = gc & 1;
        if (!mbar_wait(&accf[buf], (gc >> 1) & 1, abort, gerr, wns)) { ok = false; break; }
        fence_after();
        // the diagonals in groups of 32 staged values: every load of a group is issued
        // before its one wait (the waits, not the conversions, bound the epilogue of
        // short products); each diagonal is still added in the same order
        constexpr int DG = 32 / HW < S ? 32 / HW : S;
#pragma unroll
        for (int d0 = 0; d0 < S; d0 += DG) {
          uint32_t v[DG][HW];
#pragma unroll
          for (int dd = 0; dd < DG; ++dd)
#pragma unroll
            for (int j8 = 0; j8 < HW / 8; ++j8)
              if (d0 + dd < S && j8 < nv8)
                tmem_ld8(tmem + (uint32_t(q * 32) << 16) + buf * 256 + (d0 + dd) * SH::BN + h * HW + j8 * 8,
                         v[dd] + j8 * 8);
          tmem_wait_ld();
#pragma unroll
          for (int dd = 0; dd < DG; ++dd) {
            if (d0 + dd >= S) break;
            const int shift = BETA * (S - 1 - (d0 + dd));
#pragma unroll
            for (int u = 0; u < HW; ++u)
              if (u < nv8 * 8) R[u] += (long long)__float2int_rn(__uint_as_float(v[dd][u])) << shift;
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[buf]);
      }
      if (!ok) break;
      if (gi >= P.M) continue;
      if (!cpx) {  // real operands: column u of the warp is output column j0 + u, imaginary part 0
        if (P.ksplit > 1) {
          longlong2* Wp = reinterpret_cast<longlong2*>(ws + W.inst * ws_is + P.ws) + int64_t(W.ks) * P.M * P.N +
                          int64_t(gi) * P.N;
#pragma unroll
          for (int u = 0; u < HW; ++u)
            if (j0 + u < P.N) Wp[j0 + u] = make_longlong2(R[u], 0ll);
        } else {
          cplx* Crow = C + W.inst * c_is + P.c_off + int64_t(gi) * P.N;
#pragma unroll
          for (int u = 0; u < HW; ++u) {
            const int gj = j0 + u;
            if (gj < P.N) {
              const int e = ei + Bex[W.inst * bex_is + P.b_ex + gj] - BETA * (S + 1);
              double vr, vi;
              if (alpha_e != ALPHA_GENERAL) {
                const int k = alpha_e < 0 ? -alpha_e - ALPHA_NEG_BIAS : alpha_e - ALPHA_POS_BIAS;
                vr = scaled_i64(alpha_e < 0 ? -R[u] : R[u], e + k);
                vi = 0.0;
              } else {
                const double re = scaled_i64(R[u], e);
                vr = alpha.x * re;
                vi = alpha.y * re;
              }
              if (beta) { const cplx o = Crow[gj]; vr += o.x; vi += o.y; }
              Crow[gj] = make_double2(vr, vi);
            }
          }
        }
        continue;
      }
      if (P.ksplit > 1) {  // the exact integer partial; the reduction adds them exactly
        longlong2* Wp = reinterpret_cast<longlong2*>(ws + W.inst * ws_is + P.ws) + int64_t(W.ks) * P.M * P.N +
                        int64_t(gi) * P.N;
#pragma unroll
        for (int jj = 0; jj < HW / 2; ++jj) {
          const int gj = j0 + jj;
          if (gj < P.N) Wp[gj] = make_longlong2(R[2 * jj], R[2 * jj + 1]);
        }
      } else {
        cplx* Crow = C + W.inst * c_is + P.c_off + int64_t(gi) * P.N;
#pragma unroll
        for (int jj = 0; jj < HW / 2; ++jj) {
          const int gj = j0 + jj;
          if (gj < P.N) {
            const int e = ei + fj[jj] - BETA * (S + 1);
            double vr, vi;
            if (alpha_e != ALPHA_GENERAL) {  // alpha = +-2^k: folded into the exponent and sign
              const long long rr = alpha_e < 0 ? -R[2 * jj] : R[2 * jj], ri = alpha_e < 0 ? -R[2 * jj + 1] : R[2 * jj + 1];
              const int k = alpha_e < 0 ? -alpha_e - ALPHA_NEG_BIAS : alpha_e - ALPHA_POS_BIAS;
              vr = scaled_i64(rr, e + k);
              vi = scaled_i64(ri, e + k);
            } else {
              const double re = scaled_i64(R[2 * jj], e), im = scaled_i64(R[2 * jj + 1], e);
              vr = alpha.x * re - alpha.y * im;
              vi = alpha.x * im + alpha.y * re;
            }
            if (beta) { const cplx o = Crow[gj]; vr += o.x; vi += o.y; }
            Crow[gj] = make_double2(vr, vi);
          }
        }
      }
    }
  }
  __syncthreads();
  if (*abort && threadIdx.x == 32) {
    // wait (bounded) for MMAs still in flight before TMEM is released
    mma_commit(drain);
    volatile int dummy = 0;
    mbar_wait(drain, 0, &dummy, gerr, wns);
  }
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// The problem of every work item of a single-split launch: t2p[tile0 + x] = problem.
__global__ void __launch_bounds__(256) k_tile_probs(const EmuProb* __restrict__ probs, int* __restrict__ t2p) {
  const EmuProb& P = probs[blockIdx.x];
  const int n = P.tiles_m * P.tiles_n;
  for (int x = threadIdx.x; x < n; x += blockDim.x) t2p[P.tile0 + x] = blockIdx.x;
}

// ---------------------------------------------------------------------------
// Split kernels.  Exponent E of a row (column) = smallest integer with
// max |Re|, |Im| < 2^E (0 for an all-zero row).
__device__ __forceinline__ int exp_of(double m) { return m > 0.0 ? ilogb(m) + 1 : EXP_ZERO; }

// |x| as an order-preserving unsigned integer (IEEE bits without the sign); the
// exponent E with |x| < 2^E follows from the biased exponent field of the max.
__device__ __forceinline__ unsigned long long abits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ int exp_of_bits(unsigned long long m) {
  const int e = int(m >> 52);
  if (m == 0) return EXP_ZERO;
  if (e == 0) return exp_of(__longlong_as_double((long long)m));  // subnormal
  return e - 1022;  // |x| in [2^(e-1023), 2^(e-1022))
}

// Row exponents: one warp per (row, K range of ROW_KR), grid-stride over all
// of them; warp max -> atomicMax (max is order-independent, so the result is
// deterministic).  Exponent arrays start at EXP_ZERO (all-zero row or column).
#define ROW_KR 1024
__global__ void __launch_bounds__(256) k_row_exp(const EmuProb* __restrict__ probs, int nprobs,
                                                 const cplx* __restrict__ A, int64_t a_is, int* __restrict__ ex,
                                                 int64_t ex_is, int64_t n_items) {
  const int inst = blockIdx.y, lane = threadIdx.x & 31;
  const int64_t stride = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t it = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); it < n_items; it += stride) {
    // work items: per problem M * ceil(K / ROW_KR), the problem's first at rx0
    const EmuProb& P = probs[prob_of_unit<UNIT_RX>(probs, nprobs, it)];
    const int64_t t = it - P.rx0;
    const int nk = max((P.K + ROW_KR - 1) / ROW_KR, 1);
    const int r = int(t / nk), kc = int(t % nk);
    if (r >= P.M) continue;
    const cplx* a = A + inst * a_is + P.a_src + int64_t(r) * P.K;
    unsigned long long m = 0;
    for (int k = kc * ROW_KR + lane; k < min(P.K, (kc + 1) * ROW_KR); k += 32) {
      const cplx v = a[k];
      m = max(m, max(abits(v.x), abits(v.y)));
    }
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) atomicMax(&ex[inst * ex_is + P.a_ex + r], exp_of_bits(m));
  }
}

// Column exponents: CTA = (32 columns, 256 rows of K); 8 row lanes per column.
__global__ void __launch_bounds__(256) k_col_exp(const EmuProb* __restrict__ probs, int nprobs,
                                                 const cplx* __restrict__ B, int64_t b_is, int* __restrict__ ex,
                                                 int64_t ex_is) {
  __shared__ unsigned long long sh[8][33];
  const int inst = blockIdx.y;
  // work items: per problem ceil(N / 32) * ceil(K / 256), the problem's first at cx0
  const EmuProb P = probs[prob_of_unit<UNIT_CX>(probs, nprobs, int64_t(blockIdx.x))];
  const int t = int(int64_t(blockIdx.x) - P.cx0);
  const int nk = max((P.K + 255) / 256, 1);
  const int ct = t / nk, kc = t % nk;
  const int cl = threadIdx.x & 31, rl = threadIdx.x >> 5;
  const int j = ct * 32 + cl;
  unsigned long long m = 0;
  if (j < P.N) {
    const cplx* b = B + inst * b_is + P.b_src + j;
    for (int k = kc * 256 + rl; k < min(P.K, (kc + 1) * 256); k += 8) {
      const cplx v = b[int64_t(k) * P.N];
      m = max(m, max(abits(v.x), abits(v.y)));
    }
  }
  sh[rl][cl] = m;
  __syncthreads();
  if (rl == 0 && j < P.N) {
    for (int w = 1; w < 8; ++w) m = max(m, sh[w][cl]);
    atomicMax(&ex[inst * ex_is + P.b_ex + j], exp_of_bits(m));
  }
}

__global__ void k_fill_int(int* __restrict__ p, int64_t n, int v) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) p[i] = v;
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return uint32_t(__bfloat16_as_ushort(a)) | (uint32_t(__bfloat16_as_ushort(b)) << 16);
}

// x 2^sh rounded to the nearest integer (|x 2^sh| < 2^62), from the IEEE bits with
// integer operations only (GB300's FP64 pipe is the slowest unit on the chip).
__device__ __forceinline__ long long fixed_of(double x, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = int((b >> 52) & 0x7FF);
  if (e == 0) return 0;  // zero or subnormal: below every slice
  const long long mant = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int k = e - 1075 + sh;  // x 2^sh = mant 2^k
  long long X;
  if (k >= 0) X = mant << k;
  else if (k > -64) X = (mant + (1ll << (-k - 1))) >> (-k);
  else X = 0;
  return (b >> 63) ? -X : X;
}

// Balanced base-2^BETA digits of X = rint(x 2^(BETA S)), |x| < 1: the lower S-1
// digits in [-2^(BETA-1), 2^(BETA-1)), the leading one in [-2^BETA, 2^BETA];
// x = sum_s a_s 2^(-BETA s) + r with |r| <= 2^(-BETA S - 1).  Each digit is exact
// in BF16 (built from the exact float of a small integer).
__device__ __forceinline__ uint16_t bf16_of_int(int v) {
  // float(v) without the int-to-float conversion unit: for |v| < 2^22 the float with
  // bits 0x4B400000 + v is 1.5 * 2^23 + v exactly (unit spacing in [2^23, 2^24)), and
  // subtracting 1.5 * 2^23 leaves v exactly; |v| <= 256 then needs 9 bits of BF16
  const float f = __int_as_float(0x4B400000 + v) - 12582912.0f;
  return uint16_t(__float_as_uint(f) >> 16);
}
template <int S>
__device__ __forceinline__ void digits(long long X, uint16_t (&h)[S]) {
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const int d = int(((X + (1 << (BETA - 1))) & ((1 << BETA) - 1))) - (1 << (BETA - 1));
    h[s] = bf16_of_int(d);
    X = (X - d) >> BETA;
  }
  h[0] = bf16_of_int(int(X));
}

template <int S>
__device__ __forceinline__ void slice8(const double (&x)[8], int sh, uint4 (&out)[S], bool neg_copy,
                                       uint4 (&outn)[S]) {
  uint16_t h[8][S];
#pragma unroll
  for (int u = 0; u < 8; ++u) digits<S>(fixed_of(x[u], sh + BETA * S), h[u]);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    out[s] = make_uint4(uint32_t(h[0][s]) | (uint32_t(h[1][s]) << 16), uint32_t(h[2][s]) | (uint32_t(h[3][s]) << 16),
                        uint32_t(h[4][s]) | (uint32_t(h[5][s]) << 16), uint32_t(h[6][s]) | (uint32_t(h[7][s]) << 16));
    if (neg_copy) outn[s] = make_uint4(out[s].x ^ 0x80008000u, out[s].y ^ 0x80008000u, out[s].z ^ 0x80008000u,
                                       out[s].w ^ 0x80008000u);  // -a: flip the BF16 sign bits
  }
}

// A' = [Re A | Im A], each half Kh = K rounded up to 16 (Kp = 2 Kh, a multiple
// of KB).  Work item = (row tile mt, 32-wide range kbh of the half); unit = (row,
// 8-group), 4 units per row in adjacent lanes; grid-stride over all units.  One
// read of A per element, written at positions k (Re) and Kh + k (Im) of the tiled
// K' axis.  FUSE_EXP (every K <= 32: a row lies inside one item): the row
// exponent is formed here from the 4 lanes of the row, not by k_row_exp.
__device__ __forceinline__ int64_t kpos_off(int r, int p, int tile_elems, int S) {
  return int64_t(p / KB) * S * tile_elems + core_off(r, p % KB);
}
template <int S, bool FUSE_EXP>
__global__ void __launch_bounds__(256) k_split_a(const EmuProb* __restrict__ probs, int nprobs, int64_t total,
                                                 const cplx* __restrict__ A, int64_t a_is, int* __restrict__ ex,
                                                 int64_t ex_is, __nv_bfloat16* __restrict__ out, int64_t out_is) {
  const int inst = blockIdx.y;
  // units per item = stored rows x groups per row; the loop runs to a multiple of 32
  // so that whole warps take part in the exponent shuffles (lanes past the end idle)
  const int64_t total32 = (total + 31) & ~int64_t(31);
  for (int64_t U0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; U0 < total32; U0 += int64_t(gridDim.x) * blockDim.x) {
    const bool live = U0 < total;
    const int64_t U = live ? U0 : total - 1;
    const int pi = prob_of_unit<UNIT_A>(probs, nprobs, U);
    const EmuProb& P = probs[pi];
    const int gpr = gpr_of(P);
    const int UA = P.arows * gpr;
    const int64_t lu = U - P.au0;
    const int lt = int(lu / UA), u = int(lu - int64_t(lt) * UA);
    const int nkb = P.Kp / KB, nkh = nkh_of(P), Kh = kh_of(P);
    const int mt = lt / nkh, kbh = lt % nkh;
    const int r = gpr == 4 ? (u >> 2) : (u >> 1), g = gpr == 4 ? (u & 3) : (u & 1);
    const int gi = mt * BM + r;
    const int k0 = kbh * KB + g * 8;
    const cplx* a = A + inst * a_is + P.a_src;
    double xr[8], xi[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      xr[q] = 0.0;
      xi[q] = 0.0;
      if (gi < P.M && k0 + q < P.K) {
        const cplx v = a[int64_t(gi) * P.K + k0 + q];
        xr[q] = v.x;
        xi[q] = v.y;
      }
    }
    int sh;
    if (FUSE_EXP) {
      unsigned long long m = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) m = max(m, max(abits(xr[q]), abits(xi[q])));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 1));
      const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, m, 2);
      if (gpr == 4) m = max(m, m2);
      const int e = exp_of_bits(m);
      if (live && g == 0 && gi < P.M) ex[inst * ex_is + P.a_ex + gi] = e;
      sh = gi < P.M ? -e : 0;
    } else {
      sh = gi < P.M ? -ex[inst * ex_is + P.a_ex + gi] : 0;
    }
    if (!live || k0 >= Kh || r >= P.arows) continue;
    uint4 sr[S], si[S], dummy[S];
    slice8<S>(xr, sh, sr, false, dummy);
    const int at = P.arows * KB;
    __nv_bfloat16* o = out + inst * out_is + P.a_sl + int64_t(mt) * nkb * (S * at);
    __nv_bfloat16* o_re = o + kpos_off(r, k0, at, S);
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) *reinterpret_cast<uint4*>(o_re + s2 * at) = sr[s2];
    if (P.nh == 2) {  // complex operands: the Im half of the K' axis
      slice8<S>(xi, sh, si, false, dummy);
      __nv_bfloat16* o_im = o + kpos_off(r, Kh + k0, at, S);
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) *reinterpret_cast<uint4*>(o_im + s2 * at) = si[s2];
    }
  }
}

// B'' rows n' = 2j + c: c = 0 -> [Re B_j ; -Im B_j], c = 1 -> [Im B_j ; Re B_j] over the
// two K halves (positions k and Kh + k); real operands (nh = 1): row j = Re B_j over the
// one K range.  Work item = (column tile nt, 32-wide range kbh of the half); unit =
// (column j, 8-group), lanes along j so the strided column reads coalesce; grid-stride
// over all units.
template <int S>
__global__ void __launch_bounds__(256) k_split_b(const EmuProb* __restrict__ probs, int nprobs, int64_t total,
                                                 const cplx* __restrict__ B, int64_t b_is, const int* __restrict__ ex,
                                                 int64_t ex_is, __nv_bfloat16* __restrict__ out, int64_t out_is) {
  using SH = Shape<S>;
  const int inst = blockIdx.y;
  for (int64_t U = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; U < total; U += int64_t(gridDim.x) * blockDim.x) {
    const int pi = prob_of_unit<UNIT_B>(probs, nprobs, U);
    const EmuProb& P = probs[pi];
    const int NJ = ocols_of(P, SH::BN);   // output columns per tile
    const int nj = P.brows / P.nh;  // stored columns per tile (NJ unless compact); nh B rows a column
    const int UB = nj * (KB / 8);
    const int64_t lu = U - P.bu0;
    const int lt = int(lu / UB), u = int(lu - int64_t(lt) * UB);
    const int nkb = P.Kp / KB, nkh = nkh_of(P), Kh = kh_of(P);
    const int nt = lt / nkh, kbh = lt % nkh;
    const int jl = u % nj, g = u / nj;
    const int gj = nt * NJ + jl;
    const int k0 = kbh * KB + g * 8;
    if (k0 >= Kh) continue;
    const cplx* b = B + inst * b_is + P.b_src;
    double xr[8], xi[8];
    const int sh = gj < P.N ? -ex[inst * ex_is + P.b_ex + gj] : 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      xr[q] = 0.0;
      xi[q] = 0.0;
      if (gj < P.N && k0 + q < P.K) {
        const cplx v = b[int64_t(k0 + q) * P.N + gj];
        xr[q] = v.x;
        xi[q] = v.y;
      }
    }
    uint4 sr[S], si[S], sin_[S], dummy[S];
    slice8<S>(xr, sh, sr, false, dummy);
    const int bt = P.brows * KB;
    __nv_bfloat16* o = out + inst * out_is + P.b_sl + int64_t(nt) * nkb * (S * bt);
    if (P.nh == 1) {  // real operands: row j = Re B_j
      __nv_bfloat16* r0 = o + kpos_off(jl, k0, bt, S);
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) *reinterpret_cast<uint4*>(r0 + s2 * bt) = sr[s2];
      continue;
    }
    slice8<S>(xi, sh, si, true, sin_);
    __nv_bfloat16* re0 = o + kpos_off(2 * jl, k0, bt, S);
    __nv_bfloat16* im0 = o + kpos_off(2 * jl, Kh + k0, bt, S);
    __nv_bfloat16* re1 = o + kpos_off(2 * jl + 1, k0, bt, S);
    __nv_bfloat16* im1 = o + kpos_off(2 * jl + 1, Kh + k0, bt, S);
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
      *reinterpret_cast<uint4*>(re0 + s2 * bt) = sr[s2];    // row 2j, Re half:  Re B
      *reinterpret_cast<uint4*>(im0 + s2 * bt) = sin_[s2];  // row 2j, Im half: -Im B
      *reinterpret_cast<uint4*>(re1 + s2 * bt) = si[s2];    // row 2j+1, Re half: Im B
      *reinterpret_cast<uint4*>(im1 + s2 * bt) = sr[s2];    // row 2j+1, Im half: Re B
    }
  }
}

// C = alpha * 2^(E_i + F_j - BETA (S + 1)) sum_s R_s (+ C): the split partials are
// the exact int64 accumulators of their K ranges, so their sum is exact and the
// result does not depend on how K was split (nor on the order).  WARP: one warp
// per output element, lane l adding the splits l, l + 32, ... (long split lists);
// otherwise one thread per element.
template <bool WARP>
__global__ void __launch_bounds__(256) k_emu_reduce(const EmuProb* __restrict__ probs, int nprobs,
                                                    const cplx* __restrict__ ws, int64_t ws_is, cplx* __restrict__ C,
                                                    int64_t c_is, const int* __restrict__ Aex, int64_t aex_is,
                                                    const int* __restrict__ Bex, int64_t bex_is, int eshift,
                                                    cplx alpha, int beta, int64_t n_red) {
  const int inst = blockIdx.y, lane = WARP ? (threadIdx.x & 31) : 0;
  const int per = WARP ? 32 : 1;
  const int64_t stride = int64_t(gridDim.x) * (blockDim.x / per);
  for (int64_t it = int64_t(blockIdx.x) * (blockDim.x / per) + threadIdx.x / per; it < n_red; it += stride) {
    int pi = 0;
    while (pi + 1 < nprobs && (probs[pi].ksplit <= 1 || it >= probs[pi].red0 + int64_t(probs[pi].M) * probs[pi].N)) ++pi;
    const EmuProb& P = probs[pi];
    const int64_t n = int64_t(P.M) * P.N, e = it - P.red0;
    const longlong2* W = reinterpret_cast<const longlong2*>(ws + inst * ws_is + P.ws);
    __int128 sr = 0, si = 0;  // the sum of the partials may exceed 63 bits
    for (int s = lane; s < P.ksplit; s += per) {
      const longlong2 w = W[int64_t(s) * n + e];
      sr += w.x;
      si += w.y;
    }
    if (WARP)
      for (int o = 16; o; o >>= 1) {
        const long long rh = __shfl_xor_sync(0xffffffffu, (long long)(sr >> 64), o);
        const unsigned long long rl = __shfl_xor_sync(0xffffffffu, (unsigned long long)sr, o);
        const long long ih = __shfl_xor_sync(0xffffffffu, (long long)(si >> 64), o);
        const unsigned long long il = __shfl_xor_sync(0xffffffffu, (unsigned long long)si, o);
        sr += ((__int128)rh << 64) | (__int128)rl;
        si += ((__int128)ih << 64) | (__int128)il;
      }
    if (lane == 0) {
      const int gi = int(e / P.N), gj = int(e - int64_t(gi) * P.N);
      const int ex = Aex[inst * aex_is + P.a_ex + gi] + Bex[inst * bex_is + P.b_ex + gj] - eshift;
      const double re = scaled_i128(sr, ex), im = scaled_i128(si, ex);
      cplx* Cp = C + inst * c_is + P.c_off;
      double vr = alpha.x * re - alpha.y * im, vi = alpha.x * im + alpha.y * re;
      if (beta) { const cplx o = Cp[e]; vr += o.x; vi += o.y; }
      Cp[e] = make_double2(vr, vi);
    }
  }
}

static void launch_emu_reduce(const EmuProb* d, int np, int max_ksplit, const cplx* ws, int64_t ws_is, cplx* C,
                              int64_t c_is, const int* aex, int64_t aex_is, const int* bex, int64_t bex_is, int S,
                              cplx alpha, int beta, int64_t n_red, int ninst, int sms, cudaStream_t st) {
  const int64_t cap = int64_t(std::max(sms, 1)) * 16;
  const int eshift = BETA * (S + 1);
  if (max_ksplit >= 64) {
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n_red + 7) / 8, cap)));
    k_emu_reduce<true><<<dim3(blocks, ninst), 256, 0, st>>>(d, np, ws, ws_is, C, c_is, aex, aex_is, bex, bex_is, eshift,
                                                            alpha, beta, n_red);
  } else {
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n_red + 255) / 256, cap)));
    k_emu_reduce<false><<<dim3(blocks, ninst), 256, 0, st>>>(d, np, ws, ws_is, C, c_is, aex, aex_is, bex, bex_is,
                                                             eshift, alpha, beta, n_red);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// K' = 2K with each half padded to 16; callers keep K <= EMU_MAX_K, so this stays far
// inside int (the slice and split-K offsets derived from it are int64)
static int kp_of(int K, int nh = 2) {
  return nh == 2 ? 2 * ((std::max(K, 1) + 15) / 16) * 16 : ((std::max(K, 1) + 31) / 32) * 32;
}

// grid of a warp-per-item kernel (8 warps per CTA) and of a thread-per-unit kernel
static int row_exp_blocks(int64_t items, int sms) {
  return int(std::max<int64_t>(1, std::min<int64_t>((items + 7) / 8, int64_t(std::max(sms, 1)) * 16)));
}
static int split_blocks(int64_t units, int sms) {
  return int(std::max<int64_t>(1, std::min<int64_t>((units + 255) / 256, int64_t(std::max(sms, 1)) * 8)));
}

// epilogue encoding of alpha (see ALPHA_GENERAL)
static int alpha_code(cplx a) {
  if (a.y != 0.0 || a.x == 0.0) return ALPHA_GENERAL;
  int ex = 0;
  const double m = std::frexp(std::fabs(a.x), &ex);  // |a| = m 2^ex, m in [0.5, 1)
  if (m != 0.5 || ex - 1 < -60 || ex - 1 > 60) return ALPHA_GENERAL;
  return a.x > 0 ? (ex - 1) + ALPHA_POS_BIAS : -((ex - 1) + ALPHA_NEG_BIAS);
}

struct EmuPlan {
  int S = 5;
  std::vector<EmuProb> h;
  EmuProb* d = nullptr;
  int n_tiles = 0;                    // GEMM work items
  int64_t n_aunits = 0, n_bunits = 0;  // split-A / split-B thread units
  int total_rows = 0, total_cols = 0;
  bool fuse_a = false;  // every K <= 32: split-A forms the row exponents itself
  int n_rowexp = 0, n_colexp = 0;  // work items of the exponent scans
  __nv_bfloat16* asl = nullptr;
  __nv_bfloat16* bsl = nullptr;
  int* aex = nullptr;
  int* bex = nullptr;
  int64_t asl_is = 0, bsl_is = 0, aex_is = 0, bex_is = 0;
  bool a_const = false, b_const = false, a_ready = false, b_ready = false;
  int* d_err = nullptr;
  cplx* d_ws = nullptr;
  int64_t ws_is = 0, red_elems = 0;
  const EmuPlan* b_owner = nullptr;  // another plan that slices the same B (same tensor, layout, S) first
  // work decomposition (autotuned on the first eager run; neither choice changes the result bits)
  int gm = EMU_GM;        // row tiles per group of the work order
  double ks_mult = 1.0;   // multiplier of the default K-split count (0 = no split)
  int64_t tiles_mn = 0;   // output tiles of all problems and instances
  int64_t ws_cap = 0;     // split-K workspace allocated (elements per instance)
  bool tuned = false;
  std::vector<int> chunks;  // exact K chunks per problem
  bool asl_arena = false, bsl_arena = false;  // slices placed in the slice arena at each run
  int64_t bsl_off = 0;                        // element offset of the B slices there
};

// Largest number of exact chunks one work item may accumulate in int64: the sum over
// a K range of Kp real terms is bounded by Kp 2^(14 + 7 (S - 1) + 1) (leading digits
// up to 2^7 each, the lower diagonals adding less than the leading one), which must
// stay below 2^63.  Longer contractions are split and the partials added in 128 bits.
static int64_t max_chunks_per_split(int S) {
  const int bits = 48 - 7 * (S - 1);  // log2 of the largest Kp
  return std::max<int64_t>(1, (int64_t(1) << std::min(bits, 40)) / (KC_BLOCKS * KB));
}

// K splits, work-item numbering and split-K workspace for a split multiplier: the
// default splits long-K problems whose output tiles cannot fill the GPU into about
// 4 x SM-count / tiles pieces of whole exact chunks
static void layout_work(EmuPlan* p, int64_t sms, double mult) {
  int tile0 = 0;
  int64_t ws = 0;
  p->red_elems = 0;
  const int64_t cmax = max_chunks_per_split(p->S);
  for (size_t k = 0; k < p->h.size(); ++k) {
    EmuProb& e = p->h[k];
    const int nkb = e.Kp / KB;
    const int64_t chunks = p->chunks[k];
    int64_t ks = 1;
    if (mult > 0.0 && p->tiles_mn < 2 * sms && nkb >= 2 * KC_BLOCKS) {
      ks = std::min<int64_t>(chunks, (4 * sms + p->tiles_mn - 1) / std::max<int64_t>(p->tiles_mn, 1));
      ks = std::max<int64_t>(1, std::min<int64_t>(int64_t(double(ks) * mult + 0.5), std::min<int64_t>(chunks, 1024)));
    }
    ks = std::max<int64_t>(ks, (chunks + cmax - 1) / cmax);  // every split's int64 accumulator fits
    e.kcb = int32_t(((chunks + ks - 1) / ks) * KC_BLOCKS);
    e.ksplit = (nkb + e.kcb - 1) / e.kcb;
    e.ws = 0;
    e.red0 = 0;
    if (e.ksplit > 1) {
      e.ws = ws;
      ws += int64_t(e.ksplit) * e.M * e.N;
      e.red0 = p->red_elems;
      p->red_elems += int64_t(e.M) * e.N;
    }
    e.tile0 = tile0;
    tile0 += e.tiles_m * e.tiles_n * e.ksplit;
  }
  p->n_tiles = tile0;
  p->ws_is = ws;
}

struct BKey {
  const void* ptr;
  int64_t is;
  int S;
  std::vector<int64_t> probs;  // (b_src, K, N) per problem
  bool operator==(const BKey& o) const { return ptr == o.ptr && is == o.is && S == o.S && probs == o.probs; }
};

struct EmuState {
  std::vector<EmuPlan*> plans;
  std::vector<std::pair<BKey, EmuPlan*>> bowners;
  int* d_err = nullptr;
  cplx* tune_buf = nullptr;  // scratch output for the autotuner's trial launches
  int64_t tune_cap = 0;
  std::vector<EmuProb> set_recs;  // product records of operand-set launches (emu_set_multiply)
  EmuProb* set_d = nullptr;
  int64_t set_cap = 0;
  int* set_t2p = nullptr;  // work item -> product of such a launch
  int64_t set_t2p_cap = 0;
};

bool emu_wanted(Ctx& c, const GemmPlan& g, const std::string&) {
  if (c.cfg.precision != EXP_EMU_BF16) return false;
  if (c.cfg.emu_min_macs > 0) return double(g.flops_mac) >= c.cfg.emu_min_macs;
  // below ~4e6 complex MACs per launch (all instances) the slicing passes cost more
  // than the FP64 kernels; above, GB300's FP64 rate loses to the tensor cores (or, for
  // K <= 16, to the double-single FP32 product) at every K
  return g.flops_mac * c.ninst >= int64_t(1) << 22;
}

template <int S>
static void set_smem_attr() {
  static bool done = false;
  if (!done) {
    CK(cudaFuncSetAttribute(k_emu_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, Shape<S>::SMEM));
    done = true;
  }
}

static int bn_of(int S) { return S <= 5 ? 48 : 32; }

bool emu_major_site(const std::string& site) {
  // the particle-particle ladder, X_amij (its t1 companion over <am||ef>), the two ring products
  static const char* const kMajor[] = {"R2pp", "Xamij", "Qring", "Wmbej3"};
  for (const char* m : kMajor)
    if (site == m) return true;
  return false;
}

EmuPlan* emu_plan(Ctx& c, const GemmPlan& g, const Tensor* A, const Tensor* B, bool a_const, bool b_const,
                  bool b_shareable, const std::string& site) {
  EmuState* st = (EmuState*)c.emu_state;
  if (!st) {
    st = new EmuState();
    c.emu_state = st;
    st->d_err = (int*)c.dalloc(sizeof(int));
    CK(cudaMemsetAsync(st->d_err, 0, sizeof(int), c.stream));
    c.d_emu_err = st->d_err;
  }
  EmuPlan* p = new EmuPlan();
  st->plans.push_back(p);
  p->S = (c.cfg.n_slices_major > 0 && emu_major_site(site)) ? c.cfg.n_slices_major : c.cfg.n_slices;
  p->a_const = a_const;
  p->b_const = b_const;
  p->d_err = st->d_err;
  const int BN = bn_of(p->S);
  int64_t asl = 0, bsl = 0, aex = 0, bex = 0;
  int64_t au0 = 0, bu0 = 0;
  int64_t tiles_mn = 0;
  const int nh = c.cfg.real_arith ? 1 : 2;  // real operands: no Im half, one B row per column
  const int ocols = nh == 2 ? BN / 2 : BN;
  for (auto& q : g.h_probs)
    tiles_mn += int64_t((q.M + BM - 1) / BM) * ((q.N + ocols - 1) / ocols);
  tiles_mn *= c.ninst;
  const int64_t sms = std::max(c.sm_count, 1);
  p->fuse_a = true;
  for (auto& q : g.h_probs) {
    EmuProb e{};
    e.a_src = q.a;
    e.b_src = q.b;
    e.c_off = q.c;
    e.M = q.M;
    e.N = q.N;
    e.K = q.K;
    if (q.K > EMU_MAX_K) throw ExpError{EXP_EINVAL, "emulated GEMM: K above 2^26"};
    e.nh = nh;
    e.Kp = kp_of(q.K, nh);  // [Re | Im], each half padded to 16 (real: Re padded to 32)
    e.tiles_m = (q.M + BM - 1) / BM;
    e.tiles_n = (q.N + ocols - 1) / ocols;
    e.arows = e.tiles_m == 1 ? (q.M + 7) / 8 * 8 : BM;
    e.brows = e.tiles_n == 1 ? (nh * q.N + 7) / 8 * 8 : BN;  // nh B rows per output column
    if (q.K > 32) p->fuse_a = false;
    const int nkb = e.Kp / KB;
    p->chunks.push_back((nkb + KC_BLOCKS - 1) / KC_BLOCKS);
    e.a_sl = asl;
    e.b_sl = bsl;
    asl += int64_t(e.tiles_m) * nkb * p->S * e.arows * KB;
    bsl += int64_t(e.tiles_n) * nkb * p->S * e.brows * KB;
    e.a_ex = aex;
    e.b_ex = bex;
    aex += q.M;
    bex += q.N;
    p->total_rows += q.M;
    p->total_cols += q.N;
    e.rx0 = p->n_rowexp;
    e.cx0 = p->n_colexp;
    p->n_rowexp += q.M * std::max((q.K + ROW_KR - 1) / ROW_KR, 1);
    p->n_colexp += ((q.N + 31) / 32) * std::max((q.K + 255) / 256, 1);
    e.au0 = au0;
    e.bu0 = bu0;
    au0 += int64_t(e.tiles_m) * nkh_of(e) * e.arows * gpr_of(e);
    bu0 += int64_t(e.tiles_n) * nkh_of(e) * (e.brows / nh) * (KB / 8);
    p->h.push_back(e);
  }
  p->tiles_mn = tiles_mn;
  if (c.force_ksplit_mult >= 0.0) p->ks_mult = std::min(c.force_ksplit_mult, 4.0);
  if (c.force_group_rows > 0) p->gm = c.force_group_rows;
  layout_work(p, sms, p->ks_mult);
  p->n_aunits = au0;
  p->n_bunits = bu0;
  p->asl_is = std::max<int64_t>(asl, 1);
  p->bsl_is = std::max<int64_t>(bsl, 1);
  p->aex_is = std::max<int64_t>(aex, 1);
  p->bex_is = std::max<int64_t>(bex, 1);
  // slices of an integral (made once) or of a lasting tensor other products may share
  // get their own buffers; the per-iteration slices of this product alone live in the
  // slice arena (A first, then B) and are placed at every run
  int64_t arena_elems = 0;
  if (a_const) {
    p->asl = (__nv_bfloat16*)c.dalloc(sizeof(__nv_bfloat16) * p->asl_is * c.ninst);
  } else {
    p->asl_arena = true;
    arena_elems = p->asl_is * c.ninst;
  }
  p->aex = (int*)c.dalloc(sizeof(int) * p->aex_is * c.ninst);
  // B slices: reuse those of an earlier plan that reads the same tensor the same way
  // (plans run in creation order every iteration, so the owner has sliced it already)
  BKey key{B ? (const void*)B->d : nullptr, B ? B->is : 0, p->S, {}};
  for (auto& e : p->h) { key.probs.push_back(e.b_src); key.probs.push_back(e.K); key.probs.push_back(e.N); }
  if (B && b_shareable)
    for (auto& kv : st->bowners)
      if (kv.first == key) { p->b_owner = kv.second; break; }
  if (p->b_owner) {
    p->bsl = p->b_owner->bsl;
    p->bex = p->b_owner->bex;
  } else {
    if (b_const || b_shareable) {
      p->bsl = (__nv_bfloat16*)c.dalloc(sizeof(__nv_bfloat16) * p->bsl_is * c.ninst);
    } else {
      p->bsl_arena = true;
      p->bsl_off = (arena_elems + 127) / 128 * 128;
      arena_elems = p->bsl_off + p->bsl_is * c.ninst;
    }
    p->bex = (int*)c.dalloc(sizeof(int) * p->bex_is * c.ninst);
    if (B && b_shareable) st->bowners.push_back({key, p});
  }
  if (arena_elems) arena_reserve(c, c.slice_arena, sizeof(__nv_bfloat16) * size_t(arena_elems));
  // workspace for the largest split the tuner may try (multiplier 4)
  {
    const double m0 = p->ks_mult;
    layout_work(p, sms, 4.0);
    p->ws_cap = p->ws_is;
    layout_work(p, sms, m0);
    p->ws_cap = std::max(p->ws_cap, p->ws_is);
    if (p->ws_cap) p->d_ws = (cplx*)c.dalloc(sizeof(cplx) * p->ws_cap * c.ninst);
  }
  p->d = (EmuProb*)c.dalloc(sizeof(EmuProb) * p->h.size());
  upload(c, p->d, p->h.data(), sizeof(EmuProb) * p->h.size());
  (void)A;
  return p;
}

// profiling mode: stage boundaries of one emulated product (A scan + split, B scan
// + split, GEMM, split-K reduction), reported after the stream drains
struct EmuStageTimer {
  bool on;
  cudaStream_t st;
  cudaEvent_t ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  EmuStageTimer(bool on_, cudaStream_t s) : on(on_), st(s) {
    if (on)
      for (auto& e : ev) { CK(cudaEventCreate(&e)); }
    mark(0);
  }
  int last = -1;
  void mark(int k) {  // a skipped stage gets a zero-length interval
    if (on)
      for (; last < k; ++last) CK(cudaEventRecord(ev[last + 1], st));
  }
  void report(int64_t tiles) {
    if (!on) return;
    CK(cudaEventSynchronize(ev[6]));
    float t[6];
    for (int k = 0; k < 6; ++k) CK(cudaEventElapsedTime(&t[k], ev[k], ev[k + 1]));
    fprintf(stderr,
            "[exp_emu] exp_a %6.3f split_a %6.3f exp_b %6.3f split_b %6.3f gemm %6.3f reduce %6.3f ms  work items %lld\n",
            t[0], t[1], t[2], t[3], t[4], t[5], (long long)tiles);
    for (auto& e : ev) cudaEventDestroy(e);
  }
};

// Timeout test hook (exp_test_emu_wait): the wait limit and the k-block that CTA 0
// skips, for the launches that follow on any thread until it is reset.
static std::atomic<unsigned long long> g_wait_ns{2000000000ull};
static std::atomic<int> g_skip_kblock{-1};
static EmuWaitTest emu_wait_test() { return EmuWaitTest{g_wait_ns.load(), g_skip_kblock.load(), 0}; }

extern "C" exp_status exp_test_emu_wait(int skip_kblock, double wait_ms) {
  if (skip_kblock < -1 || !(wait_ms > 0.0) || wait_ms > 2000.0) return EXP_EINVAL;
  g_wait_ns.store((unsigned long long)(wait_ms * 1e6));
  g_skip_kblock.store(skip_kblock);
  return EXP_OK;
}

// The GEMM launch of a plan (plus its split-K reduction) into C.
template <int S>
static void launch_product(Ctx& c, EmuPlan* p, cplx* C, int64_t cis, cplx alpha, bool beta, bool reduce) {
  const int np = int(p->h.size());
  set_smem_attr<S>();
  const int n_work = p->n_tiles * c.ninst;
  k_emu_gemm<S><<<dim3(std::min(n_work, std::max(c.sm_count, 1))), Shape<S>::THREADS, Shape<S>::SMEM,
                  c.stream>>>(
      p->d, np, p->n_tiles, n_work, p->gm, p->asl, p->bsl, p->aex, p->bex, C, p->asl_is, p->bsl_is, p->aex_is,
      p->bex_is, cis, alpha, p->red_elems ? ALPHA_GENERAL : alpha_code(alpha), beta ? 1 : 0, p->d_err, p->d_ws, p->ws_is,
      emu_wait_test(), nullptr);
  KCHECK(c);
  if (reduce && p->red_elems) {
    int mks = 1;
    for (auto& e : p->h) mks = std::max(mks, int(e.ksplit));
    launch_emu_reduce(p->d, np, mks, p->d_ws, p->ws_is, C, cis, p->aex, p->aex_is, p->bex, p->bex_is, S, alpha,
                      beta ? 1 : 0, p->red_elems, c.ninst, c.sm_count, c.stream);
    KCHECK(c);
  }
}

// Autotuner: on a plan's first eager run (slices in place), time the product for
// each candidate work decomposition -- K-split multipliers {0, 1/2, 1, 2, 4} when the
// default splits K, group sizes {4, 8, 16} when there are row and column tiles to
// group -- and keep the fastest.  Trial launches write a scratch output; split-K
// partials are exact, so no candidate changes the result.  Skipped while the
// stream is being captured and for one-off products.
template <int S>
static void autotune(Ctx& c, EmuPlan* p, int64_t cis, cplx alpha) {
  p->tuned = true;
  if (!c.autotune) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(c.stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return;
  const int64_t sms = std::max(c.sm_count, 1);
  std::vector<double> mults{p->ks_mult};
  if (p->red_elems) mults = {0.0, 0.5, 1.0, 2.0, 4.0};
  std::vector<int> gms{p->gm};
  for (auto& e : p->h)
    if (e.tiles_m > 4 && e.tiles_n > 1) { gms = {4, 8, 16}; break; }
  if (mults.size() * gms.size() <= 1) return;
  EmuState* st = (EmuState*)c.emu_state;
  const int64_t need = std::max<int64_t>(cis, 1) * c.ninst;
  if (need > st->tune_cap) {
    st->tune_cap = std::max(need, 2 * st->tune_cap);
    st->tune_buf = (cplx*)c.dalloc(sizeof(cplx) * st->tune_cap);
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best_ms = 1e30, best_m = p->ks_mult;
  int best_gm = p->gm;
  bool warm = false;
  for (double m : mults) {
    layout_work(p, sms, m);
    upload(c, p->d, p->h.data(), sizeof(EmuProb) * p->h.size());
    for (int g : gms) {
      p->gm = g;
      if (!warm) launch_product<S>(c, p, st->tune_buf, cis, alpha, false, true);  // one warm-up
      warm = true;
      CK(cudaEventRecord(e0, c.stream));
      launch_product<S>(c, p, st->tune_buf, cis, alpha, false, true);
      CK(cudaEventRecord(e1, c.stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) { best_ms = ms; best_m = m; best_gm = g; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->ks_mult = best_m;
  p->gm = best_gm;
  layout_work(p, sms, best_m);
  upload(c, p->d, p->h.data(), sizeof(EmuProb) * p->h.size());
  if (c.profile)
    fprintf(stderr, "[exp_tune] %d candidates: K-split x%.1f, group %d rows, %.3f ms\n", int(mults.size() * gms.size()),
            best_m, best_gm, best_ms);
}

template <int S>
static void run_s(Ctx& c, EmuPlan* p, const cplx* A, const cplx* B, cplx* C, int64_t ais, int64_t bis, int64_t cis,
                  cplx alpha, bool beta, bool gemm_only) {
  const int np = int(p->h.size());
  if (p->asl_arena) p->asl = (__nv_bfloat16*)c.slice_arena.base;
  if (p->bsl_arena) p->bsl = (__nv_bfloat16*)c.slice_arena.base + p->bsl_off;
  if (gemm_only) {  // the tensor-core product alone, on the slices already in place
    launch_product<S>(c, p, C, cis, alpha, beta, false);
    return;
  }
  EmuStageTimer tm(c.profile, c.stream);
  if (!p->a_ready) {
    const int blocks = split_blocks(p->n_aunits, c.sm_count);
    if (p->fuse_a) {
      tm.mark(1);
      k_split_a<S, true><<<dim3(blocks, c.ninst), 256, 0, c.stream>>>(p->d, np, p->n_aunits, A, ais, p->aex, p->aex_is,
                                                                      p->asl, p->asl_is);
    } else {
      k_fill_int<<<dim3(std::max<int64_t>(1, std::min<int64_t>((p->aex_is * c.ninst + 255) / 256, 1024))), 256, 0,
                   c.stream>>>(p->aex, p->aex_is * c.ninst, EXP_ZERO);
      KCHECK(c);
      k_row_exp<<<dim3(row_exp_blocks(p->n_rowexp, c.sm_count), c.ninst), 256, 0, c.stream>>>(p->d, np, A, ais, p->aex,
                                                                                                p->aex_is, p->n_rowexp);
      KCHECK(c);
      tm.mark(1);
      k_split_a<S, false><<<dim3(blocks, c.ninst), 256, 0, c.stream>>>(p->d, np, p->n_aunits, A, ais, p->aex, p->aex_is,
                                                                       p->asl, p->asl_is);
    }
    KCHECK(c);
    if (p->a_const) p->a_ready = true;
  }
  tm.mark(2);
  if (!p->b_ready && !p->b_owner) {
    k_fill_int<<<dim3(std::max<int64_t>(1, std::min<int64_t>((p->bex_is * c.ninst + 255) / 256, 1024))), 256, 0, c.stream>>>(
        p->bex, p->bex_is * c.ninst, EXP_ZERO);
    KCHECK(c);
    k_col_exp<<<dim3(p->n_colexp, c.ninst), 256, 0, c.stream>>>(p->d, np, B, bis, p->bex, p->bex_is);
    KCHECK(c);
    tm.mark(3);
    k_split_b<S><<<dim3(split_blocks(p->n_bunits, c.sm_count), c.ninst), 256, 0, c.stream>>>(
        p->d, np, p->n_bunits, B, bis, p->bex, p->bex_is, p->bsl, p->bsl_is);
    KCHECK(c);
    if (p->b_const) p->b_ready = true;
  }
  tm.mark(4);
  if (!p->tuned) autotune<S>(c, p, cis, alpha);
  launch_product<S>(c, p, C, cis, alpha, beta, false);
  tm.mark(5);
  if (p->red_elems) {
    int mks = 1;
    for (auto& e : p->h) mks = std::max(mks, int(e.ksplit));
    launch_emu_reduce(p->d, np, mks, p->d_ws, p->ws_is, C, cis, p->aex, p->aex_is, p->bex, p->bex_is, S, alpha,
                      beta ? 1 : 0, p->red_elems, c.ninst, c.sm_count, c.stream);
    KCHECK(c);
  }
  tm.mark(6);
  tm.report(int64_t(p->n_tiles) * c.ninst);
}

void emu_run(Ctx& c, EmuPlan* p, const GemmPlan&, const cplx* A, const cplx* B, cplx* C, int64_t ais, int64_t bis,
             int64_t cis, cplx alpha, bool beta, bool gemm_only) {
  if (p->n_tiles == 0) return;
  switch (p->S) {
    case 3: run_s<3>(c, p, A, B, C, ais, bis, cis, alpha, beta, gemm_only); break;
    case 4: run_s<4>(c, p, A, B, C, ais, bis, cis, alpha, beta, gemm_only); break;
    case 5: run_s<5>(c, p, A, B, C, ais, bis, cis, alpha, beta, gemm_only); break;
    default: run_s<6>(c, p, A, B, C, ais, bis, cis, alpha, beta, gemm_only); break;
  }
}

void emu_release(Ctx& c) {
  EmuState* st = (EmuState*)c.emu_state;
  if (!st) return;
  for (auto* p : st->plans) delete p;
  delete st;
  c.emu_state = nullptr;
}

// ---------------------------------------------------------------------------
// Operand sets: matrices sliced once and multiplied in grouped products chosen at
// run time (the products of the (T) correction, whose pairing of operands
// changes from launch to launch).  A set holds the members' slice tiles and
// exponents in the layout of one side of k_emu_gemm; a product record takes the
// A-side fields of one member and the B-side fields of another.
struct EmuSet {
  int S = 5;
  bool b_side = false;
  int nh = 2;
  std::vector<EmuProb> h;  // one record per member, the fields of its side filled
  EmuProb* d = nullptr;
  int64_t d_cap = 0;  // records
  __nv_bfloat16* sl = nullptr;
  int64_t sl_cap = 0;  // bf16 elements
  int* ex = nullptr;
  int64_t ex_cap = 0;  // exponents
  int64_t units = 0;   // split-kernel units
  int64_t n_scan = 0;  // exponent-scan work items
  int64_t n_ex = 0;
};

static EmuState* emu_state_of(Ctx& c) {
  EmuState* st = (EmuState*)c.emu_state;
  if (!st) {
    st = new EmuState();
    c.emu_state = st;
    st->d_err = (int*)c.dalloc(sizeof(int));
    CK(cudaMemsetAsync(st->d_err, 0, sizeof(int), c.stream));
    c.d_emu_err = st->d_err;
  }
  return st;
}

EmuSet* emu_set_new(Ctx& c, int S, bool b_side) {
  if (S < 3 || S > 6) throw ExpError{EXP_EINVAL, "emulated product: slice count outside 3..6"};
  emu_state_of(c);
  EmuSet* s = new EmuSet();
  s->S = S;
  s->b_side = b_side;
  s->nh = c.cfg.real_arith ? 1 : 2;
  return s;
}

void emu_set_free(Ctx& c, EmuSet* s) {
  if (!s) return;
  if (s->d) c.dfree(s->d);
  if (s->sl) c.dfree(s->sl);
  if (s->ex) c.dfree(s->ex);
  delete s;
}

template <typename T>
static void grow(Ctx& c, T*& p, int64_t& cap, int64_t need) {
  if (need <= cap) return;
  if (p) {
    CK(cudaStreamSynchronize(c.stream));  // earlier launches may still read the old buffer
    c.dfree(p);
  }
  cap = std::max<int64_t>(need, cap + cap / 2);
  p = (T*)c.dalloc(sizeof(T) * size_t(cap));
}

template <int S>
static void set_slice_s(Ctx& c, EmuSet* s, const cplx* src) {
  const int np = int(s->h.size());
  k_fill_int<<<dim3(int(std::max<int64_t>(1, std::min<int64_t>((s->n_ex + 255) / 256, 1024)))), 256, 0, c.stream>>>(
      s->ex, s->n_ex, EXP_ZERO);
  KCHECK(c);
  if (s->n_scan) {
    if (!s->b_side)
      k_row_exp<<<dim3(row_exp_blocks(s->n_scan, c.sm_count), 1), 256, 0, c.stream>>>(s->d, np, src, 0, s->ex, 0,
                                                                                   s->n_scan);
    else
      k_col_exp<<<dim3(unsigned(s->n_scan), 1), 256, 0, c.stream>>>(s->d, np, src, 0, s->ex, 0);
    KCHECK(c);
  }
  if (!s->units) return;
  if (!s->b_side)
    k_split_a<S, false><<<dim3(split_blocks(s->units, c.sm_count), 1), 256, 0, c.stream>>>(s->d, np, s->units, src, 0,
                                                                                          s->ex, 0, s->sl, 0);
  else
    k_split_b<S><<<dim3(split_blocks(s->units, c.sm_count), 1), 256, 0, c.stream>>>(s->d, np, s->units, src, 0, s->ex,
                                                                                   0, s->sl, 0);
  KCHECK(c);
}

void emu_set_slice(Ctx& c, EmuSet* s, const std::vector<EmuSetMat>& mats, const cplx* src) {
  const int S = s->S, nh = s->nh;
  const int BN = bn_of(S);
  const int ocols = nh == 2 ? BN / 2 : BN;
  s->h.clear();
  int64_t sl = 0, ex = 0, u0 = 0, scan = 0;
  std::vector<std::pair<int64_t, int>> grp;  // exponent group -> (offset, rows)
  for (const EmuSetMat& m : mats) {
    if (m.rows < 0 || m.K < 0 || m.K > EMU_MAX_K) throw ExpError{EXP_EINVAL, "emulated product: member shape"};
    // the member's exponent vector: its own, or its group's (made by the first member)
    int64_t ex_at = ex;
    bool own = true;
    if (m.ex_group >= 0) {
      if (size_t(m.ex_group) >= grp.size()) grp.resize(size_t(m.ex_group) + 1, {-1, 0});
      auto& gr = grp[size_t(m.ex_group)];
      if (gr.first >= 0) {
        if (gr.second != m.rows) throw ExpError{EXP_EINVAL, "emulated product: exponent group of unequal members"};
        ex_at = gr.first;
        own = false;
      } else {
        gr = {ex, m.rows};
      }
    }
    EmuProb e{};
    e.nh = nh;
    e.K = m.K;
    e.Kp = kp_of(m.K, nh);
    const int nkb = e.Kp / KB;
    if (!s->b_side) {
      e.a_src = m.src;
      e.M = m.rows;
      e.tiles_m = (m.rows + BM - 1) / BM;
      e.arows = e.tiles_m == 1 ? (m.rows + 7) / 8 * 8 : BM;
      e.a_sl = sl;
      e.a_ex = ex_at;
      e.au0 = u0;
      sl += int64_t(e.tiles_m) * nkb * S * e.arows * KB;
      u0 += int64_t(e.tiles_m) * nkh_of(e) * e.arows * gpr_of(e);
      e.rx0 = scan;
      scan += int64_t(m.rows) * std::max((m.K + ROW_KR - 1) / ROW_KR, 1);
    } else {
      e.b_src = m.src;
      e.N = m.rows;
      e.tiles_n = (m.rows + ocols - 1) / ocols;
      e.brows = e.tiles_n == 1 ? (nh * m.rows + 7) / 8 * 8 : BN;
      e.b_sl = sl;
      e.b_ex = ex_at;
      e.bu0 = u0;
      sl += int64_t(e.tiles_n) * nkb * S * e.brows * KB;
      u0 += int64_t(e.tiles_n) * nkh_of(e) * (e.brows / nh) * (KB / 8);
      e.cx0 = scan;
      scan += int64_t((m.rows + 31) / 32) * std::max((m.K + 255) / 256, 1);
    }
    if (own) ex += m.rows;
    s->h.push_back(e);
  }
  if (s->b_side && scan > INT32_MAX) throw ExpError{EXP_EINVAL, "emulated product: operand set too large"};
  s->units = u0;
  s->n_scan = scan;
  s->n_ex = std::max<int64_t>(ex, 1);
  if (s->h.empty()) return;
  grow(c, s->sl, s->sl_cap, std::max<int64_t>(sl, 1));
  grow(c, s->ex, s->ex_cap, s->n_ex);
  grow(c, s->d, s->d_cap, int64_t(s->h.size()));
  upload_async(c, s->d, s->h.data(), sizeof(EmuProb) * s->h.size());
  switch (S) {
    case 3: set_slice_s<3>(c, s, src); break;
    case 4: set_slice_s<4>(c, s, src); break;
    case 5: set_slice_s<5>(c, s, src); break;
    default: set_slice_s<6>(c, s, src); break;
  }
}

template <int S>
static void set_multiply_s(Ctx& c, const EmuProb* d, int np, int n_tiles, const EmuSet* A, const EmuSet* B, cplx* C,
                           cplx alpha, int* gerr, const int* t2p) {
  set_smem_attr<S>();
  k_emu_gemm<S><<<dim3(std::min(n_tiles, std::max(c.sm_count, 1))), Shape<S>::THREADS, Shape<S>::SMEM,
                  c.stream>>>(
      d, np, n_tiles, n_tiles, EMU_GM, A->sl, B->sl, A->ex, B->ex, C, 0, 0, 0, 0, 0, alpha, alpha_code(alpha), 0, gerr,
      nullptr, 0, emu_wait_test(), t2p);
  KCHECK(c);
}

void emu_set_multiply(Ctx& c, const EmuSet* A, const EmuSet* B, const std::vector<EmuSetProd>& prods, cplx* C,
                      cplx alpha) {
  if (A->b_side || !B->b_side || A->S != B->S || A->nh != B->nh)
    throw ExpError{EXP_EINVAL, "emulated product: operand sets do not match"};
  const int S = A->S;
  const int64_t cmax = max_chunks_per_split(S);
  EmuState* st = emu_state_of(c);
  std::vector<EmuProb>& h = st->set_recs;
  h.clear();
  int64_t tile0 = 0;
  for (const EmuSetProd& t : prods) {
    const int sa[3] = {t.a, t.a1, t.a2}, sb[3] = {t.b, t.b1, t.b2};
    int nseg = 0;
    for (int w = 0; w < 3; ++w) {
      if (sa[w] < 0 && sb[w] < 0 && w > 0) continue;
      if (sa[w] < 0 || sa[w] >= int(A->h.size()) || sb[w] < 0 || sb[w] >= int(B->h.size()))
        throw ExpError{EXP_EINVAL, "emulated product: member index"};
      if (w != nseg) throw ExpError{EXP_EINVAL, "emulated product: segments out of order"};
      ++nseg;
    }
    const EmuProb& a = A->h[t.a];
    const EmuProb& b = B->h[t.b];
    if (a.M == 0 || b.N == 0) continue;
    EmuProb e{};
    e.a_sl = a.a_sl;
    e.a_ex = a.a_ex;
    e.b_sl = b.b_sl;
    e.b_ex = b.b_ex;
    e.c_off = t.c_off;
    e.M = a.M;
    e.N = b.N;
    e.nh = a.nh;
    e.tiles_m = a.tiles_m;
    e.tiles_n = b.tiles_n;
    e.arows = a.arows;
    e.brows = b.brows;
    // the segments that hold K, in order
    struct Seg {
      int64_t asl, bsl;
      int nkb;
    } sg[3];
    int ns = 0;
    for (int w = 0; w < nseg; ++w) {
      const EmuProb& aw = A->h[sa[w]];
      const EmuProb& bw = B->h[sb[w]];
      if (aw.K != bw.K) throw ExpError{EXP_EINVAL, "emulated product: members of different K"};
      // one exponent per output row and column across the segments, one tiling
      if (aw.M != a.M || aw.a_ex != a.a_ex || bw.N != b.N || bw.b_ex != b.b_ex)
        throw ExpError{EXP_EINVAL, "emulated product: segments outside one exponent group"};
      if (aw.K == 0) continue;
      e.K += aw.K;
      e.Kp += aw.Kp;
      sg[ns++] = Seg{aw.a_sl, bw.b_sl, aw.Kp / KB};
    }
    if (ns > 0) {
      e.a_sl = sg[0].asl;
      e.b_sl = sg[0].bsl;
    }
    if (ns > 1) {
      e.nkb0 = sg[0].nkb;
      e.nkb1 = sg[1].nkb;
      e.a_sl1 = sg[1].asl;
      e.b_sl1 = sg[1].bsl;
    }
    if (ns > 2) {
      e.a_sl2 = sg[2].asl;
      e.b_sl2 = sg[2].bsl;
    }
    if (e.K == 0) continue;  // no K at all: C is left as it is (the caller clears it)
    const int64_t chunks = (e.Kp / KB + KC_BLOCKS - 1) / KC_BLOCKS;
    // one exact int64 accumulation per output: no split-K partials for these products
    if (chunks > cmax) throw ExpError{EXP_EINVAL, "emulated product: K too long for one exact accumulation"};
    e.ksplit = 1;
    e.kcb = int32_t(chunks * KC_BLOCKS);
    e.tile0 = int32_t(tile0);
    tile0 += int64_t(e.tiles_m) * e.tiles_n;
    if (tile0 > INT32_MAX) throw ExpError{EXP_EINVAL, "emulated product: too many output tiles in one launch"};
    h.push_back(e);
  }
  if (h.empty()) return;
  grow(c, st->set_d, st->set_cap, int64_t(h.size()));
  upload_async(c, st->set_d, h.data(), sizeof(EmuProb) * h.size());
  const int np = int(h.size()), nt = int(tile0);
  // a list longer than the kernel's shared-memory copy: the work items' problems as a table
  const int* t2p = nullptr;
  if (np * int64_t(sizeof(EmuProb)) > 4096) {
    grow(c, st->set_t2p, st->set_t2p_cap, int64_t(nt));
    k_tile_probs<<<np, 256, 0, c.stream>>>(st->set_d, st->set_t2p);
    KCHECK(c);
    t2p = st->set_t2p;
  }
  switch (S) {
    case 3: set_multiply_s<3>(c, st->set_d, np, nt, A, B, C, alpha, st->d_err, t2p); break;
    case 4: set_multiply_s<4>(c, st->set_d, np, nt, A, B, C, alpha, st->d_err, t2p); break;
    case 5: set_multiply_s<5>(c, st->set_d, np, nt, A, B, C, alpha, st->d_err, t2p); break;
    default: set_multiply_s<6>(c, st->set_d, np, nt, A, B, C, alpha, st->d_err, t2p); break;
  }
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the emulated GEMM (exp_zgemm_emu_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// product: code running inside a memory-pool budget that is already spent,
// plugins that are handed a stream and buffers by a host application that
// owns every allocation, or code paths where a cudaMalloc would synchronise
// the device.  For them this entry point takes its scratch (slice tiles,
// exponents, split-K partials, the problem record and the error flag) from a
// fixed array in the module's device memory instead of an allocator.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds EXP_NOALLOC_SCRATCH_BYTES of it until the process exits.  Its
// device address is looked up on the first call on a device (cudaGetSymbolAddress,
// with that device current) and kept for that device's current context; a new
// context on the device (after cudaDeviceReset) gets a fresh lookup.  Make that
// first call before any stream capture.  All calls share the one array: the parts
// that must start at a known value (exponents, the error flag) are re-initialised
// on the stream by every call, and two calls whose work overlaps on the GPU
// (different streams, no ordering between them) race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[EXP_NOALLOC_SCRATCH_BYTES];

namespace {
struct NoallocDev {
  unsigned char* base = nullptr;
  unsigned long long ctx_id = 0;  // unique id of the context the address belongs to
  bool ready = false;
};
NoallocDev g_noalloc_dev[64];
std::mutex g_noalloc_mu;  // guards g_noalloc_dev (first calls from several host threads)

// cuCtxGetId through the runtime's driver entry-point query (no link against the
// driver library): the id of the current context, unique for the process's life
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetIdFn ctx_get_id() {
  static CtxGetIdFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return (CtxGetIdFn)f;
  }();
  return fn;
}
bool current_ctx_id(unsigned long long& id) {
  const CtxGetIdFn f = ctx_get_id();
  return f && f(nullptr, &id) == CUDA_SUCCESS;
}

int64_t carve(int64_t& off, int64_t bytes) {
  const int64_t at = (off + 255) & ~int64_t(255);
  off = at + bytes;
  return at;
}

template <int S>
exp_status noalloc_launch(cudaStream_t st, unsigned char* base, int M, int N, int K, const cplx* A, const cplx* B,
                          cplx* Cout, cplx alpha, int beta, int sms, std::string& err) {
  using SH = Shape<S>;
  const int BN = SH::BN;
  EmuProb e{};
  e.M = M;
  e.N = N;
  e.K = K;
  e.nh = 2;
  e.Kp = kp_of(K);
  e.tiles_m = (M + BM - 1) / BM;
  e.tiles_n = (N + BN / 2 - 1) / (BN / 2);
  const int nkb = e.Kp / KB;
  const int64_t tiles_mn = int64_t(e.tiles_m) * e.tiles_n;
  {
    const int64_t chunks = (nkb + KC_BLOCKS - 1) / KC_BLOCKS;
    int64_t ks = 1;
    if (tiles_mn < 2LL * sms && nkb >= 2 * KC_BLOCKS) {
      ks = std::min<int64_t>(chunks, (4LL * sms + tiles_mn - 1) / std::max<int64_t>(tiles_mn, 1));
      ks = std::max<int64_t>(1, std::min<int64_t>(ks, 512));
    }
    const int64_t cmax = max_chunks_per_split(S);
    ks = std::max<int64_t>(ks, (chunks + cmax - 1) / cmax);
    e.kcb = int32_t(((chunks + ks - 1) / ks) * KC_BLOCKS);
    e.ksplit = (nkb + e.kcb - 1) / e.kcb;
  }
  e.arows = e.tiles_m == 1 ? (M + 7) / 8 * 8 : BM;
  e.brows = e.tiles_n == 1 ? (2 * N + 7) / 8 * 8 : BN;
  e.tile0 = 0;
  e.au0 = e.bu0 = 0;
  e.red0 = 0;
  // scratch layout
  int64_t off = 0;
  const int64_t o_probs = carve(off, sizeof(EmuProb));
  const int64_t o_err = carve(off, sizeof(int));
  const int64_t o_aex = carve(off, sizeof(int) * int64_t(M));
  const int64_t o_bex = carve(off, sizeof(int) * int64_t(N));
  const int64_t o_asl = carve(off, int64_t(2) * e.tiles_m * nkb * S * e.arows * KB);
  const int64_t o_bsl = carve(off, int64_t(2) * e.tiles_n * nkb * S * e.brows * KB);
  const int64_t o_ws = carve(off, e.ksplit > 1 ? int64_t(sizeof(cplx)) * e.ksplit * M * N : 0);
  if (off > int64_t(EXP_NOALLOC_SCRATCH_BYTES)) {
    err = "exp_zgemm_emu_noalloc: problem needs " + std::to_string(off) + " bytes of scratch, more than the " +
          std::to_string(int64_t(EXP_NOALLOC_SCRATCH_BYTES)) + " bytes available";
    return EXP_EINVAL;
  }
  EmuProb recs[1] = {e};
  EmuProb* d_probs = (EmuProb*)(base + o_probs);
  int* d_err = (int*)(base + o_err);
  int* aex = (int*)(base + o_aex);
  int* bex = (int*)(base + o_bex);
  __nv_bfloat16* asl = (__nv_bfloat16*)(base + o_asl);
  __nv_bfloat16* bsl = (__nv_bfloat16*)(base + o_bsl);
  cplx* ws = (cplx*)(base + o_ws);
  if (cudaMemcpyAsync(d_probs, recs, sizeof(recs), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) {
    err = "exp_zgemm_emu_noalloc: copy to scratch failed";
    return EXP_ECUDA;
  }
  // every launch is checked before the next one is issued: on a failed launch
  // nothing after it runs (C is then unspecified, see the header)
  auto launched = [&](const char* what) {
    const cudaError_t le = cudaGetLastError();
    if (le == cudaSuccess) return true;
    err = std::string("exp_zgemm_emu_noalloc: launch of ") + what + " failed: " + cudaGetErrorString(le);
    return false;
  };
  const int64_t n_rowexp = int64_t(M) * std::max((K + ROW_KR - 1) / ROW_KR, 1);
  const int64_t n_colexp = int64_t((N + 31) / 32) * std::max((K + 255) / 256, 1);
  k_fill_int<<<std::max(1, std::min((M + 255) / 256, 1024)), 256, 0, st>>>(aex, M, EXP_ZERO);
  if (!launched("k_fill_int")) return EXP_ECUDA;
  k_fill_int<<<std::max(1, std::min((N + 255) / 256, 1024)), 256, 0, st>>>(bex, N, EXP_ZERO);
  if (!launched("k_fill_int")) return EXP_ECUDA;
  k_row_exp<<<dim3(row_exp_blocks(n_rowexp, sms), 1), 256, 0, st>>>(d_probs, 1, A, 0, aex, 0, n_rowexp);
  if (!launched("k_row_exp")) return EXP_ECUDA;
  k_col_exp<<<dim3(unsigned(n_colexp), 1), 256, 0, st>>>(d_probs, 1, B, 0, bex, 0);
  if (!launched("k_col_exp")) return EXP_ECUDA;
  const int64_t na = int64_t(e.tiles_m) * nkh_of(e) * e.arows * gpr_of(e);
  const int64_t nb = int64_t(e.tiles_n) * nkh_of(e) * (e.brows / 2) * (KB / 8);
  k_split_a<S, false><<<dim3(split_blocks(na, sms), 1), 256, 0, st>>>(d_probs, 1, na, A, 0, aex, 0, asl, 0);
  if (!launched("k_split_a")) return EXP_ECUDA;
  k_split_b<S><<<dim3(split_blocks(nb, sms), 1), 256, 0, st>>>(d_probs, 1, nb, B, 0, bex, 0, bsl, 0);
  if (!launched("k_split_b")) return EXP_ECUDA;
  if (cudaFuncSetAttribute(k_emu_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::SMEM) != cudaSuccess) {
    err = "exp_zgemm_emu_noalloc: shared-memory attribute refused";
    return EXP_ECUDA;
  }
  const int n_work = int(tiles_mn * e.ksplit);
  k_emu_gemm<S><<<dim3(unsigned(std::min(n_work, sms)), 1), SH::THREADS, SH::SMEM, st>>>(
      d_probs, 1, n_work, n_work, EMU_GM, asl, bsl, aex, bex, Cout, 0, 0, 0, 0, 0, alpha,
      e.ksplit > 1 ? ALPHA_GENERAL : alpha_code(alpha), beta, d_err, ws, 0, EmuWaitTest{2000000000ull, -1, 0}, nullptr);
  if (!launched("k_emu_gemm")) return EXP_ECUDA;
  if (e.ksplit > 1) {
    launch_emu_reduce(d_probs, 1, e.ksplit, ws, 0, Cout, 0, aex, 0, bex, 0, S, alpha, beta, int64_t(M) * N, 1, sms, st);
    if (!launched("the split-K reduction")) return EXP_ECUDA;
  }
  const cudaError_t ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    err = std::string("exp_zgemm_emu_noalloc: ") + cudaGetErrorString(ce);
    return EXP_ECUDA;
  }
  int flag = 0;
  if (cudaMemcpy(&flag, d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    err = "exp_zgemm_emu_noalloc: reading the error flag failed";
    return EXP_ECUDA;
  }
  if (flag) {
    err = "exp_zgemm_emu_noalloc: a bounded device wait gave up";
    return EXP_ETIMEOUT;
  }
  return EXP_OK;
}
}  // namespace

static thread_local std::string g_noalloc_err;

extern "C" const char* exp_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

extern "C" exp_status exp_zgemm_emu_noalloc(void* stream, int n_slices, int M, int N, int K, const void* A,
                                            const void* B, void* C, double alpha_re, double alpha_im, int beta) {
  g_noalloc_err.clear();
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || n_slices < 3 || n_slices > 6) {
    g_noalloc_err = "exp_zgemm_emu_noalloc: null pointer, M, N, K < 1 or n_slices outside 3..6";
    return EXP_EINVAL;
  }
  // before any layout arithmetic: K' = 2K padded must stay far inside int (a larger K
  // could not fit the scratch array anyway)
  if (K > EMU_MAX_K) {
    g_noalloc_err = "exp_zgemm_emu_noalloc: K above 2^26 (the scratch array cannot hold its slices)";
    return EXP_EINVAL;
  }
  {
    // an error left pending by earlier work of the caller is reported as such, not
    // as a failure of this call's launches
    const cudaError_t pe = cudaPeekAtLastError();
    if (pe != cudaSuccess) {
      g_noalloc_err = std::string("exp_zgemm_emu_noalloc: a CUDA error was pending before the call: ") +
                      cudaGetErrorString(pe);
      return EXP_ECUDA;
    }
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    g_noalloc_err = "exp_zgemm_emu_noalloc: no current CUDA device";
    return EXP_ECUDA;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDev& nd = g_noalloc_dev[dev];
    unsigned long long id = 0;
    const bool have_id = current_ctx_id(id);
    if (!nd.ready || !have_id || nd.ctx_id != id) {
      // set-up on this device (and context): the host-side name of the array is not
      // a device address; ask the runtime for the real one
      void* p = nullptr;
      const cudaError_t ce = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (ce != cudaSuccess || !p) {
        nd.ready = false;
        g_noalloc_err = std::string("exp_zgemm_emu_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(ce);
        return EXP_ECUDA;
      }
      nd.base = (unsigned char*)p;
      // the lookup made the device's context current if it was not: key the address by it
      nd.ready = current_ctx_id(nd.ctx_id);
    }
    base = nd.base;
  }
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cplx alpha = make_double2(alpha_re, alpha_im);
  cudaStream_t st = (cudaStream_t)stream;
  const cplx* a = (const cplx*)A;
  const cplx* b = (const cplx*)B;
  cplx* c = (cplx*)C;
  switch (n_slices) {
    case 3: return noalloc_launch<3>(st, base, M, N, K, a, b, c, alpha, beta != 0, sms, g_noalloc_err);
    case 4: return noalloc_launch<4>(st, base, M, N, K, a, b, c, alpha, beta != 0, sms, g_noalloc_err);
    case 5: return noalloc_launch<5>(st, base, M, N, K, a, b, c, alpha, beta != 0, sms, g_noalloc_err);
    default: return noalloc_launch<6>(st, base, M, N, K, a, b, c, alpha, beta != 0, sms, g_noalloc_err);
  }
}
