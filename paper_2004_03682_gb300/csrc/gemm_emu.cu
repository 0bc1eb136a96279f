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
// along N), warps 2-5 drain the double-buffered TMEM accumulators.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <string>

#include "emu.h"

namespace {

constexpr int BM = 128;        // rows per tile (tcgen05 M)
constexpr int KB = 32;         // real K per smem k-block (4 core matrices of 8 bf16)
constexpr int BETA = 7;        // bits per slice
constexpr int KC_BLOCKS = 16;  // k-blocks per exact chunk: KC = 512 real terms
constexpr int STAGES = 3;
constexpr int THREADS = 192;   // 6 warps
#define EXP_ZERO (-1100)       // exponent of an all-zero row / column (any x 2^-EXP_ZERO stays 0)

template <int S>
struct Shape {
  static constexpr int BN = S <= 5 ? 48 : 32;  // real output columns per tile
  static constexpr int A_TILE = BM * KB;       // bf16 elements per slice tile
  static constexpr int B_TILE = BN * KB;
  static constexpr int A_STAGE = S * A_TILE * 2;  // bytes
  static constexpr int B_STAGE = S * B_TILE * 2;
  static constexpr int STAGE = A_STAGE + B_STAGE;
  static constexpr int ACC = S * BN;             // TMEM columns per accumulator buffer
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
  static_assert(2 * ACC <= 512, "TMEM");
  static_assert(S * BN <= 256, "MMA N");
  static_assert(BN % 16 == 0, "N multiple of 16");
};

struct EmuProb {
  int64_t a_src, b_src, c_off;  // complex offsets in the per-instance A, B, C tensors
  int64_t a_sl, b_sl;           // bf16 offsets of the slice tiles (per instance)
  int64_t a_ex, b_ex;           // offsets of the exponent arrays (per instance)
  int64_t ws;                   // split-K partials offset (complex, per instance)
  int32_t M, N, K, Kp;          // Kp = 2K padded to KB
  int32_t tiles_m, tiles_n, tile0, pad;
  int32_t ksplit, kcb, pad2, pad3;  // K splits and k-blocks per split (multiple of KC_BLOCKS)
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
// Bounded wait: gives up after ~2 s (or when another role already gave up),
// recording the failure; never spins forever.
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort, int* gerr) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 255) == 0) {
      if (*abort) return false;
      if (gtimer() - t0 > 2000000000ull) {
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
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// offset (in elements) of element (r, k) inside a tile of `rows` x KB, core-matrix order
__device__ __forceinline__ int core_off(int r, int k) { return ((r >> 3) * (KB / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

// ---------------------------------------------------------------------------
// GEMM kernel
template <int S>
__global__ void __launch_bounds__(THREADS, 1)
    k_emu_gemm(const EmuProb* __restrict__ probs, int nprobs, const __nv_bfloat16* __restrict__ Asl,
               const __nv_bfloat16* __restrict__ Bsl, const int* __restrict__ Aex, const int* __restrict__ Bex,
               cplx* __restrict__ C, int64_t asl_is, int64_t bsl_is, int64_t aex_is, int64_t bex_is, int64_t c_is,
               cplx alpha, int beta, int* __restrict__ gerr, cplx* __restrict__ ws, int64_t ws_is) {
  using SH = Shape<S>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)((uintptr_t(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = (uint64_t*)(smem + STAGES * SH::STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;
  uint64_t* acce = accf + 2;
  uint64_t* drain = acce + 2;
  uint32_t* tslot = (uint32_t*)(drain + 1);
  volatile int* abort = (volatile int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x, inst = blockIdx.y;
  int pi = 0;
  while (pi + 1 < nprobs && probs[pi + 1].tile0 <= tile) ++pi;
  const EmuProb P = probs[pi];
  int lt = tile - P.tile0;  // tile -> (K split, row tile, column tile)
  const int tmn = P.tiles_m * P.tiles_n;
  const int ks = lt / tmn;
  lt -= ks * tmn;
  const int mt = lt / P.tiles_n, nt = lt % P.tiles_n;
  const int nkb_all = P.Kp / KB;
  const int kb0 = ks * P.kcb;
  const int nkb = min(nkb_all, kb0 + P.kcb) - kb0;  // k-blocks of this split
  const int nchunks = (nkb + KC_BLOCKS - 1) / KC_BLOCKS;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&accf[b], 1); mbar_init(&acce[b], 4); }
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

  const __nv_bfloat16* Ab = Asl + inst * asl_is + P.a_sl + (int64_t(mt) * nkb_all + kb0) * (S * SH::A_TILE);
  const __nv_bfloat16* Bb = Bsl + inst * bsl_is + P.b_sl + (int64_t(nt) * nkb_all + kb0) * (S * SH::B_TILE);

  if (warp == 0) {
    // ---- producer: 1-D TMA bulk copies of the pre-tiled slice tiles
    if (lane == 0) {
      int kb = 0;
      for (; kb < nkb; ++kb) {
        const int st = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(&empty[st], ((kb / STAGES) & 1) ^ 1, abort, gerr)) break;
        uint8_t* sA = smem + st * SH::STAGE;
        uint8_t* sB = sA + SH::A_STAGE;
        mbar_expect_tx(&full[st], SH::STAGE);
        bulk_g2s(sA, Ab + int64_t(kb) * S * SH::A_TILE, SH::A_STAGE, &full[st]);
        bulk_g2s(sB, Bb + int64_t(kb) * S * SH::B_TILE, SH::B_STAGE, &full[st]);
      }
      if (*abort) {
        // let the copies already issued land before the CTA exits
        for (int k = max(0, kb - STAGES); k < kb; ++k) {
          volatile int dummy = 0;
          mbar_wait(&full[k % STAGES], (k / STAGES) & 1, &dummy, gerr);
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      for (int kb = 0; kb < nkb; ++kb) {
        const int st = kb % STAGES;
        const int ch = kb / KC_BLOCKS, buf = ch & 1;
        const bool first = (kb % KC_BLOCKS) == 0;
        if (first && ch >= 2) {
          if (!mbar_wait(&acce[buf], ((ch >> 1) - 1) & 1, abort, gerr)) break;
          fence_after();
        }
        if (!mbar_wait(&full[st], (kb / STAGES) & 1, abort, gerr)) break;
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
        if ((kb % KC_BLOCKS) == KC_BLOCKS - 1 || kb == nkb - 1) mma_commit(&accf[buf]);
      }
    }
  } else {
    // ---- epilogue: 4 warps, one TMEM lane (= output row) per thread
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;
    long long R[SH::BN];
#pragma unroll
    for (int j = 0; j < SH::BN; ++j) R[j] = 0;
    bool ok = true;
    for (int ch = 0; ch < nchunks && ok; ++ch) {
      const int buf = ch & 1;
      if (!mbar_wait(&accf[buf], (ch >> 1) & 1, abort, gerr)) { ok = false; break; }
      fence_after();
#pragma unroll
      for (int dgi = 0; dgi < S; ++dgi) {
        const int shift = BETA * (S - 1 - dgi);
#pragma unroll
        for (int j16 = 0; j16 < SH::BN / 16; ++j16) {
          uint32_t v[16];
          tmem_ld16(tmem + (uint32_t(q * 32) << 16) + buf * 256 + dgi * SH::BN + j16 * 16, v);
          tmem_wait_ld();
#pragma unroll
          for (int u = 0; u < 16; ++u)
            R[j16 * 16 + u] += (long long)__float2int_rn(__uint_as_float(v[u])) << shift;
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[buf]);
    }
    if (ok) {
      const int gi = mt * BM + row;
      if (gi < P.M && P.ksplit > 1) {  // scaled partial for the fixed-order reduction
        const int ei = Aex[inst * aex_is + P.a_ex + gi];
        cplx* W = ws + inst * ws_is + P.ws + int64_t(ks) * P.M * P.N + int64_t(gi) * P.N;
#pragma unroll
        for (int jj = 0; jj < SH::BN / 2; ++jj) {
          const int gj = nt * (SH::BN / 2) + jj;
          if (gj < P.N) {
            const int e = ei + Bex[inst * bex_is + P.b_ex + gj] - BETA * (S + 1);
            W[gj] = make_double2(ldexp(double(R[2 * jj]), e), ldexp(double(R[2 * jj + 1]), e));
          }
        }
      } else if (gi < P.M) {
        const int ei = Aex[inst * aex_is + P.a_ex + gi];
        cplx* Crow = C + inst * c_is + P.c_off + int64_t(gi) * P.N;
#pragma unroll
        for (int jj = 0; jj < SH::BN / 2; ++jj) {
          const int gj = nt * (SH::BN / 2) + jj;
          if (gj < P.N) {
            const int e = ei + Bex[inst * bex_is + P.b_ex + gj] - BETA * (S + 1);
            const double re = ldexp(double(R[2 * jj]), e), im = ldexp(double(R[2 * jj + 1]), e);
            double vr = alpha.x * re - alpha.y * im, vi = alpha.x * im + alpha.y * re;
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
    mbar_wait(drain, 0, &dummy, gerr);
  }
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
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

// Row exponents: CTA = (one row, a K range of ROW_KR); block max -> atomicMax
// (max is order-independent, so the result is deterministic).  Exponent arrays
// start at EXP_ZERO (all-zero row or column).
#define ROW_KR 8192
__global__ void __launch_bounds__(256) k_row_exp(const EmuProb* __restrict__ probs, int nprobs,
                                                 const cplx* __restrict__ A, int64_t a_is, int* __restrict__ ex,
                                                 int64_t ex_is) {
  __shared__ unsigned long long sh[8];
  const int inst = blockIdx.y;
  int t = blockIdx.x, pi = 0;
  // work items: per problem M * ceil(K / ROW_KR)
  for (;; ++pi) {
    const int nk = (probs[pi].K + ROW_KR - 1) / ROW_KR;
    const int items = probs[pi].M * max(nk, 1);
    if (t < items || pi + 1 >= nprobs) break;
    t -= items;
  }
  const EmuProb P = probs[pi];
  const int nk = max((P.K + ROW_KR - 1) / ROW_KR, 1);
  const int r = t / nk, kc = t % nk;
  if (r >= P.M) return;
  const cplx* a = A + inst * a_is + P.a_src + int64_t(r) * P.K;
  unsigned long long m = 0;
  for (int k = kc * ROW_KR + threadIdx.x; k < min(P.K, (kc + 1) * ROW_KR); k += 256) {
    const cplx v = a[k];
    m = max(m, max(abits(v.x), abits(v.y)));
  }
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = max(m, sh[w]);
    atomicMax(&ex[inst * ex_is + P.a_ex + r], exp_of_bits(m));
  }
}

// Column exponents: CTA = (32 columns, 256 rows of K); 8 row lanes per column.
__global__ void __launch_bounds__(256) k_col_exp(const EmuProb* __restrict__ probs, int nprobs,
                                                 const cplx* __restrict__ B, int64_t b_is, int* __restrict__ ex,
                                                 int64_t ex_is) {
  __shared__ unsigned long long sh[8][33];
  const int inst = blockIdx.y;
  int t = blockIdx.x, pi = 0;
  for (;; ++pi) {
    const int items = ((probs[pi].N + 31) / 32) * max((probs[pi].K + 255) / 256, 1);
    if (t < items || pi + 1 >= nprobs) break;
    t -= items;
  }
  const EmuProb P = probs[pi];
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
  return uint16_t(__float_as_uint(float(v)) >> 16);  // exact: |v| <= 256 needs 9 bits
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

// A' = [Re A | Im A], each half padded to Kh = K rounded up to KB.  CTA = (row
// tile mt, half-k-block kbh): one read of A per element, writes the Re tile
// (k-block kbh) and the Im tile (k-block Kh/KB + kbh).  Thread unit = (row, 8-group).
template <int S>
__global__ void __launch_bounds__(256) k_split_a(const EmuProb* __restrict__ probs, int nprobs, const cplx* __restrict__ A,
                                                 int64_t a_is, const int* __restrict__ ex, int64_t ex_is,
                                                 __nv_bfloat16* __restrict__ out, int64_t out_is) {
  using SH = Shape<S>;
  const int inst = blockIdx.y;
  int t = blockIdx.x, pi = 0;
  while (pi + 1 < nprobs && t >= probs[pi].tile0 + probs[pi].tiles_m * (probs[pi].Kp / (2 * KB))) ++pi;
  const EmuProb P = probs[pi];
  const int nkb = P.Kp / KB, nkh = nkb / 2;
  const int lt = t - P.tile0;
  const int mt = lt / nkh, kbh = lt % nkh;
  __nv_bfloat16* o_re = out + inst * out_is + P.a_sl + (int64_t(mt) * nkb + kbh) * (S * SH::A_TILE);
  __nv_bfloat16* o_im = out + inst * out_is + P.a_sl + (int64_t(mt) * nkb + nkh + kbh) * (S * SH::A_TILE);
  const cplx* a = A + inst * a_is + P.a_src;
  const int* e = ex + inst * ex_is + P.a_ex;
  for (int u = threadIdx.x; u < BM * (KB / 8); u += blockDim.x) {
    const int r = u >> 2, g = u & 3;
    const int gi = mt * BM + r;
    const int k0 = kbh * KB + g * 8;
    double xr[8], xi[8];
    const int sh = gi < P.M ? -e[gi] : 0;
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
    uint4 sr[S], si[S], dummy[S];
    slice8<S>(xr, sh, sr, false, dummy);
    slice8<S>(xi, sh, si, false, dummy);
    const int off = core_off(r, g * 8);
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
      *reinterpret_cast<uint4*>(o_re + s2 * SH::A_TILE + off) = sr[s2];
      *reinterpret_cast<uint4*>(o_im + s2 * SH::A_TILE + off) = si[s2];
    }
  }
}

// B'' rows n' = 2j + c: c = 0 -> [Re B_j ; -Im B_j], c = 1 -> [Im B_j ; Re B_j] over the
// two K halves.  CTA = (column tile nt, half-k-block kbh); thread unit = (column j,
// 8-group); lanes run along j, so the strided column reads coalesce across a warp.
template <int S>
__global__ void __launch_bounds__(128) k_split_b(const EmuProb* __restrict__ probs, int nprobs, const cplx* __restrict__ B,
                                                 int64_t b_is, const int* __restrict__ ex, int64_t ex_is,
                                                 __nv_bfloat16* __restrict__ out, int64_t out_is, int) {
  using SH = Shape<S>;
  constexpr int NJ = SH::BN / 2;
  const int inst = blockIdx.y;
  int t = blockIdx.x, pi = 0;
  while (pi + 1 < nprobs && t >= probs[pi + 1].pad) ++pi;  // pad = first split-B CTA of the problem
  const EmuProb P = probs[pi];
  const int nkb = P.Kp / KB, nkh = nkb / 2;
  const int lt = t - P.pad;
  const int nt = lt / nkh, kbh = lt % nkh;
  __nv_bfloat16* o_re = out + inst * out_is + P.b_sl + (int64_t(nt) * nkb + kbh) * (S * SH::B_TILE);
  __nv_bfloat16* o_im = out + inst * out_is + P.b_sl + (int64_t(nt) * nkb + nkh + kbh) * (S * SH::B_TILE);
  const cplx* b = B + inst * b_is + P.b_src;
  const int* e = ex + inst * ex_is + P.b_ex;
  for (int u = threadIdx.x; u < NJ * (KB / 8); u += blockDim.x) {
    const int jl = u % NJ, g = u / NJ;
    const int gj = nt * NJ + jl;
    const int k0 = kbh * KB + g * 8;
    double xr[8], xi[8];
    const int sh = gj < P.N ? -e[gj] : 0;
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
    slice8<S>(xi, sh, si, true, sin_);
    const int off0 = core_off(2 * jl, g * 8), off1 = core_off(2 * jl + 1, g * 8);
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
      *reinterpret_cast<uint4*>(o_re + s2 * SH::B_TILE + off0) = sr[s2];    // row 2j, Re half:  Re B
      *reinterpret_cast<uint4*>(o_im + s2 * SH::B_TILE + off0) = sin_[s2];  // row 2j, Im half: -Im B
      *reinterpret_cast<uint4*>(o_re + s2 * SH::B_TILE + off1) = si[s2];    // row 2j+1, Re half: Im B
      *reinterpret_cast<uint4*>(o_im + s2 * SH::B_TILE + off1) = sr[s2];    // row 2j+1, Im half: Re B
    }
  }
}

// C = alpha * sum_s partial_s (+ C), splits in index order
__global__ void __launch_bounds__(256) k_emu_reduce(const EmuProb* __restrict__ probs, int nprobs,
                                                    const cplx* __restrict__ ws, int64_t ws_is, cplx* __restrict__ C,
                                                    int64_t c_is, cplx alpha, int beta) {
  const int inst = blockIdx.y;
  for (int p = 0; p < nprobs; ++p) {
    const EmuProb P = probs[p];
    if (P.ksplit <= 1) continue;
    const int64_t n = int64_t(P.M) * P.N;
    const cplx* W = ws + inst * ws_is + P.ws;
    cplx* Cp = C + inst * c_is + P.c_off;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
      double sr = 0.0, si = 0.0;
      for (int s = 0; s < P.ksplit; ++s) {
        const cplx w = W[int64_t(s) * n + e];
        sr += w.x;
        si += w.y;
      }
      double vr = alpha.x * sr - alpha.y * si, vi = alpha.x * si + alpha.y * sr;
      if (beta) { const cplx o = Cp[e]; vr += o.x; vi += o.y; }
      Cp[e] = make_double2(vr, vi);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
struct EmuPlan {
  int S = 5;
  std::vector<EmuProb> h;
  EmuProb* d = nullptr;
  int n_tiles = 0, n_atiles = 0, n_btiles = 0;
  int total_rows = 0, total_cols = 0;
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
};

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
};

bool emu_wanted(Ctx& c, const GemmPlan& g, const std::string&) {
  if (c.cfg.precision != EXP_EMU_BF16) return false;
  if (c.cfg.emu_min_macs > 0) return double(g.flops_mac) >= c.cfg.emu_min_macs;
  // below ~8e6 complex MACs the slicing passes cost more than the FP64 kernel;
  // contraction lengths from 64 up are faster on the tensor cores than at GB300's
  // FP64 rate, shorter ones (K = o/G ~ 14) are not (per-tile overhead dominates)
  int maxK = 0;
  for (auto& p : g.h_probs) maxK = std::max(maxK, p.K);
  return g.flops_mac >= int64_t(1) << 23 && maxK >= 64;
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

EmuPlan* emu_plan(Ctx& c, const GemmPlan& g, const Tensor* A, const Tensor* B, bool a_const, bool b_const) {
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
  p->S = c.cfg.n_slices;
  p->a_const = a_const;
  p->b_const = b_const;
  p->d_err = st->d_err;
  const int BN = bn_of(p->S);
  int64_t asl = 0, bsl = 0, aex = 0, bex = 0;
  int tile0 = 0, at0 = 0, bt0 = 0;
  int64_t tiles_mn = 0;
  for (auto& q : g.h_probs)
    tiles_mn += int64_t((q.M + BM - 1) / BM) * ((q.N + BN / 2 - 1) / (BN / 2));
  tiles_mn *= c.ninst;
  const int64_t sms = std::max(c.sm_count, 1);
  int64_t ws = 0;
  for (auto& q : g.h_probs) {
    EmuProb e{};
    e.a_src = q.a;
    e.b_src = q.b;
    e.c_off = q.c;
    e.M = q.M;
    e.N = q.N;
    e.K = q.K;
    e.Kp = 2 * std::max((q.K + KB - 1) / KB, 1) * KB;  // [Re | Im], each half padded to KB
    e.tiles_m = (q.M + BM - 1) / BM;
    e.tiles_n = (q.N + BN / 2 - 1) / (BN / 2);
    const int nkb = e.Kp / KB;
    e.ksplit = 1;
    e.kcb = ((nkb + KC_BLOCKS - 1) / KC_BLOCKS) * KC_BLOCKS;
    if (tiles_mn < 2 * sms && nkb >= 2 * KC_BLOCKS) {
      const int64_t chunks = (nkb + KC_BLOCKS - 1) / KC_BLOCKS;
      int64_t ks = std::min<int64_t>(chunks, (4 * sms + tiles_mn - 1) / std::max<int64_t>(tiles_mn, 1));
      ks = std::max<int64_t>(1, std::min<int64_t>(ks, 512));
      e.kcb = int32_t(((chunks + ks - 1) / ks) * KC_BLOCKS);
      e.ksplit = (nkb + e.kcb - 1) / e.kcb;
    }
    if (e.ksplit > 1) {
      e.ws = ws;
      ws += int64_t(e.ksplit) * q.M * q.N;
      p->red_elems += int64_t(q.M) * q.N;
    }
    e.tile0 = tile0;
    tile0 += e.tiles_m * e.tiles_n * e.ksplit;
    e.a_sl = asl;
    e.b_sl = bsl;
    asl += int64_t(e.tiles_m) * nkb * p->S * BM * KB;
    bsl += int64_t(e.tiles_n) * nkb * p->S * BN * KB;
    e.a_ex = aex;
    e.b_ex = bex;
    aex += q.M;
    bex += q.N;
    p->total_rows += q.M;
    p->total_cols += q.N;
    p->n_rowexp += q.M * std::max((q.K + ROW_KR - 1) / ROW_KR, 1);
    p->n_colexp += ((q.N + 31) / 32) * std::max((q.K + 255) / 256, 1);
    e.pad = bt0;  // first split-B CTA
    bt0 += e.tiles_n * (nkb / 2);
    at0 += e.tiles_m * (nkb / 2);
    p->h.push_back(e);
  }
  // split-A tile indexing reuses tile0 as the first split-A tile of each problem
  std::vector<EmuProb> ha = p->h;
  {
    int t = 0;
    for (auto& e : ha) { e.tile0 = t; t += e.tiles_m * (e.Kp / (2 * KB)); }
  }
  p->n_tiles = tile0;
  p->n_atiles = at0;
  p->n_btiles = bt0;
  p->asl_is = std::max<int64_t>(asl, 1);
  p->bsl_is = std::max<int64_t>(bsl, 1);
  p->aex_is = std::max<int64_t>(aex, 1);
  p->bex_is = std::max<int64_t>(bex, 1);
  p->asl = (__nv_bfloat16*)c.dalloc(sizeof(__nv_bfloat16) * p->asl_is * c.ninst);
  p->aex = (int*)c.dalloc(sizeof(int) * p->aex_is * c.ninst);
  // B slices: reuse those of an earlier plan that reads the same tensor the same way
  // (plans run in creation order every iteration, so the owner has sliced it already)
  BKey key{B ? (const void*)B->d : nullptr, B ? B->is : 0, p->S, {}};
  for (auto& e : p->h) { key.probs.push_back(e.b_src); key.probs.push_back(e.K); key.probs.push_back(e.N); }
  for (auto& kv : st->bowners)
    if (B && kv.first == key) { p->b_owner = kv.second; break; }
  if (p->b_owner) {
    p->bsl = p->b_owner->bsl;
    p->bex = p->b_owner->bex;
  } else {
    p->bsl = (__nv_bfloat16*)c.dalloc(sizeof(__nv_bfloat16) * p->bsl_is * c.ninst);
    p->bex = (int*)c.dalloc(sizeof(int) * p->bex_is * c.ninst);
    if (B) st->bowners.push_back({key, p});
  }
  if (ws) {
    p->ws_is = ws;
    p->d_ws = (cplx*)c.dalloc(sizeof(cplx) * ws * c.ninst);
  }
  // two device copies of the problem list: [0, n) for the GEMM and split-B, [n, 2n) for split-A
  std::vector<EmuProb> both = p->h;
  both.insert(both.end(), ha.begin(), ha.end());
  p->d = (EmuProb*)c.dalloc(sizeof(EmuProb) * both.size());
  upload(c, p->d, both.data(), sizeof(EmuProb) * both.size());
  (void)A;
  return p;
}

template <int S>
static void run_s(Ctx& c, EmuPlan* p, const cplx* A, const cplx* B, cplx* C, int64_t ais, int64_t bis, int64_t cis,
                  cplx alpha, bool beta) {
  const int np = int(p->h.size());
  if (!p->a_ready) {
    k_fill_int<<<dim3(std::max<int64_t>(1, std::min<int64_t>((p->aex_is * c.ninst + 255) / 256, 1024))), 256, 0, c.stream>>>(
        p->aex, p->aex_is * c.ninst, EXP_ZERO);
    KCHECK(c);
    k_row_exp<<<dim3(p->n_rowexp, c.ninst), 256, 0, c.stream>>>(p->d, np, A, ais, p->aex, p->aex_is);
    KCHECK(c);
    k_split_a<S><<<dim3(p->n_atiles, c.ninst), 256, 0, c.stream>>>(p->d + np, np, A, ais, p->aex, p->aex_is, p->asl,
                                                                   p->asl_is);
    KCHECK(c);
    if (p->a_const) p->a_ready = true;
  }
  if (!p->b_ready && !p->b_owner) {
    k_fill_int<<<dim3(std::max<int64_t>(1, std::min<int64_t>((p->bex_is * c.ninst + 255) / 256, 1024))), 256, 0, c.stream>>>(
        p->bex, p->bex_is * c.ninst, EXP_ZERO);
    KCHECK(c);
    k_col_exp<<<dim3(p->n_colexp, c.ninst), 256, 0, c.stream>>>(p->d, np, B, bis, p->bex, p->bex_is);
    KCHECK(c);
    k_split_b<S><<<dim3(p->n_btiles, c.ninst), 128, 0, c.stream>>>(p->d, np, B, bis, p->bex, p->bex_is, p->bsl,
                                                                   p->bsl_is, 0);
    KCHECK(c);
    if (p->b_const) p->b_ready = true;
  }
  set_smem_attr<S>();
  k_emu_gemm<S><<<dim3(p->n_tiles, c.ninst), THREADS, Shape<S>::SMEM, c.stream>>>(
      p->d, np, p->asl, p->bsl, p->aex, p->bex, C, p->asl_is, p->bsl_is, p->aex_is, p->bex_is, cis, alpha, beta ? 1 : 0,
      p->d_err, p->d_ws, p->ws_is);
  KCHECK(c);
  if (p->red_elems) {
    const int blocks = int(std::min<int64_t>((p->red_elems + 255) / 256, 2LL * std::max(c.sm_count, 1)));
    k_emu_reduce<<<dim3(blocks, c.ninst), 256, 0, c.stream>>>(p->d, np, p->d_ws, p->ws_is, C, cis, alpha, beta ? 1 : 0);
    KCHECK(c);
  }
}

void emu_run(Ctx& c, EmuPlan* p, const GemmPlan&, const cplx* A, const cplx* B, cplx* C, int64_t ais, int64_t bis,
             int64_t cis, cplx alpha, bool beta) {
  if (p->n_tiles == 0) return;
  switch (p->S) {
    case 3: run_s<3>(c, p, A, B, C, ais, bis, cis, alpha, beta); break;
    case 4: run_s<4>(c, p, A, B, C, ais, bis, cis, alpha, beta); break;
    case 5: run_s<5>(c, p, A, B, C, ais, bis, cis, alpha, beta); break;
    default: run_s<6>(c, p, A, B, C, ais, bis, cis, alpha, beta); break;
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
// device address is looked up once per device (cudaGetSymbolAddress, with that
// device current) on the first call on that device; make that first call
// before any stream capture.  All calls share the one array: the parts that
// must start at a known value (exponents, the error flag) are re-initialised
// on the stream by every call, and two calls whose work overlaps on the GPU
// (different streams, no ordering between them) race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[EXP_NOALLOC_SCRATCH_BYTES];

namespace {
struct NoallocDev {
  unsigned char* base = nullptr;
  bool ready = false;
};
NoallocDev g_noalloc_dev[64];

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
  e.Kp = 2 * std::max((K + KB - 1) / KB, 1) * KB;
  e.tiles_m = (M + BM - 1) / BM;
  e.tiles_n = (N + BN / 2 - 1) / (BN / 2);
  const int nkb = e.Kp / KB;
  const int64_t tiles_mn = int64_t(e.tiles_m) * e.tiles_n;
  e.ksplit = 1;
  e.kcb = ((nkb + KC_BLOCKS - 1) / KC_BLOCKS) * KC_BLOCKS;
  if (tiles_mn < 2LL * sms && nkb >= 2 * KC_BLOCKS) {
    const int64_t chunks = (nkb + KC_BLOCKS - 1) / KC_BLOCKS;
    int64_t ks = std::min<int64_t>(chunks, (4LL * sms + tiles_mn - 1) / std::max<int64_t>(tiles_mn, 1));
    ks = std::max<int64_t>(1, std::min<int64_t>(ks, 512));
    e.kcb = int32_t(((chunks + ks - 1) / ks) * KC_BLOCKS);
    e.ksplit = (nkb + e.kcb - 1) / e.kcb;
  }
  e.pad = 0;
  e.tile0 = 0;
  // scratch layout
  int64_t off = 0;
  const int64_t o_probs = carve(off, 2 * sizeof(EmuProb));
  const int64_t o_err = carve(off, sizeof(int));
  const int64_t o_aex = carve(off, sizeof(int) * int64_t(M));
  const int64_t o_bex = carve(off, sizeof(int) * int64_t(N));
  const int64_t o_asl = carve(off, int64_t(2) * e.tiles_m * nkb * S * BM * KB);
  const int64_t o_bsl = carve(off, int64_t(2) * e.tiles_n * nkb * S * BN * KB);
  const int64_t o_ws = carve(off, e.ksplit > 1 ? int64_t(sizeof(cplx)) * e.ksplit * M * N : 0);
  if (off > int64_t(EXP_NOALLOC_SCRATCH_BYTES)) {
    err = "exp_zgemm_emu_noalloc: problem needs " + std::to_string(off) + " bytes of scratch, more than the " +
          std::to_string(int64_t(EXP_NOALLOC_SCRATCH_BYTES)) + " bytes available";
    return EXP_EINVAL;
  }
  EmuProb recs[2] = {e, e};
  recs[1].tile0 = 0;  // split-A tile numbering starts at 0 as well
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
  const int64_t n_rowexp = int64_t(M) * std::max((K + ROW_KR - 1) / ROW_KR, 1);
  const int64_t n_colexp = int64_t((N + 31) / 32) * std::max((K + 255) / 256, 1);
  k_fill_int<<<std::max(1, std::min((M + 255) / 256, 1024)), 256, 0, st>>>(aex, M, EXP_ZERO);
  k_fill_int<<<std::max(1, std::min((N + 255) / 256, 1024)), 256, 0, st>>>(bex, N, EXP_ZERO);
  k_row_exp<<<dim3(unsigned(n_rowexp), 1), 256, 0, st>>>(d_probs, 1, A, 0, aex, 0);
  k_col_exp<<<dim3(unsigned(n_colexp), 1), 256, 0, st>>>(d_probs, 1, B, 0, bex, 0);
  k_split_a<S><<<dim3(e.tiles_m * (nkb / 2), 1), 256, 0, st>>>(d_probs + 1, 1, A, 0, aex, 0, asl, 0);
  k_split_b<S><<<dim3(e.tiles_n * (nkb / 2), 1), 128, 0, st>>>(d_probs, 1, B, 0, bex, 0, bsl, 0, 0);
  if (cudaFuncSetAttribute(k_emu_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::SMEM) != cudaSuccess) {
    err = "exp_zgemm_emu_noalloc: shared-memory attribute refused";
    return EXP_ECUDA;
  }
  k_emu_gemm<S><<<dim3(unsigned(tiles_mn * e.ksplit), 1), THREADS, SH::SMEM, st>>>(
      d_probs, 1, asl, bsl, aex, bex, Cout, 0, 0, 0, 0, 0, alpha, beta, d_err, ws, 0);
  if (e.ksplit > 1) {
    const int blocks = int(std::min<int64_t>((int64_t(M) * N + 255) / 256, 2LL * sms));
    k_emu_reduce<<<dim3(blocks, 1), 256, 0, st>>>(d_probs, 1, ws, 0, Cout, 0, alpha, beta);
  }
  cudaError_t ce = cudaGetLastError();
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
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
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    g_noalloc_err = "exp_zgemm_emu_noalloc: no current CUDA device";
    return EXP_ECUDA;
  }
  NoallocDev& nd = g_noalloc_dev[dev];
  if (!nd.ready) {
    // one-time set-up on this device: the host-side name of the array is not a
    // device address; ask the runtime for the real one
    void* p = nullptr;
    const cudaError_t ce = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (ce != cudaSuccess || !p) {
      g_noalloc_err = std::string("exp_zgemm_emu_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(ce);
      return EXP_ECUDA;
    }
    nd.base = (unsigned char*)p;
    nd.ready = true;
  }
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cplx alpha = make_double2(alpha_re, alpha_im);
  cudaStream_t st = (cudaStream_t)stream;
  const cplx* a = (const cplx*)A;
  const cplx* b = (const cplx*)B;
  cplx* c = (cplx*)C;
  switch (n_slices) {
    case 3: return noalloc_launch<3>(st, nd.base, M, N, K, a, b, c, alpha, beta != 0, sms, g_noalloc_err);
    case 4: return noalloc_launch<4>(st, nd.base, M, N, K, a, b, c, alpha, beta != 0, sms, g_noalloc_err);
    case 5: return noalloc_launch<5>(st, nd.base, M, N, K, a, b, c, alpha, beta != 0, sms, g_noalloc_err);
    default: return noalloc_launch<6>(st, nd.base, M, N, K, a, b, c, alpha, beta != 0, sms, g_noalloc_err);
  }
}
