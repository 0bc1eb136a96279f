// Plain complex-FP64 grouped GEMM: step 3 of the TTGT list (Sec. II.B), all
// symmetry blocks and instances of one contraction in one launch (the block
// loop of Fig. "mult" flattened into a tile list).  Row-major operands,
// C[MxN] = alpha A[MxK] B[KxN] (+ C).  SIMT FP64 FMA: GB300's FP64 rate is the
// roofline for this path.
#include <algorithm>
#include <cmath>

#include "engine.h"
#include "fpbits.h"

#define GT_K 8

// Tile TM x TN (each 16 or 64), 256 threads as 16 x 16, every thread computing
// (TM/16) x (TN/16) outputs; the plan picks 16 along a dimension whose blocks are
// all <= 16 wide, so skinny contractions do not pay for padding.
template <int TM, int TN>
__global__ void __launch_bounds__(256) k_gemm_fp64(const GemmProb* __restrict__ probs, int n_probs,
                                                   const cplx* __restrict__ A,
                                                   const cplx* __restrict__ B, cplx* __restrict__ C,
                                                   int64_t ais, int64_t bis, int64_t cis,
                                                   cplx alpha, int beta, cplx* __restrict__ ws,
                                                   int64_t ws_is) {
  constexpr int RM = TM / 16, RN = TN / 16;
  __shared__ cplx As[GT_K][TM];
  __shared__ cplx Bs[GT_K][TN];
  const int tile = blockIdx.x;
  int pi = 0;
  while (pi + 1 < n_probs && probs[pi + 1].tile0 <= tile) ++pi;
  const GemmProb P = probs[pi];
  int lt = tile - P.tile0;
  const int tmn = P.tiles_m * P.tiles_n;
  const int ks = lt / tmn;  // K split index
  lt -= ks * tmn;
  const int m0 = (lt / P.tiles_n) * TM, n0 = (lt % P.tiles_n) * TN;
  const int kbeg = ks * P.kchunk, kend = min(P.K, kbeg + P.kchunk);
  A += blockIdx.y * ais + P.a;
  B += blockIdx.y * bis + P.b;
  C += blockIdx.y * cis + P.c;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double accr[RM][RN], acci[RM][RN];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < RN; ++j) accr[i][j] = acci[i][j] = 0.0;
  for (int k0 = kbeg; k0 < kend; k0 += GT_K) {
    for (int e = threadIdx.x; e < TM * GT_K; e += 256) {
      const int mm = e >> 3, kk = e & 7;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < P.M && gk < kend) ? A[int64_t(gm) * P.K + gk] : make_double2(0, 0);
    }
    for (int e = threadIdx.x; e < TN * GT_K; e += 256) {
      const int kk = e / TN, nn = e % TN;
      const int gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < kend && gn < P.N) ? B[int64_t(gk) * P.N + gn] : make_double2(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GT_K; ++kk) {
      cplx a[RM], b[RN];
#pragma unroll
      for (int i = 0; i < RM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < RN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) {
          accr[i][j] = fma(a[i].x, b[j].x, accr[i][j]);
          accr[i][j] = fma(-a[i].y, b[j].y, accr[i][j]);
          acci[i][j] = fma(a[i].x, b[j].y, acci[i][j]);
          acci[i][j] = fma(a[i].y, b[j].x, acci[i][j]);
        }
    }
    __syncthreads();
  }
  if (P.ksplit > 1) {  // raw partial for the fixed-order reduction
    cplx* W = ws + blockIdx.y * ws_is + P.ws + int64_t(ks) * P.M * P.N;
#pragma unroll
    for (int i = 0; i < RM; ++i) {
      const int gm = m0 + ty + 16 * i;
      if (gm >= P.M) continue;
#pragma unroll
      for (int j = 0; j < RN; ++j) {
        const int gn = n0 + tx + 16 * j;
        if (gn < P.N) W[int64_t(gm) * P.N + gn] = make_double2(accr[i][j], acci[i][j]);
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= P.M) continue;
#pragma unroll
    for (int j = 0; j < RN; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= P.N) continue;
      double vr = alpha.x * accr[i][j] - alpha.y * acci[i][j];
      double vi = alpha.x * acci[i][j] + alpha.y * accr[i][j];
      cplx* dp = C + int64_t(gm) * P.N + gn;
      if (beta) { const cplx o = *dp; vr += o.x; vi += o.y; }
      *dp = make_double2(vr, vi);
    }
  }
}

// C = alpha * sum_s partial_s (+ C), splits summed in index order (deterministic)
__global__ void __launch_bounds__(256) k_splitk_reduce(const GemmProb* __restrict__ probs, int n_probs,
                                                       const cplx* __restrict__ ws, int64_t ws_is,
                                                       cplx* __restrict__ C, int64_t cis, cplx alpha, int beta) {
  const int inst = blockIdx.y;
  for (int p = 0; p < n_probs; ++p) {
    const GemmProb P = probs[p];
    if (P.ksplit <= 1) continue;
    const int64_t n = int64_t(P.M) * P.N;
    const cplx* W = ws + inst * ws_is + P.ws;
    cplx* Cp = C + inst * cis + P.c;
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

// Small products (and every matrix-vector one): one warp per output element, the
// lanes striding over K, then a fixed butterfly.  At GB300's FP64 rate (about two
// FMAs per clock per SM) a tile kernel leaves most SMs idle on these; here every
// SM takes a share of the outputs and no padded rows or columns are computed.
__global__ void __launch_bounds__(256) k_gemm_dot(const GemmProb* __restrict__ probs, int n_probs,
                                                  const cplx* __restrict__ A, const cplx* __restrict__ B,
                                                  cplx* __restrict__ C, int64_t ais, int64_t bis, int64_t cis,
                                                  cplx alpha, int beta, int64_t n_out) {
  const int lane = threadIdx.x & 31;
  A += blockIdx.y * ais;
  B += blockIdx.y * bis;
  C += blockIdx.y * cis;
  const int64_t stride = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t it = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); it < n_out; it += stride) {
    int pi = 0;
    while (pi + 1 < n_probs && it >= probs[pi + 1].ws) ++pi;  // ws = first output of the problem here
    const GemmProb& P = probs[pi];
    const int64_t e = it - P.ws;
    const int m = int(e / P.N), n = int(e - int64_t(m) * P.N);
    const cplx* a = A + P.a + int64_t(m) * P.K;
    const cplx* b = B + P.b + n;
    double sr = 0.0, si = 0.0;
    for (int k = lane; k < P.K; k += 32) {
      const cplx x = a[k], y = b[int64_t(k) * P.N];
      sr = fma(x.x, y.x, sr);
      sr = fma(-x.y, y.y, sr);
      si = fma(x.x, y.y, si);
      si = fma(x.y, y.x, si);
    }
    for (int o = 16; o; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
      double vr = alpha.x * sr - alpha.y * si, vi = alpha.x * si + alpha.y * sr;
      cplx* dp = C + P.c + e;
      if (beta) { const cplx o = *dp; vr += o.x; vi += o.y; }
      *dp = make_double2(vr, vi);
    }
  }
}

void launch_gemm_fp64(Ctx& c, const GemmPlan& g, const cplx* A, const cplx* B, cplx* C, int64_t ais,
                      int64_t bis, int64_t cis, cplx alpha, bool beta) {
  if (g.dot_outputs) {
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((g.dot_outputs + 7) / 8, 16LL * std::max(c.sm_count, 1))));
    k_gemm_dot<<<dim3(blocks, c.ninst), 256, 0, c.stream>>>(g.d_probs, g.n_probs, A, B, C, ais, bis, cis, alpha,
                                                             beta, g.dot_outputs);
    KCHECK(c);
    return;
  }
  if (g.n_tiles == 0) return;
  const dim3 grid(g.n_tiles, c.ninst);
  if (g.tm == 64 && g.tn == 64)
    k_gemm_fp64<64, 64><<<grid, 256, 0, c.stream>>>(g.d_probs, g.n_probs, A, B, C, ais, bis, cis, alpha, beta, g.d_ws, g.ws_is);
  else if (g.tm == 64)
    k_gemm_fp64<64, 16><<<grid, 256, 0, c.stream>>>(g.d_probs, g.n_probs, A, B, C, ais, bis, cis, alpha, beta, g.d_ws, g.ws_is);
  else if (g.tn == 64)
    k_gemm_fp64<16, 64><<<grid, 256, 0, c.stream>>>(g.d_probs, g.n_probs, A, B, C, ais, bis, cis, alpha, beta, g.d_ws, g.ws_is);
  else
    k_gemm_fp64<16, 16><<<grid, 256, 0, c.stream>>>(g.d_probs, g.n_probs, A, B, C, ais, bis, cis, alpha, beta, g.d_ws, g.ws_is);
  KCHECK(c);
  if (g.red_elems) {
    const int blocks = int(std::min<int64_t>((g.red_elems + 255) / 256, 2LL * std::max(c.sm_count, 1)));
    k_splitk_reduce<<<dim3(blocks, c.ninst), 256, 0, c.stream>>>(g.d_probs, g.n_probs, g.d_ws, g.ws_is, C, cis,
                                                                 alpha, beta);
    KCHECK(c);
  }
}

// ---------------------------------------------------------------------------
// Short contractions (K <= DS_KMAX) under the emulated precision: complex
// products in double-single arithmetic on the FP32 pipe (about 64x GB300's FP64
// rate), every operand split into h + l (48 bits), products and sums carried with
// error-free transformations and the result rounded once to FP64 -- a relative
// error near K 2^-47 of sum |a||b|, below that of the BF16-sliced emulation.  For
// short K that emulation pays for slicing and padding each K half to 16 and for a
// tile pipeline with one k-block per tile; here a product is one pass over A.
// CTA = DS_ROWS rows x DS_NC columns of one problem (the column chunks of a row
// block are adjacent CTAs, so its A block is read from HBM about once): the A
// block (rows contiguous, K each) is read coalesced and split into shared memory,
// the chunk of alpha B staged as double-single pairs; every thread (one row)
// forms its DS_NC outputs.
#define DS_KMAX 16
#define DS_NC 16
#define DS_NG 4  // columns per accumulator group
#define DS_ROWS 128
#define DS_AST (DS_KMAX + 1)  // A row stride in float4: odd, so the row reads of a warp spread over the banks

__global__ void __launch_bounds__(DS_ROWS) k_gemm_ds(const GemmProb* __restrict__ probs, int n_probs,
                                                     const cplx* __restrict__ A, const cplx* __restrict__ B,
                                                     cplx* __restrict__ C, int64_t ais, int64_t bis, int64_t cis,
                                                     cplx alpha, float ascale, int general, int beta) {
  __shared__ float4 As[DS_ROWS * DS_AST];  // (Re h, Re l, Im h, Im l) of A[r0 + r][k]
  __shared__ float4 Bs[DS_KMAX * DS_NC];   // the same for alpha B[k][j0 + jj]
  const int tile = blockIdx.x;
  int pi = 0;
  while (pi + 1 < n_probs && probs[pi + 1].tile0 <= tile) ++pi;
  const GemmProb P = probs[pi];
  const int lt = tile - P.tile0;
  const int rb = lt / P.tiles_n;
  const int r0 = rb * DS_ROWS, j0 = (lt - rb * P.tiles_n) * DS_NC;
  const int nr = min(DS_ROWS, P.M - r0), nc = min(DS_NC, P.N - j0);
  A += blockIdx.y * ais + P.a + int64_t(r0) * P.K;
  B += blockIdx.y * bis + P.b;
  C += blockIdx.y * cis + P.c + int64_t(r0) * P.N;
  for (int e = threadIdx.x; e < nr * P.K; e += blockDim.x) {
    const cplx x = A[e];
    const int r = e / P.K, k = e - r * P.K;
    const float2 xr = ds_split(x.x), xi = ds_split(x.y);
    As[r * DS_AST + k] = make_float4(xr.x, xr.y, xi.x, xi.y);
  }
  const int row = threadIdx.x;
  for (int t = threadIdx.x; t < P.K * DS_NC; t += blockDim.x) {
    const int k = t / DS_NC, jj = t - k * DS_NC;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (jj < nc) {
      cplx b = B[int64_t(k) * P.N + j0 + jj];
      if (general) b = make_double2(alpha.x * b.x - alpha.y * b.y, alpha.x * b.y + alpha.y * b.x);
      const float2 br = ds_split(b.x), bq = ds_split(b.y);
      // ascale = +-2^k (exact in FP32) or 1
      v = make_float4(br.x * ascale, br.y * ascale, bq.x * ascale, bq.y * ascale);
    }
    Bs[t] = v;
  }
  __syncthreads();
  if (row >= nr) return;
  // columns in groups of DS_NG (accumulators of a group in registers; a small loop
  // body, 2 DS_NG independent accumulation chains)
  cplx* crow = C + int64_t(row) * P.N + j0;
  for (int g0 = 0; g0 < nc; g0 += DS_NG) {
    float sr[DS_NG], cr[DS_NG], si[DS_NG], ci[DS_NG];
#pragma unroll
    for (int u = 0; u < DS_NG; ++u) sr[u] = cr[u] = si[u] = ci[u] = 0.f;
    for (int k = 0; k < P.K; ++k) {
      const float4 a = As[row * DS_AST + k];
#pragma unroll
      for (int u = 0; u < DS_NG; ++u) {
        const float4 b = Bs[k * DS_NC + g0 + u];  // zero past nc
        ds_mac(sr[u], cr[u], a.x, a.y, b.x, b.y);    // Re += Re a Re b
        ds_mac(sr[u], cr[u], -a.z, -a.w, b.z, b.w);  //     - Im a Im b
        ds_mac(si[u], ci[u], a.x, a.y, b.z, b.w);    // Im += Re a Im b
        ds_mac(si[u], ci[u], a.z, a.w, b.x, b.y);    //     + Im a Re b
      }
    }
#pragma unroll
    for (int u = 0; u < DS_NG; ++u) {
      if (g0 + u < nc) {
        double vr = ds_to_double(sr[u], cr[u]), vi = ds_to_double(si[u], ci[u]);
        if (beta) {
          const cplx o = crow[g0 + u];
          vr += o.x;
          vi += o.y;
        }
        crow[g0 + u] = make_double2(vr, vi);
      }
    }
  }
}

bool ds_wanted(Ctx& c, const GemmPlan& g) {
  if (c.cfg.precision != EXP_EMU_BF16 || g.dot_outputs || g.h_probs.empty()) return false;
  int kmax = 0;
  for (const GemmProb& p : g.h_probs) kmax = std::max(kmax, p.K);
  return kmax >= 1 && kmax <= DS_KMAX;
}

void ds_prepare(Ctx& c, GemmPlan& g) {
  if (g.d_ds) return;
  for (const GemmProb& p : g.h_probs)
    if (p.K > DS_KMAX) throw ExpError{EXP_EINVAL, "double-single GEMM: K above 16"};
  std::vector<GemmProb> v = g.h_probs;
  int tiles = 0;
  for (GemmProb& p : v) {  // CTAs: DS_ROWS rows x DS_NC columns, column chunks adjacent
    p.tiles_m = (p.M + DS_ROWS - 1) / DS_ROWS;
    p.tiles_n = (p.N + DS_NC - 1) / DS_NC;
    p.tile0 = tiles;
    tiles += p.tiles_m * p.tiles_n;
  }
  g.ds_tiles = tiles;
  g.d_ds = (GemmProb*)c.dalloc(sizeof(GemmProb) * std::max<size_t>(v.size(), 1));
  upload(c, g.d_ds, v.data(), sizeof(GemmProb) * v.size());
}

void launch_gemm_ds(Ctx& c, const GemmPlan& g, const cplx* A, const cplx* B, cplx* C, int64_t ais, int64_t bis,
                    int64_t cis, cplx alpha, bool beta) {
  if (!g.d_ds) throw ExpError{EXP_ESTATE, "double-single GEMM not prepared"};
  if (g.ds_tiles == 0) return;
  // alpha = +-2^k folds into the FP32 parts exactly; any other alpha multiplies B in FP64
  int ex = 0;
  const double fr = std::frexp(std::fabs(alpha.x), &ex);
  const bool pow2 = alpha.y == 0.0 && fr == 0.5 && ex > -100 && ex < 100;
  k_gemm_ds<<<dim3(g.ds_tiles, c.ninst), DS_ROWS, 0, c.stream>>>(g.d_ds, g.n_probs, A, B, C, ais, bis, cis, alpha,
                                                                 pow2 ? float(alpha.x) : 1.0f, pow2 ? 0 : 1,
                                                                 beta ? 1 : 0);
  KCHECK(c);
}
