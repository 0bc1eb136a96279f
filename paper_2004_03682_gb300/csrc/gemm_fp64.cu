// Plain complex-FP64 grouped GEMM: step 3 of the TTGT list (Sec. II.B), all
// symmetry blocks and instances of one contraction in one launch (the block
// loop of Fig. "mult" flattened into a tile list).  Row-major operands,
// C[MxN] = alpha A[MxK] B[KxN] (+ C).  SIMT FP64 FMA: GB300's FP64 rate is the
// roofline for this path.
#include <algorithm>

#include "engine.h"

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
