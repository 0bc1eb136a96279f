// Learned initial guess for T2: a 3-layer MLP (width 128) mapping per-element
// features to a complex multiplier of the first-order amplitude,
//     x = (|t_MP2| / 0.05, -D / 10, |<ij||ab>| / max|<ij||ab>|),
//     h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3,
//     t2 = (1 + y0 + i y1) t_MP2,
// trained on converged amplitudes of earlier solves (loss: mean |t2 - t2_conv|^2 /
// 0.05^2, Adam).  Hand-written forward, backward and update kernels.  bf16 mode:
// weights and activations rounded to BF16, and the three width-128 layer products
// (h1 W2^T forward, gz2 W2 and gz2^T h1 backward, the gradients rounded to BF16 as
// operands) on the tensor cores, mma m16n8k16 with FP32 accumulation; check mode:
// plain FP32 on the SIMT pipes.  The paper has no counterpart; the guess only changes
// the starting point of the amplitude iteration, never its fixed point.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "ccsd.h"

namespace {
constexpr int NF = 3, W = 128, NO = 2;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + W * NF, OFF_W2 = OFF_B1 + W, OFF_B2 = OFF_W2 + W * W,
              OFF_W3 = OFF_B2 + W, OFF_B3 = OFF_W3 + NO * W, NPARAM = OFF_B3 + NO;
constexpr int TS = 32;  // samples per CTA tile
constexpr int MLP_SMEM = (2 * W * W + W * NF + 2 * W + NO * W + NO + 3 * TS * W + TS * NF + TS * NO) * 4 + 64;

__device__ __forceinline__ float rb(float x, int bf) { return bf ? __bfloat162float(__float2bfloat16_rn(x)) : x; }

// ---------------------------------------------------------------------------
// The width-128 layer products in the bf16 mode run on the tensor cores: warp-level
// mma.m16n8k16 with BF16 operands and FP32 accumulation.  Fragment layout (PTX ISA,
// m16n8k16 .bf16; g = lane / 4, t = lane % 4): A registers {(g, 2t), (g + 8, 2t),
// (g, 2t + 8), (g + 8, 2t + 8)} with the next column in the high half; B registers
// {(2t, g), (2t + 8, g)} with the next row in the high half; D {(g, 2t), (g, 2t + 1),
// (g + 8, 2t), (g + 8, 2t + 1)}.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// D[16 x 8] += A[r0 .. r0+16, k0 .. k0+16] B[k0 .. k0+16, c0 .. c0+8] for element accessors
// A(r, k), B(k, c) (values already on the BF16 grid, or rounded here)
template <typename FA, typename FB>
__device__ __forceinline__ void mma_tile(float (&d)[4], int r0, int c0, int k0, FA A, FB B) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t a[4] = {pack_bf16(A(r0 + g, k0 + 2 * t), A(r0 + g, k0 + 2 * t + 1)),
                         pack_bf16(A(r0 + g + 8, k0 + 2 * t), A(r0 + g + 8, k0 + 2 * t + 1)),
                         pack_bf16(A(r0 + g, k0 + 2 * t + 8), A(r0 + g, k0 + 2 * t + 9)),
                         pack_bf16(A(r0 + g + 8, k0 + 2 * t + 8), A(r0 + g + 8, k0 + 2 * t + 9))};
  const uint32_t b[2] = {pack_bf16(B(k0 + 2 * t, c0 + g), B(k0 + 2 * t + 1, c0 + g)),
                         pack_bf16(B(k0 + 2 * t + 8, c0 + g), B(k0 + 2 * t + 9, c0 + g))};
  mma_16816(d, a, b);
}

struct Smem {
  float* W2;   // [u][k]
  float* W2T;  // [k][u]
  float* W1;   // [u][f]
  float* b1;
  float* b2;
  float* W3;   // [o][k]
  float* b3;
  float* h1;   // [s][u]
  float* h2;
  float* g;    // [s][u] gradient scratch
  float* x;    // [s][f]
  float* gy;   // [s][o]
};

__device__ Smem carve(float* base) {
  Smem m;
  m.W2 = base;
  m.W2T = m.W2 + W * W;
  m.W1 = m.W2T + W * W;
  m.b1 = m.W1 + W * NF;
  m.b2 = m.b1 + W;
  m.W3 = m.b2 + W;
  m.b3 = m.W3 + NO * W;
  m.h1 = m.b3 + NO;
  m.h2 = m.h1 + TS * W;
  m.g = m.h2 + TS * W;
  m.x = m.g + TS * W;
  m.gy = m.x + TS * NF;
  return m;
}

__device__ void load_params(const float* __restrict__ P, Smem& m, int bf) {
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
    const int u = e / W, k = e % W;
    const float v = rb(P[OFF_W2 + e], bf);
    m.W2[e] = v;
    m.W2T[k * W + u] = v;
  }
  for (int e = threadIdx.x; e < W * NF; e += blockDim.x) m.W1[e] = rb(P[OFF_W1 + e], bf);
  for (int e = threadIdx.x; e < W; e += blockDim.x) { m.b1[e] = P[OFF_B1 + e]; m.b2[e] = P[OFF_B2 + e]; }
  for (int e = threadIdx.x; e < NO * W; e += blockDim.x) m.W3[e] = rb(P[OFF_W3 + e], bf);
  if (threadIdx.x < NO) m.b3[threadIdx.x] = P[OFF_B3 + threadIdx.x];
}

// forward for the TS samples whose features sit in m.x (ns valid); y into m.gy
__device__ void forward_tile(Smem& m, int ns, int bf) {
  for (int e = threadIdx.x; e < TS * W; e += blockDim.x) {
    const int s = e / W, u = e % W;
    float z = m.b1[u];
#pragma unroll
    for (int f = 0; f < NF; ++f) z += m.W1[u * NF + f] * m.x[s * NF + f];
    m.h1[e] = s < ns ? rb(fmaxf(z, 0.f), bf) : 0.f;
  }
  __syncthreads();
  if (bf) {
    // z2 = h1 W2^T on the tensor cores: warp w takes the 16 units 16w .. 16w + 15 of all
    // TS = 32 samples (two 16-row by two 8-column tiles, K = 128 in steps of 16)
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float d[2][2][4] = {};
    auto A = [&](int r, int k) { return m.h1[r * W + k]; };
    auto B = [&](int k, int c) { return m.W2[c * W + k]; };
#pragma unroll
    for (int k0 = 0; k0 < W; k0 += 16)
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) mma_tile(d[mt][nt], 16 * mt, 16 * w + 8 * nt, k0, A, B);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int s = 16 * mt + g + (q >> 1) * 8, u = 16 * w + 8 * nt + 2 * t + (q & 1);
          m.h2[s * W + u] = s < ns ? rb(fmaxf(d[mt][nt][q] + m.b2[u], 0.f), bf) : 0.f;
        }
  } else {
    for (int e = threadIdx.x; e < TS * W; e += blockDim.x) {
      const int s = e / W, u = e % W;
      float z = m.b2[u];
      for (int k = 0; k < W; ++k) z += m.W2T[k * W + u] * m.h1[s * W + k];
      m.h2[e] = s < ns ? rb(fmaxf(z, 0.f), bf) : 0.f;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TS * NO; e += blockDim.x) {
    const int s = e / NO, o = e % NO;
    float y = m.b3[o];
    for (int k = 0; k < W; ++k) y += m.W3[o * W + k] * m.h2[s * W + k];
    m.gy[e] = y;
  }
  __syncthreads();
}

// Gradient of the batch loss: idx[b0 .. b0+nb) index the sample arrays.  Each CTA
// walks tiles of TS samples (grid-stride) and keeps its gradient contributions in
// registers / shared memory owned by one thread each; one atomicAdd per entry per
// CTA at the end.
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ X,
                                                  const float2* __restrict__ TM, const float2* __restrict__ TG,
                                                  const int* __restrict__ idx, int b0, int nb, float inv_n,
                                                  float* __restrict__ grad, double* __restrict__ loss, int bf) {
  extern __shared__ float sm[];
  Smem m = carve(sm);
  __shared__ float aW1[W * NF], ab1[W], ab2[W];
  __shared__ float lsum[TS];
  load_params(P, m, bf);
  float gW2[W * W / 256];  // entries threadIdx.x + 256 j
  float gW3 = 0.f, gb3 = 0.f;
#pragma unroll
  for (int j = 0; j < W * W / 256; ++j) gW2[j] = 0.f;
  for (int e = threadIdx.x; e < W * NF; e += blockDim.x) aW1[e] = 0.f;
  for (int e = threadIdx.x; e < W; e += blockDim.x) { ab1[e] = 0.f; ab2[e] = 0.f; }
  double lacc = 0.0;
  const int ntile = (nb + TS - 1) / TS;
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int t0 = b0 + tile * TS;
    const int ns = max(0, min(TS, b0 + nb - t0));
    __syncthreads();
    for (int e = threadIdx.x; e < TS * NF; e += blockDim.x) {
      const int s = e / NF;
      m.x[e] = s < ns ? X[int64_t(idx[t0 + s]) * NF + e % NF] : 0.f;
    }
    __syncthreads();
    forward_tile(m, ns, bf);
    if (threadIdx.x < TS) {
      const int s = threadIdx.x;
      float l = 0.f, g0 = 0.f, g1 = 0.f;
      if (s < ns) {
        const float2 tm = TM[idx[t0 + s]], tg = TG[idx[t0 + s]];
        const float mr = 1.f + m.gy[s * NO], mi = m.gy[s * NO + 1];
        const float rr = mr * tm.x - mi * tm.y - tg.x, ri = mr * tm.y + mi * tm.x - tg.y;
        const float c = 2.f * inv_n / (0.05f * 0.05f);
        l = (rr * rr + ri * ri) / (0.05f * 0.05f);
        g0 = c * (rr * tm.x + ri * tm.y);   // Re(conj(r) tmp2)
        g1 = c * (-rr * tm.y + ri * tm.x);  // Re(conj(r) i tmp2)
      }
      lsum[s] = l;
      m.gy[s * NO] = g0;
      m.gy[s * NO + 1] = g1;
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int s = 0; s < TS; ++s) lacc += lsum[s];
    {  // output layer: entry threadIdx.x of W3 (NO * W == 256)
      const int o = threadIdx.x / W, k = threadIdx.x % W;
      for (int s = 0; s < ns; ++s) gW3 += m.gy[s * NO + o] * m.h2[s * W + k];
      if (threadIdx.x < NO)
        for (int s = 0; s < ns; ++s) gb3 += m.gy[s * NO + threadIdx.x];
    }
    for (int e = threadIdx.x; e < TS * W; e += blockDim.x) {  // gz2 = (gy W3) . relu'(z2)
      const int s = e / W, u = e % W;
      float a = 0.f;
#pragma unroll
      for (int o = 0; o < NO; ++o) a += m.gy[s * NO + o] * m.W3[o * W + u];
      m.g[e] = m.h2[e] > 0.f ? a : 0.f;
    }
    __syncthreads();
    if (bf) {
      // gW2 += gz2^T h1 on the tensor cores (gz2 rounded to BF16): warp w holds the 16 rows
      // u = 16w .. 16w + 15 of all 128 columns, 16 column tiles x 4 entries per thread
      const int w = threadIdx.x >> 5;
      auto A = [&](int u, int sm_) { return m.g[sm_ * W + u]; };
      auto B = [&](int sm_, int k) { return m.h1[sm_ * W + k]; };
#pragma unroll
      for (int k0 = 0; k0 < TS; k0 += 16)
#pragma unroll
        for (int nt = 0; nt < W / 8; ++nt) {
          float* acc = gW2 + 4 * nt;
          float d[4] = {acc[0], acc[1], acc[2], acc[3]};
          mma_tile(d, 16 * w, 8 * nt, k0, A, B);
          acc[0] = d[0];
          acc[1] = d[1];
          acc[2] = d[2];
          acc[3] = d[3];
        }
    } else {
#pragma unroll
      for (int j = 0; j < W * W / 256; ++j) {
        const int e = threadIdx.x + 256 * j, u = e / W, k = e % W;
        float a = 0.f;
        for (int s = 0; s < ns; ++s) a += m.g[s * W + u] * m.h1[s * W + k];
        gW2[j] += a;
      }
    }
    if (threadIdx.x < W) {
      float a = 0.f;
      for (int s = 0; s < ns; ++s) a += m.g[s * W + threadIdx.x];
      ab2[threadIdx.x] += a;
    }
    __syncthreads();
    if (bf) {  // gz1 = (gz2 W2) . relu'(z1), over h2: on the tensor cores, warp w the columns 16w ..
      const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
      float d[2][2][4] = {};
      auto A = [&](int sm_, int u) { return m.g[sm_ * W + u]; };
      auto B = [&](int u, int k) { return m.W2T[k * W + u]; };
#pragma unroll
      for (int k0 = 0; k0 < W; k0 += 16)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) mma_tile(d[mt][nt], 16 * mt, 16 * w + 8 * nt, k0, A, B);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int sm_ = 16 * mt + g + (q >> 1) * 8, k = 16 * w + 8 * nt + 2 * t + (q & 1);
            m.h2[sm_ * W + k] = m.h1[sm_ * W + k] > 0.f ? d[mt][nt][q] : 0.f;
          }
    } else {
      for (int e = threadIdx.x; e < TS * W; e += blockDim.x) {  // gz1 = (gz2 W2) . relu'(z1), over h2
        const int s = e / W, k = e % W;
        float a = 0.f;
        for (int u = 0; u < W; ++u) a += m.g[s * W + u] * m.W2[u * W + k];
        m.h2[e] = m.h1[e] > 0.f ? a : 0.f;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < W * NF; e += blockDim.x) {
      const int u = e / NF, f = e % NF;
      float a = 0.f;
      for (int s = 0; s < ns; ++s) a += m.h2[s * W + u] * m.x[s * NF + f];
      aW1[e] += a;
    }
    if (threadIdx.x < W) {
      float a = 0.f;
      for (int s = 0; s < ns; ++s) a += m.h2[s * W + threadIdx.x];
      ab1[threadIdx.x] += a;
    }
  }
  __syncthreads();
  if (bf) {  // gW2 fragments: warp w rows 16w + g (+8), column tile nt, columns 2t (+1)
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < W / 8; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int u = 16 * w + g + (q >> 1) * 8, k = 8 * nt + 2 * t + (q & 1);
        atomicAdd(&grad[OFF_W2 + u * W + k], gW2[4 * nt + q]);
      }
  } else {
#pragma unroll
    for (int j = 0; j < W * W / 256; ++j) atomicAdd(&grad[OFF_W2 + threadIdx.x + 256 * j], gW2[j]);
  }
  atomicAdd(&grad[OFF_W3 + threadIdx.x], gW3);
  if (threadIdx.x < NO) atomicAdd(&grad[OFF_B3 + threadIdx.x], gb3);
  for (int e = threadIdx.x; e < W * NF; e += blockDim.x) atomicAdd(&grad[OFF_W1 + e], aW1[e]);
  for (int e = threadIdx.x; e < W; e += blockDim.x) {
    atomicAdd(&grad[OFF_B1 + e], ab1[e]);
    atomicAdd(&grad[OFF_B2 + e], ab2[e]);
  }
  if (threadIdx.x == 0) atomicAdd(loss, lacc * inv_n);
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M1,
                       float* __restrict__ M2, int step, float lr) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NPARAM) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float g = G[k];
  const float m = b1 * M1[k] + (1.f - b1) * g, v = b2 * M2[k] + (1.f - b2) * g * g;
  M1[k] = m;
  M2[k] = v;
  const float mh = m / (1.f - powf(b1, float(step))), vh = v / (1.f - powf(b2, float(step)));
  P[k] -= lr * mh / (sqrtf(vh) + eps);
}

// features of element p of instance inst from <ab||ij> (Vd), D and the instance's max |V|
__device__ __forceinline__ void elem_features(cplx v, double d, float vmax, float* x, float2* tm) {
  const double ar = v.x / d, ai = v.y / d;
  *tm = make_float2(float(ar), float(ai));
  x[0] = float(hypot(ar, ai) / 0.05);
  x[1] = float(-d / 10.0);
  x[2] = vmax > 0.f ? float(hypot(v.x, v.y)) / vmax : 0.f;
}

__global__ void k_vmax(const cplx* __restrict__ V, int64_t vis, int64_t n2, float* __restrict__ vmax) {
  const int inst = blockIdx.y;
  float m = 0.f;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n2; k += int64_t(gridDim.x) * blockDim.x) {
    const cplx v = V[inst * vis + k];
    m = fmaxf(m, float(hypot(v.x, v.y)));
  }
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax((int*)&vmax[inst], __float_as_int(m));  // m >= 0: int order = float order
}

// training samples from the unique elements (a<b, i<j, no ghost) of converged instances
__global__ void k_extract(const cplx* __restrict__ V, int64_t vis, const double* __restrict__ D, const cplx* __restrict__ T,
                          int64_t namp, int64_t n1, const int64_t* __restrict__ elems, int ne,
                          const float* __restrict__ vmax, const int* __restrict__ inst_list, float* __restrict__ X,
                          float2* __restrict__ TM, float2* __restrict__ TG, int64_t base) {
  const int ii = blockIdx.y;
  const int inst = inst_list[ii];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += gridDim.x * blockDim.x) {
    const int64_t p = elems[k];
    const int64_t o = base + int64_t(ii) * ne + k;
    float x[NF];
    float2 tm;
    elem_features(V[inst * vis + p], D[inst * namp + n1 + p], vmax[inst], x, &tm);
    for (int f = 0; f < NF; ++f) X[o * NF + f] = x[f];
    TM[o] = tm;
    const cplx t = T[inst * namp + n1 + p];
    TG[o] = make_float2(float(t.x), float(t.y));
  }
}

// inference over every t2 element of every instance: t2 = (1 + y0 + i y1) <ab||ij> / D
__global__ void __launch_bounds__(256) k_mlp_apply(const float* __restrict__ P, const cplx* __restrict__ V, int64_t vis,
                                                   const double* __restrict__ D, cplx* __restrict__ T, int64_t namp,
                                                   int64_t n1, int64_t n2, const float* __restrict__ vmax, int bf) {
  extern __shared__ float sm[];
  Smem m = carve(sm);
  load_params(P, m, bf);
  const int inst = blockIdx.y;
  __syncthreads();
  for (int64_t t0 = int64_t(blockIdx.x) * TS; t0 < n2; t0 += int64_t(gridDim.x) * TS) {
    const int ns = int(n2 - t0 < TS ? n2 - t0 : TS);
    for (int e = threadIdx.x; e < TS; e += blockDim.x) {
      if (e < ns) {
        float2 tm;
        elem_features(V[inst * vis + t0 + e], D[inst * namp + n1 + t0 + e], vmax[inst], &m.x[e * NF], &tm);
      } else {
        for (int f = 0; f < NF; ++f) m.x[e * NF + f] = 0.f;
      }
    }
    __syncthreads();
    forward_tile(m, ns, bf);
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
      const cplx v = V[inst * vis + t0 + s];
      const double d = D[inst * namp + n1 + t0 + s];
      const double mr = 1.0 + m.gy[s * NO], mi = m.gy[s * NO + 1];
      const double ar = v.x / d, ai = v.y / d;
      T[inst * namp + n1 + t0 + s] = make_double2(mr * ar - mi * ai, mr * ai + mi * ar);
    }
    __syncthreads();
  }
}

__global__ void k_zero_t1(cplx* __restrict__ T, int64_t namp, int64_t n1) {
  const int inst = blockIdx.y;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n1; k += int64_t(gridDim.x) * blockDim.x)
    T[inst * namp + k] = make_double2(0.0, 0.0);
}

__global__ void k_init_params(float* __restrict__ P, uint64_t seed) {
  // He-style initialisation of W1, W2 from a hashed counter; zero biases and output layer
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NPARAM) return;
  float v = 0.f;
  if (k < OFF_B1 || (k >= OFF_W2 && k < OFF_B2)) {
    uint64_t z = seed * 0x9E3779B97F4A7C15ull + uint64_t(k) * 0xBF58476D1CE4E5B9ull;
    z ^= z >> 31; z *= 0x94D049BB133111EBull; z ^= z >> 29;
    const float u1 = ((z >> 11) + 0.5f) * 0x1p-53f, u2 = (((z * 0x2545F4914F6CDD1Dull) >> 11) + 0.5f) * 0x1p-53f;
    const float g = sqrtf(-2.f * logf(u1)) * cosf(6.2831853f * u2);
    v = g * (k < OFF_B1 ? sqrtf(2.f / NF) : sqrtf(2.f / W));
  }
  P[k] = v;
}
}  // namespace

// ---------------------------------------------------------------------------
struct exp_mlp {
  exp_allocator alloc{};
  cudaStream_t stream = nullptr;
  int bf = 1;
  int step = 0;
  float* P = nullptr;
  float* G = nullptr;
  float* M1 = nullptr;
  float* M2 = nullptr;
  double* d_loss = nullptr;
  float* X = nullptr;
  float2* TM = nullptr;
  float2* TG = nullptr;
  int* idx = nullptr;
  int64_t n = 0, cap = 0;
  std::vector<void*> owned;
  std::string err;
  void* al(size_t b) {
    void* p = alloc.alloc(std::max<size_t>(b, 256), alloc.user);
    if (!p) throw ExpError{EXP_ENOMEM, "allocator returned NULL"};
    owned.push_back(p);
    return p;
  }
};

static thread_local std::string g_mlp_err;

#define MLP_TRY try {
#define MLP_CATCH(m)                                                                     \
  }                                                                                      \
  catch (const ExpError& e) {                                                            \
    g_mlp_err = e.msg;                                                                   \
    if (m) (m)->err = e.msg;                                                             \
    return e.s;                                                                          \
  }                                                                                      \
  catch (const CudaError& e) {                                                           \
    g_mlp_err = std::string(e.where) + ": " + cudaGetErrorString(e.e);                   \
    if (m) (m)->err = g_mlp_err;                                                         \
    return EXP_ECUDA;                                                                    \
  }

extern "C" int exp_mlp_num_params(void) { return NPARAM; }

extern "C" exp_status exp_mlp_create(const exp_allocator* alloc, void* stream, uint64_t seed, int bf16,
                                     exp_mlp** out) {
  exp_mlp* m = nullptr;
  MLP_TRY
  if (!alloc || !alloc->alloc || !alloc->free || !out) throw ExpError{EXP_EINVAL, "null argument"};
  m = new exp_mlp();
  m->alloc = *alloc;
  m->stream = (cudaStream_t)stream;
  m->bf = bf16 ? 1 : 0;
  m->P = (float*)m->al(sizeof(float) * NPARAM);
  m->G = (float*)m->al(sizeof(float) * NPARAM);
  m->M1 = (float*)m->al(sizeof(float) * NPARAM);
  m->M2 = (float*)m->al(sizeof(float) * NPARAM);
  m->d_loss = (double*)m->al(sizeof(double));
  CK(cudaMemsetAsync(m->M1, 0, sizeof(float) * NPARAM, m->stream));
  CK(cudaMemsetAsync(m->M2, 0, sizeof(float) * NPARAM, m->stream));
  k_init_params<<<(NPARAM + 255) / 256, 256, 0, m->stream>>>(m->P, seed);
  CK(cudaGetLastError());
  CK(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, MLP_SMEM));
  CK(cudaFuncSetAttribute(k_mlp_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, MLP_SMEM));
  CK(cudaStreamSynchronize(m->stream));
  *out = m;
  return EXP_OK;
  }
  catch (const ExpError& e) {
    g_mlp_err = e.msg;
    if (m) { for (void* p : m->owned) m->alloc.free(p, m->alloc.user); delete m; }
    return e.s;
  }
  catch (const CudaError& e) {
    g_mlp_err = std::string(e.where) + ": " + cudaGetErrorString(e.e);
    if (m) { for (void* p : m->owned) m->alloc.free(p, m->alloc.user); delete m; }
    return EXP_ECUDA;
  }
}

extern "C" void exp_mlp_destroy(exp_mlp* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  for (void* p : m->owned) m->alloc.free(p, m->alloc.user);
  delete m;
}

extern "C" const char* exp_mlp_last_error(const exp_mlp* m) {
  return m && !m->err.empty() ? m->err.c_str() : g_mlp_err.c_str();
}

extern "C" exp_status exp_mlp_params(exp_mlp* m, float* get, const float* set) {
  MLP_TRY
  if (!m) throw ExpError{EXP_EINVAL, "null model"};
  if (set) {
    CK(cudaMemcpyAsync(m->P, set, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, m->stream));
    CK(cudaMemsetAsync(m->M1, 0, sizeof(float) * NPARAM, m->stream));
    CK(cudaMemsetAsync(m->M2, 0, sizeof(float) * NPARAM, m->stream));
    m->step = 0;
  }
  if (get) CK(cudaMemcpyAsync(get, m->P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return EXP_OK;
  MLP_CATCH(m)
}

static void ensure_capacity(exp_mlp* m, int64_t need) {
  if (need <= m->cap) return;
  const int64_t cap = std::max<int64_t>(need, 2 * m->cap);
  float* X = (float*)m->al(sizeof(float) * NF * cap);
  float2* TM = (float2*)m->al(sizeof(float2) * cap);
  float2* TG = (float2*)m->al(sizeof(float2) * cap);
  int* idx = (int*)m->al(sizeof(int) * cap);
  if (m->n) {
    CK(cudaMemcpyAsync(X, m->X, sizeof(float) * NF * m->n, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(TM, m->TM, sizeof(float2) * m->n, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(TG, m->TG, sizeof(float2) * m->n, cudaMemcpyDeviceToDevice, m->stream));
  }
  m->X = X;
  m->TM = TM;
  m->TG = TG;
  m->idx = idx;
  m->cap = cap;
}

// vmax per instance of a context, on the context stream
static float* ctx_vmax(exp_mlp* m, Ctx& c) {
  const Tensor* Vd = ccsd_driver_integral(c);
  float* vm = (float*)m->al(sizeof(float) * c.ninst);
  CK(cudaMemsetAsync(vm, 0, sizeof(float) * c.ninst, c.stream));
  k_vmax<<<dim3(std::max<int64_t>(1, std::min<int64_t>((c.n2 + 255) / 256, 304)), c.ninst), 256, 0, c.stream>>>(
      Vd->d, Vd->is, c.n2, vm);
  CK(cudaGetLastError());
  return vm;
}

extern "C" exp_status exp_mlp_add_training_data(exp_mlp* m, exp_ctx* x) {
  MLP_TRY
  if (!m || !x) throw ExpError{EXP_EINVAL, "null argument"};
  Ctx& c = x->c;
  if (!c.guessed) throw ExpError{EXP_ESTATE, "context has no amplitudes"};
  CK(cudaStreamSynchronize(m->stream));
  // converged instances only
  std::vector<int> st(4 * c.ninst), list;
  CK(cudaMemcpy(st.data(), c.d_diis_state, sizeof(int) * 4 * c.ninst, cudaMemcpyDeviceToHost));
  for (int k = 0; k < c.ninst; ++k)
    if (st[k * 4 + 2] == 1) list.push_back(k);  // converged (2 = failed)
  if (list.empty()) return EXP_OK;
  // unique real elements a<b, i<j of the t2 layout
  std::vector<SubBlock> sb;
  enumerate_blocks(c.t2.L, c.spaces, sb);
  std::vector<int64_t> el;
  const Space& SO = c.spaces[SP_OCC];
  const Space& SV = c.spaces[SP_VIRT];
  for (auto& b : sb)
    for (int la = 0; la < b.n[0]; ++la)
      for (int lb = 0; lb < b.n[1]; ++lb) {
        const int ga = SV.off[b.irr[0]] + la, gb = SV.off[b.irr[1]] + lb;
        if (ga >= gb) continue;
        for (int li = 0; li < b.n[2]; ++li)
          for (int lj = 0; lj < b.n[3]; ++lj) {
            const int gi = SO.off[b.irr[2]] + li, gj = SO.off[b.irr[3]] + lj;
            if (gi >= gj || c.occ_real[gi] < 0 || c.occ_real[gj] < 0) continue;
            el.push_back(b.base + la * b.st[0] + lb * b.st[1] + li * b.st[2] + lj * b.st[3]);
          }
      }
  const int ne = int(el.size());
  const int64_t add = int64_t(ne) * list.size();
  ensure_capacity(m, m->n + add);
  CK(cudaStreamSynchronize(m->stream));
  int64_t* d_el = (int64_t*)c.dalloc(sizeof(int64_t) * std::max(ne, 1));
  int* d_list = (int*)c.dalloc(sizeof(int) * list.size());
  upload(c, d_el, el.data(), sizeof(int64_t) * ne);
  upload(c, d_list, list.data(), sizeof(int) * list.size());
  float* vm = ctx_vmax(m, c);
  const Tensor* Vd = ccsd_driver_integral(c);
  k_extract<<<dim3(std::max(1, std::min((ne + 255) / 256, 1024)), int(list.size())), 256, 0, c.stream>>>(
      Vd->d, Vd->is, c.d_D, c.d_T, c.namp, c.n1, d_el, ne, vm, d_list, m->X, m->TM, m->TG, m->n);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c.stream));
  m->n += add;
  return EXP_OK;
  MLP_CATCH(m)
}

static void grad_batch(exp_mlp* m, const float* X, const float2* TM, const float2* TG, const int* idx, int64_t b0,
                       int64_t nb) {
  CK(cudaMemsetAsync(m->G, 0, sizeof(float) * NPARAM, m->stream));
  const int blocks = int(std::min<int64_t>((nb + TS - 1) / TS, 304));
  k_mlp_grad<<<blocks, 256, MLP_SMEM, m->stream>>>(m->P, X, TM, TG, idx, int(b0), int(nb), 1.f / float(nb), m->G,
                                                   m->d_loss, m->bf);
  CK(cudaGetLastError());
}

extern "C" exp_status exp_mlp_train(exp_mlp* m, int epochs, int batch, double lr, uint64_t seed, double* loss_out) {
  MLP_TRY
  if (!m || epochs < 0 || batch < 1 || !(lr > 0)) throw ExpError{EXP_EINVAL, "bad argument"};
  if (m->n == 0) throw ExpError{EXP_ESTATE, "no training data"};
  std::vector<int> perm(m->n);
  std::mt19937_64 rng(seed);
  for (int ep = 0; ep < epochs; ++ep) {
    std::iota(perm.begin(), perm.end(), 0);
    std::shuffle(perm.begin(), perm.end(), rng);
    CK(cudaMemcpyAsync(m->idx, perm.data(), sizeof(int) * m->n, cudaMemcpyHostToDevice, m->stream));
    CK(cudaMemsetAsync(m->d_loss, 0, sizeof(double), m->stream));
    int nbat = 0;
    for (int64_t b0 = 0; b0 < m->n; b0 += batch) {
      const int64_t nb = std::min<int64_t>(batch, m->n - b0);
      grad_batch(m, m->X, m->TM, m->TG, m->idx, b0, nb);
      ++m->step;
      k_adam<<<(NPARAM + 255) / 256, 256, 0, m->stream>>>(m->P, m->G, m->M1, m->M2, m->step, float(lr));
      CK(cudaGetLastError());
      ++nbat;
    }
    double l = 0.0;
    CK(cudaMemcpyAsync(&l, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));  // the permutation buffer is reused next epoch
    if (loss_out) loss_out[ep] = l / nbat;
  }
  return EXP_OK;
  MLP_CATCH(m)
}

extern "C" int64_t exp_mlp_num_samples(const exp_mlp* m) { return m ? m->n : 0; }

extern "C" exp_status exp_mlp_samples(exp_mlp* m, int64_t first, int64_t count, float* x, float* tmp2, float* target) {
  MLP_TRY
  if (!m || first < 0 || count < 0 || first + count > m->n) throw ExpError{EXP_EINVAL, "bad range"};
  if (x) CK(cudaMemcpyAsync(x, m->X + first * NF, sizeof(float) * NF * count, cudaMemcpyDeviceToHost, m->stream));
  if (tmp2) CK(cudaMemcpyAsync(tmp2, m->TM + first, sizeof(float2) * count, cudaMemcpyDeviceToHost, m->stream));
  if (target) CK(cudaMemcpyAsync(target, m->TG + first, sizeof(float2) * count, cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return EXP_OK;
  MLP_CATCH(m)
}

extern "C" exp_status exp_mlp_eval(exp_mlp* m, double* loss) {
  MLP_TRY
  if (!m || !loss) throw ExpError{EXP_EINVAL, "null argument"};
  if (m->n == 0) throw ExpError{EXP_ESTATE, "no training data"};
  std::vector<int> id(m->n);
  std::iota(id.begin(), id.end(), 0);
  CK(cudaMemcpyAsync(m->idx, id.data(), sizeof(int) * m->n, cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemsetAsync(m->d_loss, 0, sizeof(double), m->stream));
  grad_batch(m, m->X, m->TM, m->TG, m->idx, 0, m->n);
  CK(cudaMemcpyAsync(loss, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return EXP_OK;
  MLP_CATCH(m)
}

extern "C" exp_status exp_mlp_loss_grad(exp_mlp* m, int n, const float* x, const double* tmp2, const double* target,
                                        double* loss, float* grad) {
  MLP_TRY
  if (!m || n < 1 || !x || !tmp2 || !target) throw ExpError{EXP_EINVAL, "bad argument"};
  std::vector<float2> tm(n), tg(n);
  for (int k = 0; k < n; ++k) {
    tm[k] = make_float2(float(tmp2[2 * k]), float(tmp2[2 * k + 1]));
    tg[k] = make_float2(float(target[2 * k]), float(target[2 * k + 1]));
  }
  std::vector<int> id(n);
  std::iota(id.begin(), id.end(), 0);
  float* dX = (float*)m->al(sizeof(float) * NF * n);
  float2* dTM = (float2*)m->al(sizeof(float2) * n);
  float2* dTG = (float2*)m->al(sizeof(float2) * n);
  int* dI = (int*)m->al(sizeof(int) * n);
  CK(cudaMemcpyAsync(dX, x, sizeof(float) * NF * n, cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemcpyAsync(dTM, tm.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemcpyAsync(dTG, tg.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemcpyAsync(dI, id.data(), sizeof(int) * n, cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemsetAsync(m->d_loss, 0, sizeof(double), m->stream));
  grad_batch(m, dX, dTM, dTG, dI, 0, n);
  if (loss) CK(cudaMemcpyAsync(loss, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  if (grad) CK(cudaMemcpyAsync(grad, m->G, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return EXP_OK;
  MLP_CATCH(m)
}

extern "C" exp_status exp_mlp_apply(exp_mlp* m, exp_ctx* x) {
  MLP_TRY
  if (!m || !x) throw ExpError{EXP_EINVAL, "null argument"};
  Ctx& c = x->c;
  if (!c.have_integrals) throw ExpError{EXP_ESTATE, "exp_init_integrals must come first"};
  CK(cudaStreamSynchronize(m->stream));
  float* vm = ctx_vmax(m, c);
  const Tensor* Vd = ccsd_driver_integral(c);
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((c.n2 + TS - 1) / TS, 2 * 304)));
  k_mlp_apply<<<dim3(blocks, c.ninst), 256, MLP_SMEM, c.stream>>>(m->P, Vd->d, Vd->is, c.d_D, c.d_T, c.namp, c.n1,
                                                                   c.n2, vm, m->bf);
  CK(cudaGetLastError());
  k_zero_t1<<<dim3(std::max<int64_t>(1, std::min<int64_t>((c.n1 + 255) / 256, 64)), c.ninst), 256, 0, c.stream>>>(
      c.d_T, c.namp, c.n1);
  CK(cudaGetLastError());
  ccsd_mark_guessed(c);
  CK(cudaStreamSynchronize(c.stream));
  return EXP_OK;
  MLP_CATCH(m)
}
