// The perturbative triples correction (T) to CCSD: the CCSD(T) model of the paper's
// model list (Sec. III.A), for a Hartree-Fock reference (f diagonal), evaluated on
// the amplitudes a context holds (converged, or set by the caller):
//
//   c_ijk^abc = P(i/jk) P(a/bc) [ sum_e <bc||ei> t_jk^ae - sum_m <ma||jk> t_im^bc ]
//   d_ijk^abc = P(i/jk) P(a/bc) t_i^a <bc||jk>
//   E(T)      = sum over i<j<k, a<b<c of conj(c + d) c / D_ijk^abc,
//   D_ijk^abc = e_i + e_j + e_k - e_a - e_b - e_c,
//
// with P(p/qr) f = f - f(p<->q) - f(p<->r) and the integrals <created created ||
// annihilated annihilated> of Eq. (ham).
//
// Contraction layout.  Before P(a/bc) the connected part is
// Y_ijk[a, bc] = X^(i;jk) - X^(j;ik) - X^(k;ji) with
//
//   X^(p;qr)[a, bc] = sum_e t_qr^ae <bc||ep> - sum_m <ma||qr> t_pm^bc
//                   = sum_k A_qr[a, k] B_p[k, bc],    k = (e | m),
//   A_qr[a, k] = [ t_qr^ae | -<ma||qr> ],    B_p[k, bc] = [ <bc||ep> ; t_pm^bc ].
//
// Under the Z_G symmetry of Sec. II.C, e and m carry the same irrep G = h - G(p)
// (h = G(b) + G(c)), and a carries G(q) + G(r) - G.  So for one p and one pair irrep h
// the contraction is a single matrix product with K = v_G + o_G: its B operand
// B_{p,h} is the same for the whole evaluation, its rows (q, r, a) run over every
// occupied pair of a block.  Y is antisymmetric in (b, c), so X keeps the pair-packed
// columns b < c only.
//
// Schedule.  The occupied spinors (irrep-sorted) are cut into blocks of nb.  The B
// members B_{p,h} are written and, in the emulated precision, sliced once.  For each
// block triple I <= J <= K the three orderings (I; J x K), (J; I x K), (K; J x I)
// gather their A members and run as one grouped product launch that writes X for
// every (p; q, r) the block triple's i<j<k need; then one CTA per triple i<j<k and
// pair irrep of (b, c) forms c (three X per P(a/bc) term), d, D and its energy.
// Fixed-order sums over the pair irreps, then over the triples, give the per-triple
// energies and E(T): the result does not depend on the launch configuration.  The
// element arithmetic runs in FP64 under EXP_FP64 and in double-single FP32 (about
// 48 bits, each pair's sum added in FP64) under the emulated precision, where the
// FP64 pipe would bound it.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "ccsd.h"
#include "emu.h"
#include "fpbits.h"
#include "gen.h"

namespace {

constexpr int T3_THREADS = 256;

// ---------------------------------------------------------------------------
// Index tables of one context (irrep-sorted local indices; global spinor index =
// occupied local index, or o + virtual local index).
struct T3Tables {
  int G = 1;
  const int* go = nullptr;     // [o] irrep of each occupied spinor
  const int* gv = nullptr;     // [v] irrep of each virtual spinor
  const int* girr = nullptr;   // [o + v] irrep of each global spinor index
  const int* voff = nullptr;   // [G] first virtual of each irrep
  const int* vcnt = nullptr;   // [G]
  const int* ooff = nullptr;   // [G]
  const int* ocnt = nullptr;   // [G]
  const int* npair = nullptr;  // [G] virtual pairs b < c per pair irrep
  const int* poff = nullptr;   // [G] their first entry in pairs
  const int32_t* pairs = nullptr;  // (b << 16 | c), b < c, grouped by pair irrep
  const int32_t* pidx = nullptr;   // [v * v] column of pair (b, c) in its irrep block + 1 (b < c), 0 otherwise
};

// Dense integral block dst[i0][i1][i2][i3] = scale <p q || r s>, the four V arguments
// taken from slots m[0..3] (global index g0[slot] + i[slot]); symmetry-forbidden
// tuples (G_p + G_q - G_r - G_s != 0 mod G) are zero, as in every stored block.
struct T3Dense4 {
  int n[4];
  int g0[4];
  int m[4];
};

__global__ void __launch_bounds__(T3_THREADS) k_t3_dense4(cplx* __restrict__ dst, T3Dense4 D, int64_t count, int ngen,
                                                          uint64_t seed, double sc, int real, const int* __restrict__ girr,
                                                          int G) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < count; e += int64_t(gridDim.x) * blockDim.x) {
    int64_t r = e;
    int i[4];
    i[3] = int(r % D.n[3]);
    r /= D.n[3];
    i[2] = int(r % D.n[2]);
    r /= D.n[2];
    i[1] = int(r % D.n[1]);
    i[0] = int(r / D.n[1]);
    int g[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) g[k] = D.g0[D.m[k]] + i[D.m[k]];
    const int s = girr[g[0]] + girr[g[1]] - girr[g[2]] - girr[g[3]];
    if (((s % G) + G) % G != 0) {
      dst[e] = make_double2(0.0, 0.0);
      continue;
    }
    const cplx v = v_element(uint64_t(g[0]), uint64_t(g[1]), uint64_t(g[2]), uint64_t(g[3]), uint64_t(ngen), seed);
    dst[e] = make_double2(sc * v.x, real ? 0.0 : sc * v.y);
  }
}

// One row of a B member B_{p,h} (K = v_G + o_G rows, npair[h] columns): rows k < v_G
// are <bc||ep> (e = voff[G] + k), the rest t_pm^bc (m = ooff[G] + k - v_G).
struct T3BRow {
  int64_t dst;  // element offset of the row in the B buffer
  int p, h;
  int kind;     // 0: integral row (index = e), 1: amplitude row (index = m)
  int index;
};

__global__ void __launch_bounds__(T3_THREADS) k_t3_brows(cplx* __restrict__ B, const T3BRow* __restrict__ rows,
                                                         T3Tables T, const cplx* __restrict__ t2, int o, int v, int ngen,
                                                         uint64_t seed, double sc, int real) {
  const T3BRow R = rows[blockIdx.x];
  const int n = T.npair[R.h];
  const int32_t* pr = T.pairs + T.poff[R.h];
  cplx* dst = B + R.dst;
  for (int u = threadIdx.x; u < n; u += blockDim.x) {
    const int b = pr[u] >> 16, c = pr[u] & 0xFFFF;
    if (R.kind == 0) {
      const cplx x = v_element(uint64_t(o + b), uint64_t(o + c), uint64_t(o + R.index), uint64_t(R.p), uint64_t(ngen), seed);
      dst[u] = make_double2(sc * x.x, real ? 0.0 : sc * x.y);
    } else {
      dst[u] = t2[((int64_t(R.p) * o + R.index) * v + b) * v + c];
    }
  }
}

// The rows (q, r, a) of one occupied pair in an A member of irrep G (K = v_G + o_G):
// [ t_qr^ae | -<ma||qr> ], read from the dense t2[q][r][a][e] and W[q][r][a][m] = <ma||qr>.
struct T3AUnit {
  int64_t dst;  // element offset of the pair's first row in the A buffer
  int q, r;
  int a0, na;   // first virtual and count of the irrep G(q) + G(r) - G
  int g;        // G
  int K;
};

__global__ void __launch_bounds__(T3_THREADS) k_t3_arows(cplx* __restrict__ A, const T3AUnit* __restrict__ units,
                                                         T3Tables T, const cplx* __restrict__ t2,
                                                         const cplx* __restrict__ W, int o, int v) {
  const T3AUnit U = units[blockIdx.x];
  const int ve = T.vcnt[U.g], e0 = T.voff[U.g], m0 = T.ooff[U.g];
  const int64_t qr = int64_t(U.q) * o + U.r;
  const int64_t n = int64_t(U.na) * U.K;
  for (int64_t x = threadIdx.x; x < n; x += blockDim.x) {
    const int al = int(x / U.K), k = int(x - int64_t(al) * U.K);
    const int a = U.a0 + al;
    cplx y;
    if (k < ve) {
      y = t2[(qr * v + a) * v + e0 + k];
    } else {
      const cplx w = W[(qr * v + a) * o + m0 + (k - ve)];
      y = make_double2(-w.x, -w.y);
    }
    A[U.dst + x] = y;
  }
}

// Where X^(p;qr) lives for one block triple: ordering w (0: (I; J x K), 1: (J; I x K),
// 2: (K; J x I)) has p in block P_w and pairs (q, r) in Q_w x R_w.
struct T3Block {
  int p0[3], q0[3], r0[3];  // first spinor of P_w, Q_w, R_w
  int nr[3];                // |R_w| (pair slot = (q - q0) |R_w| + (r - r0))
  int nb;                   // block size (stride of the per-p tables)
};

struct T3Tri {
  int i, j, k;
  int idx;  // position of the triple in the per-triple output (combinatorial number of i<j<k)
};

__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---------------------------------------------------------------------------
// Double-single arithmetic (x = hi + lo, two FP32 numbers, about 48 bits) for the
// per-element work of the emulated precision: GB300's FP32 pipe runs many times its
// FP64 rate.  Error-free sums (Knuth) and products (Dekker, through FMA) with the
// rounding intrinsics, so the compiler cannot contract them.
struct dsc {  // complex double-single
  float2 re, im;
};
__device__ __forceinline__ float2 ds_norm(float s, float e) {  // |e| small against s
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ float2 ds_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float z = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, z)), __fsub_rn(b.x, z));
  return ds_norm(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 ds_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 ds_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = __fmaf_rn(a.x, b.x, -p);
  return ds_norm(p, __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e)));
}
// 1 / a: the FP32 reciprocal refined by one Newton step in double-single
__device__ __forceinline__ float2 ds_rcp(float2 a) {
  const float r = __frcp_rn(a.x);
  const float2 q = ds_mul(a, make_float2(r, 0.f));
  const float2 e = ds_add(make_float2(1.f, 0.f), ds_neg(q));
  return ds_add(make_float2(r, 0.f), ds_mul(make_float2(r, 0.f), e));
}
__device__ __forceinline__ dsc dsc_of(cplx z) { return dsc{ds_split(z.x), ds_split(z.y)}; }
__device__ __forceinline__ dsc dsc_add(dsc a, dsc b) { return dsc{ds_add(a.re, b.re), ds_add(a.im, b.im)}; }
__device__ __forceinline__ dsc dsc_sub(dsc a, dsc b) { return dsc{ds_add(a.re, ds_neg(b.re)), ds_add(a.im, ds_neg(b.im))}; }
__device__ __forceinline__ dsc dsc_mul(dsc a, dsc b) {
  return dsc{ds_add(ds_mul(a.re, b.re), ds_neg(ds_mul(a.im, b.im))), ds_add(ds_mul(a.re, b.im), ds_mul(a.im, b.re))};
}

// Energy of one triple i<j<k and one pair irrep h of (b, c) per CTA: the sum over
// a<b<c with G_b + G_c = h (and G_a = G_i + G_j + G_k - h) of conj(c + d) c / D.
// Thread = pair (b, c) of h, looping over a < b.  The per-(ordering, pair irrep)
// bases of the three X blocks and of the pair's rows are formed once per CTA.  DS:
// the element arithmetic in double-single (the emulated precision), each pair's sum
// added in FP64; otherwise FP64 throughout.  Output: e3h[idx G + h].
template <bool DS>
__global__ void __launch_bounds__(T3_THREADS) k_t3_energy(const T3Tri* __restrict__ tris, T3Block Bk, T3Tables T,
                                                          const cplx* __restrict__ X, const int64_t* __restrict__ xoff,
                                                          const int32_t* __restrict__ rowoff,
                                                          const cplx* __restrict__ t1, const cplx* __restrict__ V,
                                                          const double* __restrict__ eps, int o, int v,
                                                          cplx* __restrict__ e3h) {
  const T3Tri tr = tris[blockIdx.x];
  const int h = blockIdx.y;
  const int G = T.G;
  __shared__ int64_t sxb[3][EXP_MAX_G];  // X block of ordering w, pair irrep hh: element offset
  __shared__ int32_t srb[3][EXP_MAX_G];  // its first row of the triple's pair (q, r)
  __shared__ int32_t snp[EXP_MAX_G];     // pairs per irrep
  __shared__ double red[2][T3_THREADS / 32];
  const int P[3] = {tr.i, tr.j, tr.k}, Q[3] = {tr.j, tr.i, tr.j}, R[3] = {tr.k, tr.k, tr.i};
  if (int(threadIdx.x) < 3 * G) {
    const int w = threadIdx.x / G, hh = threadIdx.x - w * G;
    const int slot = (Q[w] - Bk.q0[w]) * Bk.nr[w] + (R[w] - Bk.r0[w]);
    const int g = ((hh - T.go[P[w]]) % G + G) % G;
    srb[w][hh] = rowoff[(w * G + g) * Bk.nb * Bk.nb + slot];
    sxb[w][hh] = xoff[(w * Bk.nb + (P[w] - Bk.p0[w])) * G + hh];
  }
  if (int(threadIdx.x) < G) snp[threadIdx.x] = T.npair[threadIdx.x];
  __syncthreads();
  const int gijk = (T.go[tr.i] + T.go[tr.j] + T.go[tr.k]) % G;
  const int ga = ((gijk - h) % G + G) % G;
  const int na = T.vcnt[ga], a0 = T.voff[ga];
  const int n = snp[h];
  const int32_t* pr = T.pairs + T.poff[h];
  const double* ev = eps + o;
  const double eijk = eps[tr.i] + eps[tr.j] + eps[tr.k];
  const int gx[3] = {T.go[tr.i], T.go[tr.j], T.go[tr.k]};
  const int Yx[3] = {tr.j, tr.i, tr.j}, Zx[3] = {tr.k, tr.k, tr.i};

  // Y(alpha; pair column col of irrep hh) = X^(i;jk) - X^(j;ik) - X^(k;ji)  (FP64 sums)
  auto Y = [&](int alpha, int hh, int col) {
    const int64_t al = alpha - T.voff[T.gv[alpha]];
    const int64_t np = snp[hh];
    const cplx x0 = X[sxb[0][hh] + (srb[0][hh] + al) * np + col];
    const cplx x1 = X[sxb[1][hh] + (srb[1][hh] + al) * np + col];
    const cplx x2 = X[sxb[2][hh] + (srb[2][hh] + al) * np + col];
    return make_double2(x0.x - x1.x - x2.x, x0.y - x1.y - x2.y);
  };
  auto Vv = [&](int b, int c, int y, int z) { return V[((int64_t(y) * o + z) * v + b) * v + c]; };

  double sr = 0.0, si = 0.0;
  for (int u = threadIdx.x; u < n; u += blockDim.x) {
    const int b = pr[u] >> 16, c = pr[u] & 0xFFFF;
    const int gb = T.gv[b], gc = T.gv[c];
    const double dbc = eijk - ev[b] - ev[c];
    double pr_re = 0.0, pr_im = 0.0;                          // FP64 path: this pair's sum
    float2 ar = make_float2(0.f, 0.f), ai = make_float2(0.f, 0.f);  // DS path
    const float2 dbc_ds = DS ? ds_split(dbc) : make_float2(0.f, 0.f);
    for (int a = a0; a < a0 + na && a < b; ++a) {
      // c_abc = Y(a; bc) - Y(b; ac) + Y(c; ab)
      const int hac = (ga + gc) % G, hab = (ga + gb) % G;
      const int cac = T.pidx[a * v + c] - 1, cab = T.pidx[a * v + b] - 1;
      const cplx y1 = Y(a, h, u), y2 = Y(b, hac, cac), y3 = Y(c, hab, cab);
      if (DS) {
        const dsc cc = dsc_add(dsc_sub(dsc_of(y1), dsc_of(y2)), dsc_of(y3));
        // d_abc = P(i/jk) P(a/bc) t_i^a <bc||jk>: only t1 of matching irreps is nonzero
        dsc d = dsc{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
        for (int w = 0; w < 3; ++w) {
          const int x = P[w], y = Yx[w], z = Zx[w];
          const bool neg = w > 0;
          if (ga == gx[w]) { const dsc s = dsc_mul(dsc_of(t1[int64_t(x) * v + a]), dsc_of(Vv(b, c, y, z))); d = neg ? dsc_sub(d, s) : dsc_add(d, s); }
          if (gb == gx[w]) { const dsc s = dsc_mul(dsc_of(t1[int64_t(x) * v + b]), dsc_of(Vv(a, c, y, z))); d = neg ? dsc_add(d, s) : dsc_sub(d, s); }
          if (gc == gx[w]) { const dsc s = dsc_mul(dsc_of(t1[int64_t(x) * v + c]), dsc_of(Vv(b, a, y, z))); d = neg ? dsc_add(d, s) : dsc_sub(d, s); }
        }
        const dsc wv = dsc_add(cc, d);
        const float2 rD = ds_rcp(ds_add(dbc_ds, ds_neg(ds_split(ev[a]))));
        // conj(w) c / D
        const float2 pre = ds_add(ds_mul(wv.re, cc.re), ds_mul(wv.im, cc.im));
        const float2 pim = ds_add(ds_mul(wv.re, cc.im), ds_neg(ds_mul(wv.im, cc.re)));
        ar = ds_add(ar, ds_mul(pre, rD));
        ai = ds_add(ai, ds_mul(pim, rD));
      } else {
        const cplx cc = make_double2(y1.x - y2.x + y3.x, y1.y - y2.y + y3.y);
        double dr = 0.0, di = 0.0;
#pragma unroll
        for (int w = 0; w < 3; ++w) {
          const int x = P[w], y = Yx[w], z = Zx[w];
          const double sg = w > 0 ? -1.0 : 1.0;
          if (ga == gx[w]) { const cplx s = cmul(t1[int64_t(x) * v + a], Vv(b, c, y, z)); dr += sg * s.x; di += sg * s.y; }
          if (gb == gx[w]) { const cplx s = cmul(t1[int64_t(x) * v + b], Vv(a, c, y, z)); dr -= sg * s.x; di -= sg * s.y; }
          if (gc == gx[w]) { const cplx s = cmul(t1[int64_t(x) * v + c], Vv(b, a, y, z)); dr -= sg * s.x; di -= sg * s.y; }
        }
        const double rD = 1.0 / (dbc - ev[a]);
        const double wr = cc.x + dr, wi = cc.y + di;
        pr_re += (wr * cc.x + wi * cc.y) * rD;
        pr_im += (wr * cc.y - wi * cc.x) * rD;
      }
    }
    if (DS) {
      sr += ds_to_double(ar.x, ar.y);
      si += ds_to_double(ai.x, ai.y);
    } else {
      sr += pr_re;
      si += pr_im;
    }
  }
  // fixed-order block reduction
  for (int off = 16; off; off >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, off);
    si += __shfl_down_sync(0xffffffffu, si, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][warp] = sr;
    red[1][warp] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      x += red[0][w];
      y += red[1][w];
    }
    e3h[int64_t(tr.idx) * G + h] = make_double2(x, y);
  }
}

// per-triple energy = sum over the pair irreps of its parts, fixed order
__global__ void __launch_bounds__(T3_THREADS) k_t3_fold(const cplx* __restrict__ e3h, int64_t n, int G,
                                                        cplx* __restrict__ e3) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
    double x = 0.0, y = 0.0;
    for (int h = 0; h < G; ++h) {
      x += e3h[t * G + h].x;
      y += e3h[t * G + h].y;
    }
    e3[t] = make_double2(x, y);
  }
}

// E(T) = sum of the per-triple energies, one CTA, fixed order
__global__ void __launch_bounds__(T3_THREADS) k_t3_sum(const cplx* __restrict__ e3, int64_t n, cplx* __restrict__ out) {
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    a += e3[i].x;
    b += e3[i].y;
  }
  __shared__ double red[2][T3_THREADS];
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int s = T3_THREADS / 2; s; s >>= 1) {
    if (int(threadIdx.x) < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = make_double2(red[0][0], red[1][0]);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host driver
namespace {

struct HostTables {
  int o = 0, v = 0, G = 1;
  std::vector<int> go, gv, girr, voff, vcnt, ooff, ocnt, npair, poff;
  std::vector<int32_t> pairs, pidx;
};

HostTables host_tables(const Ctx& c) {
  HostTables H;
  H.o = c.no;
  H.v = c.nv;
  H.G = c.G;
  const Space& SO = c.spaces[SP_OCC];
  const Space& SV = c.spaces[SP_VIRT];
  H.voff = SV.off;
  H.vcnt = SV.cnt;
  H.ooff = SO.off;
  H.ocnt = SO.cnt;
  H.go.resize(H.o);
  H.gv.resize(H.v);
  for (int g = 0; g < H.G; ++g) {
    for (int k = 0; k < SO.cnt[g]; ++k) H.go[SO.off[g] + k] = g;
    for (int k = 0; k < SV.cnt[g]; ++k) H.gv[SV.off[g] + k] = g;
  }
  H.girr = H.go;
  H.girr.insert(H.girr.end(), H.gv.begin(), H.gv.end());
  // pair-packed virtual pairs b < c, grouped by pair irrep, b-major inside a group
  H.npair.assign(H.G, 0);
  H.poff.assign(H.G, 0);
  H.pidx.assign(size_t(H.v) * H.v, 0);
  std::vector<std::vector<int32_t>> by(H.G);
  for (int b = 0; b < H.v; ++b)
    for (int cc = b + 1; cc < H.v; ++cc) {
      const int h = (H.gv[b] + H.gv[cc]) % H.G;
      H.pidx[size_t(b) * H.v + cc] = int32_t(by[h].size()) + 1;
      by[h].push_back((b << 16) | cc);
    }
  for (int h = 0; h < H.G; ++h) {
    H.poff[h] = int(H.pairs.size());
    H.npair[h] = int(by[h].size());
    H.pairs.insert(H.pairs.end(), by[h].begin(), by[h].end());
  }
  return H;
}

// Device copies of the tables (one allocation, freed by the caller)
struct DevTables {
  T3Tables T;
  void* mem = nullptr;
};

DevTables upload_tables(Ctx& c, const HostTables& H) {
  std::vector<int32_t> buf;
  auto put = [&](const std::vector<int>& x) {
    const size_t at = buf.size();
    buf.insert(buf.end(), x.begin(), x.end());
    return at;
  };
  const size_t a_go = put(H.go), a_gv = put(H.gv), a_girr = put(H.girr), a_voff = put(H.voff), a_vcnt = put(H.vcnt),
               a_ooff = put(H.ooff), a_ocnt = put(H.ocnt), a_npair = put(H.npair), a_poff = put(H.poff);
  const size_t a_pairs = buf.size();
  buf.insert(buf.end(), H.pairs.begin(), H.pairs.end());
  const size_t a_pidx = buf.size();
  buf.insert(buf.end(), H.pidx.begin(), H.pidx.end());
  DevTables D;
  D.mem = c.dalloc(sizeof(int32_t) * std::max<size_t>(buf.size(), 1));
  upload(c, D.mem, buf.data(), sizeof(int32_t) * buf.size());
  const int32_t* p = (const int32_t*)D.mem;
  D.T.G = H.G;
  D.T.go = p + a_go;
  D.T.gv = p + a_gv;
  D.T.girr = p + a_girr;
  D.T.voff = p + a_voff;
  D.T.vcnt = p + a_vcnt;
  D.T.ooff = p + a_ooff;
  D.T.ocnt = p + a_ocnt;
  D.T.npair = p + a_npair;
  D.T.poff = p + a_poff;
  D.T.pairs = p + a_pairs;
  D.T.pidx = p + a_pidx;
  return D;
}

int64_t choose3(int64_t n) { return n < 3 ? 0 : n * (n - 1) * (n - 2) / 6; }
int64_t choose2(int64_t n) { return n < 2 ? 0 : n * (n - 1) / 2; }

// One block triple's plan: the A members (ordering w, irrep g), the products and
// where each X block and each pair's rows sit.
struct BlockPlan {
  T3Block bk{};
  int ns[3] = {0, 0, 0};                  // |P_w|, used for the per-p tables
  std::vector<EmuSetMat> amats;           // [3 G] A members (src, rows, K)
  std::vector<T3AUnit> aunits;            // gather units
  std::vector<int32_t> rowoff;            // [3 G nb^2]
  std::vector<int64_t> xoff;              // [3 nb G]
  std::vector<EmuSetProd> prods;          // products (A member, B member, X offset)
  std::vector<GemmProb> fprods;           // the same products for the FP64 kernel
  std::vector<std::pair<int64_t, int64_t>> zeros;  // X regions of K = 0 products (offset, count)
  std::vector<T3Tri> tris;
  int64_t a_elems = 0, x_elems = 0;
  double macs_run = 0.0, macs_need = 0.0;
};

// Blocks: [b nb, min((b + 1) nb, o)).  Pairs (q, r) of ordering w are kept when some p
// of P_w completes them to a triple i<j<k: w = 0 (p = i; q = j, r = k), 1 (p = j; q = i,
// r = k), 2 (p = k; q = j, r = i).
void plan_block(const HostTables& H, int nb, int I, int J, int K, const std::vector<int64_t>& boff,
                BlockPlan& bp, bool build) {
  const int o = H.o, G = H.G;
  auto lo = [&](int b) { return b * nb; };
  auto hi = [&](int b) { return std::min((b + 1) * nb, o); };
  const int PB[3] = {I, J, K}, QB[3] = {J, I, J}, RB[3] = {K, K, I};
  bp.bk.nb = nb;
  for (int w = 0; w < 3; ++w) {
    bp.bk.p0[w] = lo(PB[w]);
    bp.bk.q0[w] = lo(QB[w]);
    bp.bk.r0[w] = lo(RB[w]);
    bp.bk.nr[w] = hi(RB[w]) - lo(RB[w]);
    bp.ns[w] = hi(PB[w]) - lo(PB[w]);
  }
  const int nb2 = nb * nb;
  bp.amats.assign(3 * G, EmuSetMat{0, 0, 0});
  if (build) {
    bp.rowoff.assign(size_t(3) * G * nb2, 0);
    bp.xoff.assign(size_t(3) * nb * G, -1);
    bp.aunits.clear();
    bp.prods.clear();
    bp.fprods.clear();
    bp.zeros.clear();
    bp.tris.clear();
  }
  bp.a_elems = bp.x_elems = 0;
  bp.macs_run = bp.macs_need = 0.0;
  // does some p of P_w make (q, r) part of a triple i<j<k?
  auto pair_used = [&](int w, int q, int r) {
    const int p0 = lo(PB[w]), p1 = hi(PB[w]);
    if (w == 0) return q < r && p0 < q;               // i < j < k: p < q < r
    if (w == 1) return std::max(p0, q + 1) <= std::min(p1 - 1, r - 1);  // q < p < r
    return r < q && p1 - 1 > q;                        // r < q < p
  };
  for (int w = 0; w < 3; ++w)
    for (int g = 0; g < G; ++g) {
      const int Kg = H.vcnt[g] + H.ocnt[g];
      int64_t rows = 0;
      for (int q = lo(QB[w]); q < hi(QB[w]); ++q)
        for (int r = lo(RB[w]); r < hi(RB[w]); ++r) {
          const int slot = (q - lo(QB[w])) * bp.bk.nr[w] + (r - lo(RB[w]));
          if (!pair_used(w, q, r)) continue;
          const int ga = ((H.go[q] + H.go[r] - g) % G + G) % G;
          const int na = H.vcnt[ga];
          if (build) {
            bp.rowoff[(size_t(w) * G + g) * nb2 + slot] = int32_t(rows);
            if (na && Kg) bp.aunits.push_back(T3AUnit{bp.a_elems + rows * Kg, q, r, H.voff[ga], na, g, Kg});
          }
          rows += na;
        }
      bp.amats[w * G + g] = EmuSetMat{bp.a_elems, int(rows), Kg};
      bp.a_elems += rows * Kg;
    }
  // products: X^(p;.)[h] = A_(w, h - G(p)) B_(p, h)
  for (int w = 0; w < 3; ++w)
    for (int p = lo(PB[w]); p < hi(PB[w]); ++p)
      for (int h = 0; h < G; ++h) {
        const int g = ((h - H.go[p]) % G + G) % G;
        const EmuSetMat& am = bp.amats[w * G + g];
        const int64_t n = H.npair[h];
        if (am.rows == 0 || n == 0) continue;
        if (build) bp.xoff[(size_t(w) * nb + (p - lo(PB[w]))) * G + h] = bp.x_elems;
        if (build && am.K == 0) {
          bp.zeros.push_back({bp.x_elems, int64_t(am.rows) * n});
        } else if (build) {
          bp.prods.push_back(EmuSetProd{w * G + g, p * G + h, bp.x_elems});
          GemmProb f{};
          f.a = am.src;
          f.b = boff[size_t(p) * G + h];
          f.c = bp.x_elems;
          f.M = am.rows;
          f.N = int32_t(n);
          f.K = am.K;
          bp.fprods.push_back(f);
        }
        bp.macs_run += double(am.rows) * double(n) * double(am.K);
        bp.x_elems += int64_t(am.rows) * n;
      }
  // triples i<j<k of the block triple, and the products they need
  for (int i = lo(I); i < hi(I); ++i)
    for (int j = std::max(lo(J), i + 1); j < hi(J); ++j)
      for (int k = std::max(lo(K), j + 1); k < hi(K); ++k) {
        const int gijk = (H.go[i] + H.go[j] + H.go[k]) % G;
        const int Pn[3] = {i, j, k};
        for (int w = 0; w < 3; ++w)
          for (int h = 0; h < G; ++h) {
            const int ga = ((gijk - h) % G + G) % G;
            const int g = ((h - H.go[Pn[w]]) % G + G) % G;
            bp.macs_need += double(H.vcnt[ga]) * double(H.npair[h]) * double(H.vcnt[g] + H.ocnt[g]);
          }
        if (build) bp.tris.push_back(T3Tri{i, j, k, int(choose3(k) + choose2(j) + i)});
      }
}

// RAII guard: the FP64 grouped kernel launches one grid row per context instance;
// (T) runs one instance's operands at a time
struct OneInstance {
  Ctx& c;
  int saved;
  explicit OneInstance(Ctx& cc) : c(cc), saved(cc.ninst) { c.ninst = 1; }
  ~OneInstance() { c.ninst = saved; }
};

}  // namespace

// E(T) of instance `inst` from its current amplitudes, in occupied blocks of `block`
// spinors (0: the largest within the scratch budget); per_triple (host, nullable)
// receives the energy of every i<j<k at its combinatorial index C(k,3) + C(j,2) + i.
void ccsd_t(Ctx& c, int inst, int block, exp_t3_info* info, double* per_triple) {
  if (c.nact) throw ExpError{EXP_ESTATE, "(T): the context has an active space (create one without)"};
  if (!c.have_integrals) throw ExpError{EXP_ESTATE, "exp_init_integrals must come first"};
  if (!c.guessed) throw ExpError{EXP_ESTATE, "(T): no amplitudes yet (iterate or set them first)"};
  if (inst < 0 || inst >= c.ninst) throw ExpError{EXP_EINVAL, "instance out of range"};
  if (c.nv > 65535) throw ExpError{EXP_EINVAL, "(T): more than 65535 virtual spinors"};
  if (block < 0) throw ExpError{EXP_EINVAL, "(T): negative block size"};
  const HostTables H = host_tables(c);
  const int o = H.o, v = H.v, G = H.G;
  const int64_t ntri = choose3(o);
  if (ntri > INT32_MAX) throw ExpError{EXP_EINVAL, "(T): too many occupied triples"};
  const bool emulated = c.cfg.precision == EXP_EMU_BF16;

  // device scratch, released on every exit path
  struct Scratch {
    Ctx& c;
    std::vector<void*> bufs;
    EmuSet* A = nullptr;
    EmuSet* B = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    explicit Scratch(Ctx& cc) : c(cc) {}
    void* get(size_t bytes) {
      void* p = c.dalloc(std::max<size_t>(bytes, 16));
      bufs.push_back(p);
      return p;
    }
    ~Scratch() {
      cudaStreamSynchronize(c.stream);
      if (A) emu_set_free(c, A);
      if (B) emu_set_free(c, B);
      for (void* p : bufs) c.dfree(p);
      for (auto e : ev)
        if (e) cudaEventDestroy(e);
    }
  } sc(c);
  CK(cudaEventCreate(&sc.ev[0]));
  CK(cudaEventCreate(&sc.ev[1]));
  CK(cudaEventRecord(sc.ev[0], c.stream));

  uint64_t seed = 0;
  CK(cudaMemcpyAsync(&seed, c.d_seed + inst, sizeof(seed), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  const double scale = c.h_scale[inst];
  const int real = c.cfg.real_arith;
  const double* eps = c.d_eps + size_t(inst) * (o + v);
  const DevTables DT = upload_tables(c, H);
  sc.bufs.push_back(DT.mem);

  // dense amplitudes and integral blocks
  cplx* t1d = (cplx*)sc.get(sizeof(cplx) * size_t(o) * v);
  cplx* t2d = (cplx*)sc.get(sizeof(cplx) * size_t(o) * o * v * v);
  ccsd_dense_io(c, inst, t1d, t2d, true);
  auto dense4 = [&](cplx* dst, T3Dense4 D) {
    const int64_t n = int64_t(D.n[0]) * D.n[1] * D.n[2] * D.n[3];
    if (!n) return;
    const int blocks = int(std::min<int64_t>((n + T3_THREADS - 1) / T3_THREADS, int64_t(std::max(c.sm_count, 1)) * 32));
    k_t3_dense4<<<blocks, T3_THREADS, 0, c.stream>>>(dst, D, n, c.n_gen, seed, scale, real, DT.T.girr, G);
    KCHECK(c);
  };
  cplx* Vd = (cplx*)sc.get(sizeof(cplx) * size_t(o) * o * v * v);  // Vd[j][k][b][c] = <bc||jk>
  dense4(Vd, T3Dense4{{o, o, v, v}, {0, 0, o, o}, {2, 3, 0, 1}});
  cplx* Wd = (cplx*)sc.get(sizeof(cplx) * size_t(o) * o * v * o);  // Wd[q][r][a][m] = <ma||qr>
  dense4(Wd, T3Dense4{{o, o, v, o}, {0, 0, o, 0}, {3, 2, 0, 1}});

  // B members B_{p,h} (K = v_G + o_G rows x npair[h] columns, G = h - G(p))
  std::vector<int64_t> boff(size_t(o) * G);
  std::vector<EmuSetMat> bmats(size_t(o) * G);
  std::vector<T3BRow> brows;
  int64_t bsz = 0;
  for (int p = 0; p < o; ++p)
    for (int h = 0; h < G; ++h) {
      const int g = ((h - H.go[p]) % G + G) % G;
      const int K = H.vcnt[g] + H.ocnt[g], N = H.npair[h];
      boff[size_t(p) * G + h] = bsz;
      bmats[size_t(p) * G + h] = EmuSetMat{bsz, N, K};
      if (N)
        for (int k = 0; k < K; ++k) {
          const bool vr = k < H.vcnt[g];
          brows.push_back(T3BRow{bsz + int64_t(k) * N, p, h, vr ? 0 : 1, vr ? H.voff[g] + k : H.ooff[g] + k - H.vcnt[g]});
        }
      bsz += int64_t(K) * N;
    }
  cplx* Bbuf = (cplx*)sc.get(sizeof(cplx) * size_t(std::max<int64_t>(bsz, 1)));
  if (!brows.empty()) {
    T3BRow* d_rows = (T3BRow*)sc.get(sizeof(T3BRow) * brows.size());
    upload(c, d_rows, brows.data(), sizeof(T3BRow) * brows.size());
    k_t3_brows<<<unsigned(brows.size()), T3_THREADS, 0, c.stream>>>(Bbuf, d_rows, DT.T, t2d, o, v, c.n_gen, seed, scale,
                                                                     real);
    KCHECK(c);
  }
  if (emulated) {
    sc.B = emu_set_new(c, c.cfg.n_slices, true);
    sc.A = emu_set_new(c, c.cfg.n_slices, false);
    emu_set_slice(c, sc.B, bmats, Bbuf);
  }

  // block size: the largest whose A and X buffers fit the budget
  const int64_t budget = int64_t(1) << 30;  // complex elements (16 GiB)
  const int nbmax = std::max(1, std::min(o, block > 0 ? block : 64));
  int nb = 1;
  int64_t max_a = 0, max_x = 0;
  for (int cand = nbmax; cand >= 1; --cand) {
    const int nblk = (o + cand - 1) / cand;
    int64_t ma = 0, mx = 0;
    BlockPlan probe;
    for (int I = 0; I < nblk; ++I)
      for (int J = I; J < nblk; ++J)
        for (int K = J; K < nblk; ++K) {
          plan_block(H, cand, I, J, K, boff, probe, false);
          ma = std::max(ma, probe.a_elems);
          mx = std::max(mx, probe.x_elems);
        }
    nb = cand;
    max_a = ma;
    max_x = mx;
    if (block > 0 || ma + mx <= budget) break;  // a requested block size is taken as given
  }
  const int nblk = o ? (o + nb - 1) / nb : 0;
  cplx* Abuf = (cplx*)sc.get(sizeof(cplx) * size_t(std::max<int64_t>(max_a, 1)));
  cplx* X = (cplx*)sc.get(sizeof(cplx) * size_t(std::max<int64_t>(max_x, 1)));
  cplx* e3 = (cplx*)sc.get(sizeof(cplx) * size_t(std::max<int64_t>(ntri, 1)));
  cplx* e3h = (cplx*)sc.get(sizeof(cplx) * size_t(std::max<int64_t>(ntri, 1)) * G);  // per (triple, pair irrep)
  CK(cudaMemsetAsync(e3h, 0, sizeof(cplx) * size_t(std::max<int64_t>(ntri, 1)) * G, c.stream));
  const size_t nb2 = size_t(nb) * nb;
  int32_t* d_rowoff = (int32_t*)sc.get(sizeof(int32_t) * 3 * G * nb2);
  int64_t* d_xoff = (int64_t*)sc.get(sizeof(int64_t) * 3 * size_t(nb) * G);
  T3Tri* d_tris = (T3Tri*)sc.get(sizeof(T3Tri) * nb2 * nb);
  T3AUnit* d_units = (T3AUnit*)sc.get(sizeof(T3AUnit) * 3 * G * nb2);
  GemmProb* d_fp = (GemmProb*)sc.get(sizeof(GemmProb) * 3 * size_t(nb) * G);

  double macs_need = 0.0, macs_run = 0.0, x_total = 0.0;
  int n_bt = 0;
  BlockPlan bp;
  // per block triple: events around its product launch and its energy launch
  std::vector<cudaEvent_t> evs;
  struct EvGuard {
    std::vector<cudaEvent_t>& e;
    ~EvGuard() {
      for (auto x : e) cudaEventDestroy(x);
    }
  } evg{evs};
  auto mark = [&]() {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    evs.push_back(e);
    CK(cudaEventRecord(e, c.stream));
  };
  for (int I = 0; I < nblk; ++I)
    for (int J = I; J < nblk; ++J)
      for (int K = J; K < nblk; ++K) {
        plan_block(H, nb, I, J, K, boff, bp, true);
        if (bp.tris.empty()) continue;
        ++n_bt;
        x_total += double(bp.x_elems);
        macs_need += bp.macs_need;
        macs_run += bp.macs_run;
        // A members
        if (!bp.aunits.empty()) {
          upload(c, d_units, bp.aunits.data(), sizeof(T3AUnit) * bp.aunits.size());
          k_t3_arows<<<unsigned(bp.aunits.size()), T3_THREADS, 0, c.stream>>>(Abuf, d_units, DT.T, t2d, Wd, o, v);
          KCHECK(c);
        }
        for (auto& z : bp.zeros) CK(cudaMemsetAsync(X + z.first, 0, sizeof(cplx) * size_t(z.second), c.stream));
        // X = A B for every product of the three orderings
        if (emulated) emu_set_slice(c, sc.A, bp.amats, Abuf);
        mark();
        if (emulated) {
          emu_set_multiply(c, sc.A, sc.B, bp.prods, X, make_double2(1.0, 0.0));
        } else if (!bp.fprods.empty()) {
          GemmPlan g;
          g.tm = g.tn = 64;
          int tile0 = 0;
          for (GemmProb& f : bp.fprods) {
            f.tiles_m = (f.M + g.tm - 1) / g.tm;
            f.tiles_n = (f.N + g.tn - 1) / g.tn;
            f.ksplit = 1;
            f.kchunk = (f.K + 7) / 8 * 8;
            f.tile0 = tile0;
            tile0 += f.tiles_m * f.tiles_n;
          }
          g.n_tiles = tile0;
          g.n_probs = int(bp.fprods.size());
          upload(c, d_fp, bp.fprods.data(), sizeof(GemmProb) * bp.fprods.size());
          g.d_probs = d_fp;
          OneInstance one(c);
          launch_gemm_fp64(c, g, Abuf, Bbuf, X, 0, 0, 0, make_double2(1.0, 0.0), false);
        }
        mark();
        // energies of the block triple's i<j<k
        upload(c, d_rowoff, bp.rowoff.data(), sizeof(int32_t) * bp.rowoff.size());
        upload(c, d_xoff, bp.xoff.data(), sizeof(int64_t) * bp.xoff.size());
        upload(c, d_tris, bp.tris.data(), sizeof(T3Tri) * bp.tris.size());
        mark();
        const dim3 eg(unsigned(bp.tris.size()), unsigned(G));
        if (emulated)
          k_t3_energy<true><<<eg, T3_THREADS, 0, c.stream>>>(d_tris, bp.bk, DT.T, X, d_xoff, d_rowoff, t1d, Vd, eps, o, v,
                                                             e3h);
        else
          k_t3_energy<false><<<eg, T3_THREADS, 0, c.stream>>>(d_tris, bp.bk, DT.T, X, d_xoff, d_rowoff, t1d, Vd, eps, o,
                                                              v, e3h);
        KCHECK(c);
        mark();
      }
  cplx* d_E = (cplx*)sc.get(sizeof(cplx));
  if (ntri) {
    k_t3_fold<<<unsigned(std::min<int64_t>((ntri + T3_THREADS - 1) / T3_THREADS, 4096)), T3_THREADS, 0, c.stream>>>(
        e3h, ntri, G, e3);
    KCHECK(c);
  }
  k_t3_sum<<<1, T3_THREADS, 0, c.stream>>>(e3, ntri, d_E);
  KCHECK(c);
  CK(cudaEventRecord(sc.ev[1], c.stream));
  cplx E;
  CK(cudaMemcpyAsync(&E, d_E, sizeof(cplx), cudaMemcpyDeviceToHost, c.stream));
  if (per_triple && ntri)
    CK(cudaMemcpyAsync(per_triple, e3, sizeof(cplx) * size_t(ntri), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  if (c.d_emu_err) {
    int err = 0;
    CK(cudaMemcpy(&err, c.d_emu_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) throw ExpError{EXP_ETIMEOUT, "emulated GEMM: a bounded device wait gave up"};
  }
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, sc.ev[0], sc.ev[1]));
  double ms_prod = 0.0, ms_en = 0.0;
  for (size_t k = 0; k + 3 < evs.size(); k += 4) {
    float a = 0.f, b = 0.f;
    CK(cudaEventElapsedTime(&a, evs[k], evs[k + 1]));
    CK(cudaEventElapsedTime(&b, evs[k + 2], evs[k + 3]));
    ms_prod += a;
    ms_en += b;
  }
  if (c.profile)
    fprintf(stderr,
            "[exp_t3] o=%d v=%d G=%d nb=%d block triples %d: %.3f ms (products %.3f, energies %.3f), %.3e needed / "
            "%.3e run complex MACs\n",
            o, v, G, nb, n_bt, ms, ms_prod, ms_en, macs_need, macs_run);
  if (info) {
    info->e_re = E.x;
    info->e_im = E.y;
    info->ms = ms;
    info->ms_products = ms_prod;
    info->ms_energy = ms_en;
    info->macs = macs_need;
    info->macs_run = macs_run;
    info->x_elems = x_total;
    info->n_triples = ntri;
    info->n_block_triples = n_bt;
    info->block = nb;
  }
}
