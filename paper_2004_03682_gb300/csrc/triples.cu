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
// (h = G(b) + G(c)), and a carries G(i) + G(j) + G(k) - h for all three terms.  So for
// one triple and one pair irrep h, Y is a single matrix product over the K of the
// three terms concatenated (K_w = v_G + o_G of each), computed transposed:
//
//   Y_ijk^T[bc, a] = sum_w  Bt_{p_w,h}[bc, k] s_w A_{q_w r_w}^T[k, a],
//
// (p, q, r, s)_w = (i, j, k, +), (j, i, k, -), (k, j, i, -), with Bt_{p,h} = B_{p,h}^T
// the same for the whole evaluation and the three A^T segments gathered per triple.
// Y is antisymmetric in (b, c), so it keeps the pair-packed rows b < c only.
//
// Operands.  The integrals are the context's own: <bc||jk> copied out of its driver
// integral, <ma||qr> and <bc||ep> gathered from layouts it caches (derived by a permute
// from a held layout of the same symmetry family, else drawn once); t1 and t2 from its
// amplitudes.
//
// Schedule.  The members Bt_{p,h} are written and, in the emulated precision, sliced
// once, all members of one h sharing one exponent per row bc.  The occupied spinors
// (irrep-sorted) are cut into blocks of nb, and the triples i<j<k of each block triple
// I <= J <= K form one batch: its A^T segments are gathered (and sliced, the three
// of one (triple, h) sharing one exponent per column a), one grouped launch forms Y
// for every (triple, h) of the batch -- each product accumulating its three segments
// exactly, on the tensor cores -- then one CTA per triple and pair irrep of (b, c)
// forms c from three Y elements (the P(a/bc) terms), d, D and its energy.  Fixed-order sums over the
// pair irreps, then over the triples, give the per-triple energies and E(T): the
// result does not depend on the batching.  The element arithmetic runs in FP64 under
// EXP_FP64 (where the three segments are three FP64 product launches into Y) and in
// double-single FP32 (about 48 bits, each pair's sum added in FP64) under the emulated
// precision, where the FP64 pipe would bound it.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "ccsd.h"
#include "emu.h"
#include "fpbits.h"

namespace {

constexpr int T3_THREADS = 256;

// ---------------------------------------------------------------------------
// Index tables of one context (irrep-sorted local indices; global spinor index =
// occupied local index, or o + virtual local index).
struct T3Tables {
  int G = 1;
  const int* go = nullptr;     // [o] irrep of each occupied spinor
  const int* gv = nullptr;     // [v] irrep of each virtual spinor
  const int* voff = nullptr;   // [G] first virtual of each irrep
  const int* vcnt = nullptr;   // [G]
  const int* ooff = nullptr;   // [G]
  const int* ocnt = nullptr;   // [G]
  const int* npair = nullptr;  // [G] virtual pairs b < c per pair irrep
  const int* poff = nullptr;   // [G] their first entry in pairs
  const int32_t* pairs = nullptr;  // (b << 16 | c), b < c, grouped by pair irrep
  const int32_t* pidx = nullptr;   // [v * v] column of pair (b, c) in its irrep block + 1 (b < c), 0 otherwise
};

// The amplitude columns of a member Bt_{p,h} = B_{p,h}^T (npair[h] rows x K columns,
// K = v_G + o_G): column k >= v_G is t_pm^bc (m = ooff[G] + k - v_G); the integral
// columns k < v_G (<bc||ep>) come from the context's integrals (k_t3_gather_bt).
struct T3BRow {
  int64_t dst;  // element offset of the member in the Bt buffer
  int p, h;
  int m;        // the occupied index of this column
  int k, K;     // this column and the member's column count
};

__global__ void __launch_bounds__(T3_THREADS) k_t3_brows(cplx* __restrict__ B, const T3BRow* __restrict__ rows,
                                                         T3Tables T, const cplx* __restrict__ t2, int o, int v) {
  const T3BRow R = rows[blockIdx.x];
  const int n = T.npair[R.h];
  const int32_t* pr = T.pairs + T.poff[R.h];
  cplx* dst = B + R.dst + R.k;
  for (int u = threadIdx.x; u < n; u += blockDim.x) {
    const int b = pr[u] >> 16, c = pr[u] & 0xFFFF;
    dst[int64_t(u) * R.K] = t2[((int64_t(R.p) * o + R.m) * v + b) * v + c];
  }
}

// Gathers from an integral tensor of the context (its layout's sub-blocks as
// generator tasks, 4096 elements per chunk; slot k of an element has global spinor index
// g0[k] + i[k], virtual ones from o on).  Dense: dst[sum_k x_k ds[k]] with x_k the slot's
// local index.  Members: slots (b, c, e, p) of <bc||ep> into Bt_{p,h}[pair (b, c)][e].
__device__ __forceinline__ void t3_task_index(const GenTask& Tk, int64_t e, int i[4]) {
  int64_t r = e;
  i[3] = int(r % Tk.n[3]);
  r /= Tk.n[3];
  i[2] = int(r % Tk.n[2]);
  r /= Tk.n[2];
  i[1] = int(r % Tk.n[1]);
  i[0] = int(r / Tk.n[1]);
}

struct T3Dense {
  int64_t ds[4];  // destination stride of each slot's local index
  int virt[4];    // slot holds a virtual spinor (local index = global - o)
};

__global__ void __launch_bounds__(T3_THREADS) k_t3_gather_dense(cplx* __restrict__ dst, const cplx* __restrict__ src,
                                                                const GenTask* __restrict__ tasks,
                                                                const ChunkRef* __restrict__ chunks, T3Dense D, int o) {
  const ChunkRef ch = chunks[blockIdx.x];
  const GenTask Tk = tasks[ch.task];
  const int64_t end = min(ch.start + (int64_t)4096, Tk.count);
  for (int64_t e = ch.start + threadIdx.x; e < end; e += blockDim.x) {
    int i[4];
    t3_task_index(Tk, e, i);
    int64_t d = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) d += int64_t(Tk.g0[k] + i[k] - (D.virt[k] ? o : 0)) * D.ds[k];
    dst[d] = src[Tk.base + i[0] * Tk.st[0] + i[1] * Tk.st[1] + i[2] * Tk.st[2] + i[3] * Tk.st[3]];
  }
}

__global__ void __launch_bounds__(T3_THREADS) k_t3_gather_bt(cplx* __restrict__ Bt, const cplx* __restrict__ src,
                                                             const GenTask* __restrict__ tasks,
                                                             const ChunkRef* __restrict__ chunks, T3Tables T,
                                                             const int64_t* __restrict__ boff, int o, int v) {
  const ChunkRef ch = chunks[blockIdx.x];
  const GenTask Tk = tasks[ch.task];
  const int64_t end = min(ch.start + (int64_t)4096, Tk.count);
  const int G = T.G;
  for (int64_t e = ch.start + threadIdx.x; e < end; e += blockDim.x) {
    int i[4];
    t3_task_index(Tk, e, i);
    const int b = Tk.g0[0] + i[0] - o, c = Tk.g0[1] + i[1] - o;
    if (b >= c) continue;  // the members keep b < c
    const int ee = Tk.g0[2] + i[2] - o, p = Tk.g0[3] + i[3];
    const int h = (T.gv[b] + T.gv[c]) % G, g = T.gv[ee];
    const int K = T.vcnt[g] + T.ocnt[g];
    const int64_t u = T.pidx[int64_t(b) * v + c] - 1;
    Bt[boff[int64_t(p) * G + h] + u * K + (ee - T.voff[g])] =
        src[Tk.base + i[0] * Tk.st[0] + i[1] * Tk.st[1] + i[2] * Tk.st[2] + i[3] * Tk.st[3]];
  }
}

// One segment of a (triple, h) product: s A_qr^T (K x na, row-major) with
// A_qr[a, k] = [ t_qr^ae | -<ma||qr> ] of irrep G, read from the dense t2[q][r][a][e]
// and W[q][r][a][m] = <ma||qr>.
struct T3Seg {
  int64_t dst;  // element offset of the segment in the segment buffer
  int q, r;
  int a0, na;   // first virtual and count of the irrep of a
  int g, K;     // G and v_G + o_G
  int neg;      // s = -1
};

__global__ void __launch_bounds__(T3_THREADS) k_t3_segs(cplx* __restrict__ Sg, const T3Seg* __restrict__ segs,
                                                        T3Tables T, const cplx* __restrict__ t2,
                                                        const cplx* __restrict__ W, int o, int v) {
  const T3Seg U = segs[blockIdx.x];
  const int ve = T.vcnt[U.g], e0 = T.voff[U.g], m0 = T.ooff[U.g];
  const int64_t qr = int64_t(U.q) * o + U.r;
  const int64_t n = int64_t(U.na) * U.K;
  for (int64_t x = threadIdx.x; x < n; x += blockDim.x) {
    const int k = int(x / U.na), al = int(x - int64_t(k) * U.na);
    const int a = U.a0 + al;
    cplx y;
    if (k < ve) {
      y = t2[(qr * v + a) * v + e0 + k];
    } else {
      const cplx w = W[(qr * v + a) * o + m0 + (k - ve)];
      y = make_double2(-w.x, -w.y);
    }
    Sg[U.dst + x] = U.neg ? make_double2(-y.x, -y.y) : y;
  }
}

struct T3Tri {
  int i, j, k;
  int idx;  // position of the triple in the per-triple output (combinatorial number of i<j<k)
};

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
// Thread = pair (b, c) of h, looping over a < b.  The triple's Y^T blocks per pair
// irrep (offset, columns) are read once per CTA.  DS: the element arithmetic in
// double-single (the emulated precision), each pair's sum added in FP64; otherwise
// FP64 throughout.  Output: e3h[idx G + h].
template <bool DS>
__global__ void __launch_bounds__(T3_THREADS, 3) k_t3_energy(const T3Tri* __restrict__ tris, T3Tables T,
                                                          const cplx* __restrict__ Yt, const int64_t* __restrict__ yoff,
                                                          const cplx* __restrict__ t1, const cplx* __restrict__ V,
                                                          const double* __restrict__ eps, int o, int v,
                                                          cplx* __restrict__ e3h) {
  const T3Tri tr = tris[blockIdx.x];
  const int h = blockIdx.y;
  const int G = T.G;
  __shared__ int64_t syo[EXP_MAX_G];  // Y^T block of pair irrep hh: element offset (rows bc, columns a)
  __shared__ int32_t sna[EXP_MAX_G];  // its columns
  __shared__ double red[2][T3_THREADS / 32];
  const int P[3] = {tr.i, tr.j, tr.k};
  const int gijk = (T.go[tr.i] + T.go[tr.j] + T.go[tr.k]) % G;
  if (int(threadIdx.x) < G) {
    const int hh = threadIdx.x;
    syo[hh] = yoff[int64_t(blockIdx.x) * G + hh];
    sna[hh] = T.vcnt[((gijk - hh) % G + G) % G];
  }
  __syncthreads();
  const int ga = ((gijk - h) % G + G) % G;
  const int na = T.vcnt[ga], a0 = T.voff[ga];
  const int n = T.npair[h];
  const int32_t* pr = T.pairs + T.poff[h];
  const double* ev = eps + o;
  const double eijk = eps[tr.i] + eps[tr.j] + eps[tr.k];
  const int gx[3] = {T.go[tr.i], T.go[tr.j], T.go[tr.k]};
  const int Yx[3] = {tr.j, tr.i, tr.j}, Zx[3] = {tr.k, tr.k, tr.i};

  // Y(alpha; pair column col of irrep hh) = X^(i;jk) - X^(j;ik) - X^(k;ji), one product
  auto Y = [&](int alpha, int hh, int col) {
    const int64_t al = alpha - T.voff[T.gv[alpha]];
    return Yt[syo[hh] + int64_t(col) * sna[hh] + al];
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
  std::vector<int> go, gv, voff, vcnt, ooff, ocnt, npair, poff;
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
  const size_t a_go = put(H.go), a_gv = put(H.gv), a_voff = put(H.voff), a_vcnt = put(H.vcnt),
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

// One batch (the triples i<j<k of a block triple): the A^T segments, the products
// and where each (triple, h) block of Y^T sits.
struct BlockPlan {
  std::vector<T3Tri> tris;
  std::vector<T3Seg> segs;                // gather units, one per segment with K > 0
  std::vector<EmuSetMat> smats;           // the segments as B-set members (K x na), one exponent group per (triple, h)
  std::vector<EmuSetProd> prods;          // per (triple, h): its segments with their Bt members
  std::vector<GemmProb> fprods[3];        // FP64: the w-th segment of every product
  std::vector<int64_t> yoff;              // [tris G] Y^T block of (triple, h)
  std::vector<std::pair<int64_t, int64_t>> zeros;  // Y^T blocks of products with no K (offset, count)
  int64_t y_elems = 0, s_elems = 0;
  double macs_run = 0.0, macs_need = 0.0;
};

// Blocks: [b nb, min((b + 1) nb, o)).  The batch of block triple I <= J <= K is its
// triples i<j<k with i in I, j in J, k in K.
void plan_block(const HostTables& H, int nb, int I, int J, int K, const std::vector<int64_t>& boff,
                BlockPlan& bp, bool build) {
  const int o = H.o, G = H.G;
  auto lo = [&](int b) { return b * nb; };
  auto hi = [&](int b) { return std::min((b + 1) * nb, o); };
  if (build) {
    bp.tris.clear();
    bp.segs.clear();
    bp.smats.clear();
    bp.prods.clear();
    for (auto& f : bp.fprods) f.clear();
    bp.yoff.clear();
    bp.zeros.clear();
  }
  bp.y_elems = bp.s_elems = 0;
  bp.macs_run = bp.macs_need = 0.0;
  // products grouped by pair irrep: one h's members Bt_{p,h} (all p) then stay in L2
  // while its products run
  std::vector<std::vector<EmuSetProd>> by_h(build ? G : 0);
  int tl = 0;
  for (int i = lo(I); i < hi(I); ++i)
    for (int j = std::max(lo(J), i + 1); j < hi(J); ++j)
      for (int k = std::max(lo(K), j + 1); k < hi(K); ++k, ++tl) {
        if (build) bp.tris.push_back(T3Tri{i, j, k, int(choose3(k) + choose2(j) + i)});
        const int gijk = (H.go[i] + H.go[j] + H.go[k]) % G;
        const int Pw[3] = {i, j, k}, Qw[3] = {j, i, j}, Rw[3] = {k, k, i};
        for (int h = 0; h < G; ++h) {
          const int ga = ((gijk - h) % G + G) % G;
          const int na = H.vcnt[ga];
          const int64_t n = H.npair[h];
          if (build) bp.yoff.push_back(bp.y_elems);
          if (na == 0 || n == 0) continue;
          EmuSetProd pd{-1, -1, bp.y_elems};
          int* sa[3] = {&pd.a, &pd.a1, &pd.a2};
          int* sb[3] = {&pd.b, &pd.b1, &pd.b2};
          int ns = 0, ksum = 0;
          for (int w = 0; w < 3; ++w) {
            const int g = ((h - H.go[Pw[w]]) % G + G) % G;
            const int Kw = H.vcnt[g] + H.ocnt[g];
            bp.macs_need += double(na) * double(n) * double(Kw);
            if (Kw == 0) continue;
            if (build) {
              bp.segs.push_back(T3Seg{bp.s_elems, Qw[w], Rw[w], H.voff[ga], na, g, Kw, w > 0 ? 1 : 0});
              *sa[ns] = Pw[w] * G + h;
              *sb[ns] = int(bp.smats.size());
              bp.smats.push_back(EmuSetMat{bp.s_elems, na, Kw, tl * G + h});
              GemmProb f{};
              f.a = boff[size_t(Pw[w]) * G + h];
              f.b = bp.s_elems;
              f.c = bp.y_elems;
              f.M = int32_t(n);
              f.N = na;
              f.K = Kw;
              bp.fprods[ns].push_back(f);
            }
            ++ns;
            ksum += Kw;
            bp.s_elems += int64_t(Kw) * na;
          }
          if (build) {
            if (ns)
              by_h[h].push_back(pd);
            else
              bp.zeros.push_back({bp.y_elems, n * na});
          }
          bp.macs_run += double(na) * double(n) * double(ksum);
          bp.y_elems += n * na;
        }
      }
  for (auto& v : by_h) bp.prods.insert(bp.prods.end(), v.begin(), v.end());
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

  const double* eps = c.d_eps + size_t(inst) * (o + v);
  const DevTables DT = upload_tables(c, H);
  sc.bufs.push_back(DT.mem);

  // dense amplitudes and integral blocks
  cplx* t1d = (cplx*)sc.get(sizeof(cplx) * size_t(o) * v);
  cplx* t2d = (cplx*)sc.get(sizeof(cplx) * size_t(o) * o * v * v);
  ccsd_dense_io(c, inst, t1d, t2d, true);
  cplx* Vd = (cplx*)sc.get(sizeof(cplx) * size_t(o) * o * v * v);  // Vd[j][k][b][c] = <bc||jk>
  ccsd_dense_driver_integral(c, inst, Vd);  // the context's own (scaled) driver integral
  // An integral of the context in the layout (slot k = argument k, two row slots):
  // cached by the context (derived by a permute from a layout of its symmetry family
  // when one is held, else drawn once), with its sub-blocks as gather tasks on the device.
  struct Gathered {
    const Tensor* t = nullptr;
    const GenTask* tasks = nullptr;
    const ChunkRef* chunks = nullptr;
    int n_chunks = 0;
  };
  auto held = [&](const IntRef& V) {
    Gathered g;
    const int ident[4] = {0, 1, 2, 3};
    g.t = integral(c, V, ident, 2);
    std::vector<GenTask> tk;
    std::vector<ChunkRef> ch;
    gen_tasks(c, g.t->L, tk, ch);
    GenTask* d_tk = (GenTask*)sc.get(sizeof(GenTask) * std::max<size_t>(tk.size(), 1));
    ChunkRef* d_ch = (ChunkRef*)sc.get(sizeof(ChunkRef) * std::max<size_t>(ch.size(), 1));
    upload_async(c, d_tk, tk.data(), sizeof(GenTask) * tk.size());
    upload_async(c, d_ch, ch.data(), sizeof(ChunkRef) * ch.size());
    g.tasks = d_tk;
    g.chunks = d_ch;
    g.n_chunks = int(ch.size());
    return g;
  };
  cplx* Wd = (cplx*)sc.get(sizeof(cplx) * size_t(o) * o * v * o);  // Wd[q][r][a][m] = <ma||qr>
  {
    const IntRef OVOO{{SP_OCC, SP_VIRT, SP_OCC, SP_OCC}};
    const Gathered gw = held(OVOO);  // slots (m, a, q, r); forbidden blocks stay zero
    CK(cudaMemsetAsync(Wd, 0, sizeof(cplx) * size_t(o) * o * v * o, c.stream));
    const T3Dense D{{1, o, int64_t(o) * v * o, int64_t(v) * o}, {0, 1, 0, 0}};
    if (gw.n_chunks) {
      k_t3_gather_dense<<<unsigned(gw.n_chunks), T3_THREADS, 0, c.stream>>>(Wd, gw.t->d + size_t(inst) * gw.t->is,
                                                                            gw.tasks, gw.chunks, D, o);
      KCHECK(c);
    }
  }

  // members Bt_{p,h} = B_{p,h}^T (npair[h] rows x K = v_G + o_G columns, G = h - G(p))
  std::vector<int64_t> boff(size_t(o) * G);
  std::vector<EmuSetMat> bmats(size_t(o) * G);
  std::vector<T3BRow> brows;
  int64_t bsz = 0;
  for (int p = 0; p < o; ++p)
    for (int h = 0; h < G; ++h) {
      const int g = ((h - H.go[p]) % G + G) % G;
      const int K = H.vcnt[g] + H.ocnt[g], N = H.npair[h];
      boff[size_t(p) * G + h] = bsz;
      bmats[size_t(p) * G + h] = EmuSetMat{bsz, N, K, h};  // one row exponent per (h, bc) over every p
      if (N)
        for (int k = H.vcnt[g]; k < K; ++k) brows.push_back(T3BRow{bsz, p, h, H.ooff[g] + k - H.vcnt[g], k, K});
      bsz += int64_t(K) * N;
    }
  cplx* Bbuf = (cplx*)sc.get(sizeof(cplx) * size_t(std::max<int64_t>(bsz, 1)));
  {  // the <bc||ep> columns, from the context's integrals
    const IntRef VVVO{{SP_VIRT, SP_VIRT, SP_VIRT, SP_OCC}};
    const Gathered gv = held(VVVO);
    if (gv.n_chunks) {
      int64_t* d_boff = (int64_t*)sc.get(sizeof(int64_t) * boff.size());
      upload_async(c, d_boff, boff.data(), sizeof(int64_t) * boff.size());
      k_t3_gather_bt<<<unsigned(gv.n_chunks), T3_THREADS, 0, c.stream>>>(Bbuf, gv.t->d + size_t(inst) * gv.t->is,
                                                                         gv.tasks, gv.chunks, DT.T, d_boff, o, v);
      KCHECK(c);
    }
  }
  if (!brows.empty()) {
    T3BRow* d_rows = (T3BRow*)sc.get(sizeof(T3BRow) * brows.size());
    upload(c, d_rows, brows.data(), sizeof(T3BRow) * brows.size());
    k_t3_brows<<<unsigned(brows.size()), T3_THREADS, 0, c.stream>>>(Bbuf, d_rows, DT.T, t2d, o, v);
    KCHECK(c);
  }
  if (emulated) {
    sc.A = emu_set_new(c, c.cfg.n_slices, false);
    sc.B = emu_set_new(c, c.cfg.n_slices, true);
    emu_set_slice(c, sc.A, bmats, Bbuf);
  }

  // block size: the largest whose segment and Y^T buffers fit the budget
  const int64_t budget = int64_t(1) << 30;  // complex elements (16 GiB)
  const int nbmax = std::max(1, std::min(o, block > 0 ? block : 64));
  // a lower bound of one triple's Y elements (the smallest over the triples' irreps):
  // a block size whose largest batch times it exceeds the budget is skipped unprobed
  int64_t per = INT64_MAX;
  for (int gijk = 0; gijk < G; ++gijk) {
    int64_t y = 0;
    for (int h = 0; h < G; ++h) y += int64_t(H.npair[h]) * H.vcnt[((gijk - h) % G + G) % G];
    per = std::min(per, y);
  }
  auto most_triples = [&](int cand) {  // triples in the largest batch of block size cand
    const int nblk = (o + cand - 1) / cand;
    auto sz = [&](int b) { return int64_t(std::min((b + 1) * cand, o) - b * cand); };
    int64_t m = 0;
    for (int I = 0; I < nblk; ++I)
      for (int J = I; J < nblk; ++J)
        for (int K = J; K < nblk; ++K) {
          int64_t t;
          if (I < J && J < K) t = sz(I) * sz(J) * sz(K);
          else if (I == J && J < K) t = sz(I) * (sz(I) - 1) / 2 * sz(K);
          else if (I < J) t = sz(I) * sz(J) * (sz(J) - 1) / 2;
          else t = choose3(sz(I));
          m = std::max(m, t);
        }
    return m;
  };
  int nb = 1;
  int64_t max_s = 0, max_y = 0;
  for (int cand = nbmax; cand >= 1; --cand) {
    if (block == 0 && cand > 1 && per > 0 && most_triples(cand) > budget / per) continue;
    const int nblk = (o + cand - 1) / cand;
    int64_t ms = 0, my = 0;
    BlockPlan probe;
    for (int I = 0; I < nblk; ++I)
      for (int J = I; J < nblk; ++J)
        for (int K = J; K < nblk; ++K) {
          plan_block(H, cand, I, J, K, boff, probe, false);
          ms = std::max(ms, probe.s_elems);
          my = std::max(my, probe.y_elems);
        }
    nb = cand;
    max_s = ms;
    max_y = my;
    if (block > 0 || ms + my <= budget) break;  // a requested block size is taken as given
  }
  const int nblk = o ? (o + nb - 1) / nb : 0;
  cplx* Sbuf = (cplx*)sc.get(sizeof(cplx) * size_t(std::max<int64_t>(max_s, 1)));
  cplx* Yt = (cplx*)sc.get(sizeof(cplx) * size_t(std::max<int64_t>(max_y, 1)));
  cplx* e3 = (cplx*)sc.get(sizeof(cplx) * size_t(std::max<int64_t>(ntri, 1)));
  cplx* e3h = (cplx*)sc.get(sizeof(cplx) * size_t(std::max<int64_t>(ntri, 1)) * G);  // per (triple, pair irrep)
  CK(cudaMemsetAsync(e3h, 0, sizeof(cplx) * size_t(std::max<int64_t>(ntri, 1)) * G, c.stream));
  const size_t nb3 = size_t(nb) * nb * nb;  // triples of a batch, at most
  int64_t* d_yoff = (int64_t*)sc.get(sizeof(int64_t) * nb3 * G);
  T3Tri* d_tris = (T3Tri*)sc.get(sizeof(T3Tri) * nb3);
  T3Seg* d_segs = (T3Seg*)sc.get(sizeof(T3Seg) * nb3 * G * 3);
  GemmProb* d_fp = (GemmProb*)sc.get(sizeof(GemmProb) * nb3 * G);

  double macs_need = 0.0, macs_run = 0.0, y_total = 0.0;
  int n_bt = 0;
  BlockPlan bp;
  // per batch: events around its product launch and its energy launch
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
        y_total += double(bp.y_elems);
        macs_need += bp.macs_need;
        macs_run += bp.macs_run;
        // the A^T segments of every (triple, h)
        if (!bp.segs.empty()) {
          upload_async(c, d_segs, bp.segs.data(), sizeof(T3Seg) * bp.segs.size());
          k_t3_segs<<<unsigned(bp.segs.size()), T3_THREADS, 0, c.stream>>>(Sbuf, d_segs, DT.T, t2d, Wd, o, v);
          KCHECK(c);
        }
        for (auto& z : bp.zeros) CK(cudaMemsetAsync(Yt + z.first, 0, sizeof(cplx) * size_t(z.second), c.stream));
        if (emulated) emu_set_slice(c, sc.B, bp.smats, Sbuf);
        mark();
        // Y^T = sum of the segment products, for every (triple, h) of the batch
        if (emulated) {
          emu_set_multiply(c, sc.A, sc.B, bp.prods, Yt, make_double2(1.0, 0.0));
        } else {
          for (int w = 0; w < 3; ++w) {
            std::vector<GemmProb>& fp = bp.fprods[w];
            if (fp.empty()) continue;
            GemmPlan g;
            g.tm = 64;  // N = the virtuals of one irrep: 16-wide column tiles
            g.tn = 16;
            int tile0 = 0;
            for (GemmProb& f : fp) {
              f.tiles_m = (f.M + g.tm - 1) / g.tm;
              f.tiles_n = (f.N + g.tn - 1) / g.tn;
              f.ksplit = 1;
              f.kchunk = (f.K + 7) / 8 * 8;
              f.tile0 = tile0;
              tile0 += f.tiles_m * f.tiles_n;
            }
            g.n_tiles = tile0;
            g.n_probs = int(fp.size());
            upload_async(c, d_fp, fp.data(), sizeof(GemmProb) * fp.size());
            g.d_probs = d_fp;
            OneInstance one(c);
            // the first segment of every product writes its Y^T block, the others add to it
            launch_gemm_fp64(c, g, Bbuf, Sbuf, Yt, 0, 0, 0, make_double2(1.0, 0.0), w > 0);
          }
        }
        mark();
        // energies of the batch's i<j<k
        upload_async(c, d_yoff, bp.yoff.data(), sizeof(int64_t) * bp.yoff.size());
        upload_async(c, d_tris, bp.tris.data(), sizeof(T3Tri) * bp.tris.size());
        mark();
        const dim3 eg(unsigned(bp.tris.size()), unsigned(G));
        if (emulated)
          k_t3_energy<true><<<eg, T3_THREADS, 0, c.stream>>>(d_tris, DT.T, Yt, d_yoff, t1d, Vd, eps, o, v, e3h);
        else
          k_t3_energy<false><<<eg, T3_THREADS, 0, c.stream>>>(d_tris, DT.T, Yt, d_yoff, t1d, Vd, eps, o, v, e3h);
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
    info->x_elems = y_total;
    info->n_triples = ntri;
    info->n_block_triples = n_bt;
    info->block = nb;
  }
}
