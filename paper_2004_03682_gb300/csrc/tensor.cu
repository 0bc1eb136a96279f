// Device kernels on symmetry-blocked tensors: the permute ("tensor
// transposition", steps 1, 2 and 4 of the TTGT list in Sec. II.B), the
// integral generator (step I of the flowchart, Sec. II.B, writing the
// synthetic Hamiltonian of Eq. (ham) straight into blocked layouts), the
// energy denominators of Eq. (amplitudes), and the tau builders.
#include "engine.h"
#include "packed.h"
#include "gen.h"

#include <algorithm>


struct Coefs {
  cplx c[EXP_MAX_TERMS];
};

__device__ __forceinline__ uint32_t udiv(uint32_t x, uint32_t m, uint32_t l) {
  const uint32_t t = __umulhi(m, x);
  return l == 0 ? x : (t + ((x - t) >> 1)) >> (l - 1);
}

// Each CTA handles one chunk of one sub-block task.  Elements are walked in
// destination order (dim 3 innermost, stride 1 in dst) so that stores are
// coalesced; sources are gathered through the task's strides.  SIGNS: every
// coefficient is +1 or -1, applied as a sign-bit flip (GB300 issues FP64
// arithmetic at a small fraction of its integer rate), so a term costs one
// FP64 add and a single-term copy none.
template <int NT, bool SIGNS>
__global__ void __launch_bounds__(256) k_permute(const PermTask* __restrict__ tasks,
                                                 const ChunkRef* __restrict__ chunks,
                                                 cplx* __restrict__ dst,
                                                 const cplx* __restrict__ src, int64_t dis,
                                                 int64_t sis, Coefs co, int acc, int conj) {
  __shared__ PermTask T;
  const ChunkRef ch = chunks[blockIdx.x];
  if (threadIdx.x < sizeof(PermTask) / 8)
    reinterpret_cast<int64_t*>(&T)[threadIdx.x] =
        reinterpret_cast<const int64_t*>(&tasks[ch.task])[threadIdx.x];
  __syncthreads();
  dst += blockIdx.y * dis;
  src += blockIdx.y * sis;
  const uint32_t end = uint32_t(min(ch.start + (int64_t)EXP_CHUNK, T.count));
  const uint32_t n1 = T.n[1], n2 = T.n[2], n3 = T.n[3];
  unsigned long long sgn[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) sgn[t] = co.c[t].x < 0.0 ? 0x8000000000000000ull : 0ull;
  // U elements per step (blockDim apart, so every store instruction stays coalesced):
  // their gathers are all issued before the first store, for U x NT loads in flight
  constexpr int U = NT <= 2 ? 4 : 2;
  for (uint32_t e0 = uint32_t(ch.start) + threadIdx.x; e0 < end; e0 += U * blockDim.x) {
    int64_t dp[U];
    bool live[U];
    double vr[U], vi[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t e = e0 + u * blockDim.x;
      const uint32_t q3 = udiv(e, T.mg[3], T.ml[3]);
      const int i3 = int(e - q3 * n3);
      const uint32_t q2 = udiv(q3, T.mg[2], T.ml[2]);
      const int i2 = int(q3 - q2 * n2);
      const uint32_t q1 = udiv(q2, T.mg[1], T.ml[1]);
      const int i1 = int(q2 - q1 * n1);
      const int i0 = int(q1);
      live[u] = e < end && !(((T.tri & 1) && i0 >= i1) || ((T.tri & 2) && i2 >= i3));
      dp[u] = T.dst + i0 * T.dst_st[0] + i1 * T.dst_st[1] + i2 * T.dst_st[2] + i3 * T.dst_st[3];
      vr[u] = 0.0;
      vi[u] = 0.0;
      // loads not under a branch (a dead element reads its task's first source element,
      // always in bounds), so the U x NT gathers issue back to back
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int64_t sp = live[u] ? T.src[t] + i0 * T.src_st[t][0] + i1 * T.src_st[t][1] + i2 * T.src_st[t][2] +
                                         i3 * T.src_st[t][3]
                                   : T.src[t];
        cplx x = src[sp];
        if (conj) x.y = -x.y;
        if (SIGNS) {
          const double xr = __longlong_as_double(__double_as_longlong(x.x) ^ (long long)sgn[t]);
          const double xi = __longlong_as_double(__double_as_longlong(x.y) ^ (long long)sgn[t]);
          if (t == 0) { vr[u] = xr; vi[u] = xi; } else { vr[u] += xr; vi[u] += xi; }
        } else {
          vr[u] += co.c[t].x * x.x - co.c[t].y * x.y;
          vi[u] += co.c[t].x * x.y + co.c[t].y * x.x;
        }
      }
    }
    if (acc) {
      cplx o[U];
#pragma unroll
      for (int u = 0; u < U; ++u) o[u] = dst[live[u] ? dp[u] : T.dst];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        vr[u] += o[u].x;
        vi[u] += o[u].y;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (live[u]) dst[dp[u]] = make_double2(vr[u], vi[u]);
  }
}

template <int NT>
static void permute_nt(Ctx& c, const PermPlan& p, cplx* dst, const cplx* src, int64_t dst_is, int64_t src_is,
                       const Coefs& co, bool signs, bool accumulate, bool conj) {
  dim3 grid(p.n_chunks, c.ninst);
  if (signs)
    k_permute<NT, true><<<grid, 256, 0, c.stream>>>(p.d_tasks, p.d_chunks, dst, src, dst_is, src_is, co, accumulate,
                                                    conj);
  else
    k_permute<NT, false><<<grid, 256, 0, c.stream>>>(p.d_tasks, p.d_chunks, dst, src, dst_is, src_is, co, accumulate,
                                                     conj);
}

void launch_permute(Ctx& c, const PermPlan& p, cplx* dst, const cplx* src, int64_t dst_is,
                    int64_t src_is, const cplx* coef, bool accumulate, bool conj_src) {
  if (p.n_chunks == 0) return;
  Coefs co;
  bool signs = true;
  for (int t = 0; t < EXP_MAX_TERMS; ++t) {
    co.c[t] = t < p.n_terms ? coef[t] : make_double2(0, 0);
    if (t < p.n_terms && !(co.c[t].y == 0.0 && (co.c[t].x == 1.0 || co.c[t].x == -1.0))) signs = false;
  }
  switch (p.n_terms) {
    case 1: permute_nt<1>(c, p, dst, src, dst_is, src_is, co, signs, accumulate, conj_src); break;
    case 2: permute_nt<2>(c, p, dst, src, dst_is, src_is, co, signs, accumulate, conj_src); break;
    case 3: permute_nt<3>(c, p, dst, src, dst_is, src_is, co, signs, accumulate, conj_src); break;
    default: permute_nt<4>(c, p, dst, src, dst_is, src_is, co, signs, accumulate, conj_src); break;
  }
  KCHECK(c);
}

struct Map4 {
  int m[4];
};

// genmap (nullable): global spinor index -> generator index, -1 for a ghost spinor
// (every integral with a ghost index is zero).  n = number of generator indices.
__global__ void __launch_bounds__(256) k_generate(cplx* __restrict__ dst, int64_t is,
                                                  const GenTask* __restrict__ tasks,
                                                  const ChunkRef* __restrict__ chunks, Map4 map,
                                                  int n, const uint64_t* __restrict__ seeds,
                                                  const double* __restrict__ scales,
                                                  const int* __restrict__ genmap, int real) {
  const ChunkRef ch = chunks[blockIdx.x];
  const GenTask T = tasks[ch.task];
  const int inst = blockIdx.y;
  dst += inst * is;
  const uint64_t seed = seeds[inst];
  const double sc = scales[inst];
  const int64_t end = min(ch.start + (int64_t)EXP_CHUNK, T.count);
  for (int64_t e = ch.start + threadIdx.x; e < end; e += blockDim.x) {
    int64_t r = e;
    int i[4];
    i[3] = int(r % T.n[3]); r /= T.n[3];
    i[2] = int(r % T.n[2]); r /= T.n[2];
    i[1] = int(r % T.n[1]);
    i[0] = int(r / T.n[1]);
    uint64_t g[4];
    bool ghost = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int gi = T.g0[k] + i[k];
      if (genmap) {
        gi = genmap[gi];
        ghost |= gi < 0;
      }
      g[k] = uint64_t(gi < 0 ? 0 : gi);
    }
    const int64_t dp = T.base + i[0] * T.st[0] + i[1] * T.st[1] + i[2] * T.st[2] + i[3] * T.st[3];
    if (ghost) {
      dst[dp] = make_double2(0.0, 0.0);
      continue;
    }
    const cplx v = v_element(g[map.m[0]], g[map.m[1]], g[map.m[2]], g[map.m[3]], uint64_t(n), seed);
    // real arithmetic: the recipe on Re A, i.e. the real part (every step is real-linear)
    dst[dp] = make_double2(sc * v.x, real ? 0.0 : sc * v.y);
  }
}

void launch_generate(Ctx& c, cplx* dst, int64_t is, const GenTask* d_tasks, const ChunkRef* d_chunks,
                     int n_chunks, const int map[4]) {
  if (!n_chunks) return;
  Map4 m;
  // generator tasks use padded dims: slot k of a rank-4 tensor is dim k
  for (int k = 0; k < 4; ++k) m.m[k] = map[k];
  k_generate<<<dim3(n_chunks, c.ninst), 256, 0, c.stream>>>(dst, is, d_tasks, d_chunks, m,
                                                            c.n_gen, c.d_seed, c.d_scale, c.d_genmap,
                                                            c.cfg.real_arith);
  KCHECK(c);
}

// D = -sum_k sign_k eps(g_k)  (D_i^a = e_i - e_a, D_ij^ab = e_i + e_j - e_a - e_b)
struct Sgn4 {
  int s[4];
};
__global__ void k_fill_denom(double* __restrict__ dst, int64_t is, const GenTask* __restrict__ tasks,
                             const ChunkRef* __restrict__ chunks, Sgn4 sg, int n,
                             const double* __restrict__ eps) {
  const ChunkRef ch = chunks[blockIdx.x];
  const GenTask T = tasks[ch.task];
  const int inst = blockIdx.y;
  dst += inst * is;
  eps += inst * n;
  const int64_t end = min(ch.start + (int64_t)EXP_CHUNK, T.count);
  for (int64_t e = ch.start + threadIdx.x; e < end; e += blockDim.x) {
    int64_t r = e;
    int i[4];
    i[3] = int(r % T.n[3]); r /= T.n[3];
    i[2] = int(r % T.n[2]); r /= T.n[2];
    i[1] = int(r % T.n[1]);
    i[0] = int(r / T.n[1]);
    double d = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (sg.s[k]) d -= sg.s[k] * eps[T.g0[k] + i[k]];
    dst[T.base + i[0] * T.st[0] + i[1] * T.st[1] + i[2] * T.st[2] + i[3] * T.st[3]] = d;
  }
}

void launch_fill_denom(Ctx& c, double* dst, int64_t is, const GenTask* d_tasks, const ChunkRef* d_chunks,
                       int n_chunks, int nslots, const int sgn[4], const double* eps) {
  if (!n_chunks) return;
  Sgn4 s;
  const int pad = 4 - nslots;
  for (int k = 0; k < 4; ++k) s.s[k] = 0;
  for (int k = 0; k < nslots; ++k) s.s[pad + k] = sgn[k];
  k_fill_denom<<<dim3(n_chunks, c.ninst), 256, 0, c.stream>>>(dst, is, d_tasks, d_chunks, s, c.no + c.nv,
                                                              eps ? eps : c.d_eps);
  KCHECK(c);
}

// dst_abij = c0 t2_abij + c1 t1_ai t1_bj + c2 t1_bi t1_aj over the t2 layout.
// t1_index[a_local * no + i_local] = offset of t1_ai in its layout, or -1.
__global__ void k_tau(cplx* __restrict__ dst, int64_t dis, const cplx* __restrict__ t2,
                      const cplx* __restrict__ t1, int64_t tis, const int32_t* __restrict__ t1i,
                      const GenTask* __restrict__ tasks, const ChunkRef* __restrict__ chunks,
                      double c0, double c1, double c2, int no, int vbase) {
  const ChunkRef ch = chunks[blockIdx.x];
  const GenTask T = tasks[ch.task];
  dst += blockIdx.y * dis;
  t2 += blockIdx.y * tis;
  t1 += blockIdx.y * tis;
  const int64_t end = min(ch.start + (int64_t)EXP_CHUNK, T.count);
  for (int64_t e = ch.start + threadIdx.x; e < end; e += blockDim.x) {
    int64_t r = e;
    int i[4];
    i[3] = int(r % T.n[3]); r /= T.n[3];
    i[2] = int(r % T.n[2]); r /= T.n[2];
    i[1] = int(r % T.n[1]);
    i[0] = int(r / T.n[1]);
    const int a = T.g0[0] + i[0] - vbase, b = T.g0[1] + i[1] - vbase;
    const int ii = T.g0[2] + i[2], jj = T.g0[3] + i[3];
    const int64_t p = T.base + i[0] * T.st[0] + i[1] * T.st[1] + i[2] * T.st[2] + i[3] * T.st[3];
    const cplx x = t2[p];
    double vr = c0 * x.x, vi = c0 * x.y;
    const int ai = t1i[a * no + ii], bj = t1i[b * no + jj];
    if (ai >= 0 && bj >= 0) {
      const cplx u = t1[ai], w = t1[bj];
      vr += c1 * (u.x * w.x - u.y * w.y);
      vi += c1 * (u.x * w.y + u.y * w.x);
    }
    const int bi = t1i[b * no + ii], aj = t1i[a * no + jj];
    if (bi >= 0 && aj >= 0) {
      const cplx u = t1[bi], w = t1[aj];
      vr += c2 * (u.x * w.x - u.y * w.y);
      vi += c2 * (u.x * w.y + u.y * w.x);
    }
    dst[p] = make_double2(vr, vi);
  }
}

// The three tau-like tensors of one iteration in one pass (the t1 products are
// formed once): with A = t1_ai t1_bj and B = t1_bi t1_aj,
//   tau = t2 + A - B,   taut = t2 + (A - B)/2,   zeta = t2/2 + A.
__global__ void k_tau3(cplx* __restrict__ tau, cplx* __restrict__ taut, cplx* __restrict__ zeta, int64_t dis,
                       const cplx* __restrict__ t2, const cplx* __restrict__ t1, int64_t tis,
                       const int32_t* __restrict__ t1i, const GenTask* __restrict__ tasks,
                       const ChunkRef* __restrict__ chunks, int no, int vbase) {
  const ChunkRef ch = chunks[blockIdx.x];
  const GenTask T = tasks[ch.task];
  tau += blockIdx.y * dis;
  taut += blockIdx.y * dis;
  zeta += blockIdx.y * dis;
  t2 += blockIdx.y * tis;
  t1 += blockIdx.y * tis;
  const uint32_t n1 = T.n[1], n2 = T.n[2], n3 = T.n[3];
  const uint32_t end = uint32_t(min(ch.start + (int64_t)EXP_CHUNK, T.count));
  for (uint32_t e = uint32_t(ch.start) + threadIdx.x; e < end; e += blockDim.x) {
    uint32_t r = e;
    const int i3 = int(r % n3);
    r /= n3;
    const int i2 = int(r % n2);
    r /= n2;
    const int i1 = int(r % n1);
    const int i0 = int(r / n1);
    const int a = T.g0[0] + i0 - vbase, b = T.g0[1] + i1 - vbase;
    const int ii = T.g0[2] + i2, jj = T.g0[3] + i3;
    const int64_t p = T.base + i0 * T.st[0] + i1 * T.st[1] + i2 * T.st[2] + i3 * T.st[3];
    const cplx x = t2[p];
    const int kai = t1i[a * no + ii], kbj = t1i[b * no + jj];
    const int kbi = t1i[b * no + ii], kaj = t1i[a * no + jj];
    if ((kai < 0 || kbj < 0) && (kbi < 0 || kaj < 0)) {
      // no t1 product is symmetry-allowed here (most elements under Z_G): the same values
      // without the FP64 adds of zero (GB300's FP64 pipe bounds this kernel otherwise)
      tau[p] = x;
      taut[p] = x;
      zeta[p] = make_double2(0.5 * x.x, 0.5 * x.y);
      continue;
    }
    double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;
    if (kai >= 0 && kbj >= 0) {
      const cplx u = t1[kai], w = t1[kbj];
      ar = u.x * w.x - u.y * w.y;
      ai = u.x * w.y + u.y * w.x;
    }
    if (kbi >= 0 && kaj >= 0) {
      const cplx u = t1[kbi], w = t1[kaj];
      br = u.x * w.x - u.y * w.y;
      bi = u.x * w.y + u.y * w.x;
    }
    const double dr = ar - br, di = ai - bi;
    tau[p] = make_double2(x.x + dr, x.y + di);
    taut[p] = make_double2(fma(0.5, dr, x.x), fma(0.5, di, x.y));
    zeta[p] = make_double2(fma(0.5, x.x, ar), fma(0.5, x.y, ai));
  }
}

void launch_tau3(Ctx& c, cplx* tau, cplx* taut, cplx* zeta, int64_t dst_is, const cplx* t2, const cplx* t1,
                 int64_t t_is, const int32_t* t1_index, const GenTask* d_tasks, const ChunkRef* d_chunks,
                 int n_chunks) {
  if (!n_chunks) return;
  k_tau3<<<dim3(n_chunks, c.ninst), 256, 0, c.stream>>>(tau, taut, zeta, dst_is, t2, t1, t_is, t1_index, d_tasks,
                                                        d_chunks, c.no, c.no);
  KCHECK(c);
}

void launch_tau(Ctx& c, cplx* dst, int64_t dst_is, const cplx* t2, const cplx* t1, int64_t t_is,
                const int32_t* t1_index, const GenTask* d_tasks, const ChunkRef* d_chunks,
                int n_chunks, double c0, double c1, double c2) {
  if (!n_chunks) return;
  k_tau<<<dim3(n_chunks, c.ninst), 256, 0, c.stream>>>(dst, dst_is, t2, t1, t_is, t1_index, d_tasks,
                                                       d_chunks, c0, c1, c2, c.no, c.no);
  KCHECK(c);
}

// ---------------------------------------------------------------------------
// Integrals straight into a pair-packed matrix: element (p, q; r, s) of block g
// with the pairs (p, q) from the row table and (r, s) from the column table.
__global__ void __launch_bounds__(256) k_generate_pairs(cplx* __restrict__ dst, int64_t is, PackDims D,
                                                        const int32_t* __restrict__ rpair,
                                                        const int32_t* __restrict__ cpair, int n,
                                                        const uint64_t* __restrict__ seeds,
                                                        const double* __restrict__ scales,
                                                        const int* __restrict__ genmap, int herm, int real) {
  const int inst = blockIdx.y;
  dst += inst * is;
  const uint64_t seed = seeds[inst];
  const double sc = scales[inst];
  const int64_t total = D.blk[D.G];
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    int g = 0;
    while (g + 1 < D.G && e >= D.blk[g + 1]) ++g;
    const uint32_t loc = uint32_t(e - D.blk[g]);
    const uint32_t p = loc / uint32_t(D.nc[g]), q = loc - p * uint32_t(D.nc[g]);
    // herm (rows and columns from one table): element (q, p) is conj of (p, q) -- the
    // recipe's Hermitisation adds the same two terms -- so only p <= q is drawn
    if (herm && q < p) continue;
    const int32_t rc = rpair[D.roff[g] + p], cc = cpair[D.coff[g] + q];
    int gi[4] = {rc >> 16, rc & 0xFFFF, cc >> 16, cc & 0xFFFF};
    bool ghost = false;
    if (genmap)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        gi[k] = genmap[gi[k]];
        ghost |= gi[k] < 0;
      }
    cplx v = make_double2(0.0, 0.0);
    if (!ghost) {
      const cplx w = v_element(uint64_t(gi[0]), uint64_t(gi[1]), uint64_t(gi[2]), uint64_t(gi[3]), uint64_t(n), seed);
      v = make_double2(sc * w.x, real ? 0.0 : sc * w.y);
    }
    dst[e] = v;
    if (herm && q > p) dst[D.blk[g] + int64_t(q) * D.nc[g] + p] = make_double2(v.x, -v.y);
  }
}

void launch_generate_pairs(Ctx& c, cplx* dst, int64_t is, const PackDims& D, const PairTable& R, const PairTable& C) {
  const int64_t total = D.blk[D.G];
  if (total == 0) return;
  const int blocks = int(std::min<int64_t>((total + 255) / 256, int64_t(std::max(c.sm_count, 1)) * 8));
  k_generate_pairs<<<dim3(blocks, c.ninst), 256, 0, c.stream>>>(dst, is, D, R.d_pair, C.d_pair, c.n_gen, c.d_seed,
                                                                c.d_scale, c.d_genmap, &R == &C ? 1 : 0,
                                                                c.cfg.real_arith);
  KCHECK(c);
}
