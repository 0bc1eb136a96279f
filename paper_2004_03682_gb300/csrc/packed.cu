// Pair-packed antisymmetric compounds (p<q per pair irrep) and the packed
// particle-particle ladder.  The blocked layouts of Sec. II.C store t2, tau and
// <ab||cd> with full pair compounds; antisymmetry makes three quarters of
// <ab||cd> and half of each tau column redundant, and the ladder of
// Eq. (amplitudes) needs only
//     Z_ij^ab = sum_{c<d} <ab||cd> tau_ij^cd,   r2_ij^ab += Z, with Z_ij^ba = -Z_ij^ab.
// Packed operands are plain per-irrep matrices, so the product is one more
// grouped GEMM (step 3 of the TTGT list, Sec. II.B) on the same kernels.
#include <algorithm>
#include <cstdio>
#include <functional>
#include <map>
#include <memory>

#include "emu.h"
#include "packed.h"

static inline int imod(int a, int G) { return ((a % G) + G) % G; }

void build_pair_table(Ctx& c, const Layout& L, bool rows, bool packed, PairTable& T) {
  const int G = c.G;
  if (G > PK_MAXG) throw ExpError{EXP_EINVAL, "packed pairs: too many irreps"};
  const int ns = rows ? L.nrow : L.rank - L.nrow;
  if (ns != 2) throw ExpError{EXP_EINVAL, "packed pairs: compound must have two slots"};
  const int s0 = rows ? 0 : L.nrow, s1 = s0 + 1;
  const Space& S0 = c.spaces[L.sp[s0]];
  const Space& S1 = c.spaces[L.sp[s1]];
  const int sg0 = L.sg[s0], sg1 = L.sg[s1];
  if (packed && (L.sp[s0] != L.sp[s1] || sg0 != sg1))
    throw ExpError{EXP_EINVAL, "packed pairs: slots of different spaces or signs"};
  if (S0.gbase + S0.n > 32768 || S1.gbase + S1.n > 32768) throw ExpError{EXP_EINVAL, "packed pairs: too many spinors"};
  const std::vector<int64_t>& tup = rows ? L.rtup : L.ctup;
  auto in_block = [&](int g0, int g1) {
    const int s = sg0 * g0 + sg1 * g1;
    return (rows ? imod(s, G) : imod(-s, G));
  };
  T.G = G;
  T.n.assign(G, 0);
  T.off.assign(G, 0);
  T.fn.assign(G, 0);
  T.foff.assign(G, 0);
  T.pair.clear();
  T.full.clear();
  T.inv.clear();
  T.swp.clear();
  for (int g = 0; g < G; ++g) {
    const int64_t fsz = rows ? L.rows[g] : L.cols[g];
    if (fsz >= (int64_t(1) << 31)) throw ExpError{EXP_EINVAL, "packed pairs: block above 2^31"};
    T.fn[g] = int32_t(fsz);
    T.foff[g] = int32_t(T.inv.size());
    T.off[g] = int32_t(T.pair.size());
    const size_t inv0 = T.inv.size();
    T.inv.resize(inv0 + size_t(fsz), 0);
    auto full_index = [&](int g0, int x0, int g1, int x1) {
      return int32_t(tup[size_t(g0) * G + g1] + int64_t(x0) * S1.cnt[g1] + x1);
    };
    auto code = [&](int g0, int x0, int g1, int x1) {
      return int32_t(((S0.gbase + S0.off[g0] + x0) << 16) | (S1.gbase + S1.off[g1] + x1));
    };
    if (!packed) {  // every tuple, layout order
      for (int g0 = 0; g0 < G; ++g0)
        for (int g1 = 0; g1 < G; ++g1) {
          if (in_block(g0, g1) != g) continue;
          for (int x0 = 0; x0 < S0.cnt[g0]; ++x0)
            for (int x1 = 0; x1 < S1.cnt[g1]; ++x1) {
              const int32_t f = full_index(g0, x0, g1, x1);
              const int32_t k = int32_t(T.pair.size()) - T.off[g];
              T.pair.push_back(code(g0, x0, g1, x1));
              T.full.push_back(f);
              T.swp.push_back(f);
              T.inv[inv0 + f] = k + 1;
            }
        }
    } else {  // canonical p<q: irrep pairs g0 < g1 whole, g0 = g1 strict triangle
      for (int g0 = 0; g0 < G; ++g0)
        for (int g1 = g0; g1 < G; ++g1) {
          if (in_block(g0, g1) != g) continue;
          for (int x0 = 0; x0 < S0.cnt[g0]; ++x0)
            for (int x1 = (g0 == g1 ? x0 + 1 : 0); x1 < S1.cnt[g1]; ++x1) {
              const int32_t k = int32_t(T.pair.size()) - T.off[g];
              T.pair.push_back(code(g0, x0, g1, x1));
              T.full.push_back(full_index(g0, x0, g1, x1));
              T.swp.push_back(full_index(g1, x1, g0, x0));
              T.inv[inv0 + full_index(g0, x0, g1, x1)] = k + 1;
              T.inv[inv0 + full_index(g1, x1, g0, x0)] = -(k + 1);
            }
        }
    }
    T.n[g] = int32_t(T.pair.size()) - T.off[g];
  }
  auto up = [&](const std::vector<int32_t>& v) {
    int32_t* d = (int32_t*)c.dalloc(sizeof(int32_t) * std::max<size_t>(v.size(), 1));
    if (!v.empty()) upload(c, d, v.data(), sizeof(int32_t) * v.size());
    return d;
  };
  T.d_pair = up(T.pair);
  T.d_full = up(T.full);
  T.d_inv = up(T.inv);
  T.d_swp = up(T.swp);
}

PackDims pack_dims(const PairTable& R, const PairTable& C) {
  PackDims D{};
  D.G = R.G;
  int64_t o = 0, fo = 0;
  for (int g = 0; g < R.G; ++g) {
    D.blk[g] = o;
    D.fblk[g] = fo;
    D.nr[g] = R.n[g];
    D.nc[g] = C.n[g];
    D.roff[g] = R.off[g];
    D.coff[g] = C.off[g];
    D.fnr[g] = R.fn[g];
    D.fnc[g] = C.fn[g];
    D.froff[g] = R.foff[g];
    D.fcoff[g] = C.foff[g];
    o += int64_t(R.n[g]) * C.n[g];
    fo += int64_t(R.fn[g]) * C.fn[g];
  }
  D.blk[R.G] = o;
  D.fblk[R.G] = fo;
  return D;
}


__global__ void __launch_bounds__(256) k_pack_gather(cplx* __restrict__ dst, int64_t dis, const cplx* __restrict__ src,
                                                     int64_t sis, PackDims D, const int32_t* __restrict__ rfull,
                                                     const int32_t* __restrict__ cfull) {
  const int inst = blockIdx.y;
  dst += inst * dis;
  src += inst * sis;
  const int64_t total = D.blk[D.G];
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int g = find_block(D.blk, D.G, e);
    const uint32_t loc = uint32_t(e - D.blk[g]);
    const uint32_t p = loc / uint32_t(D.nc[g]), q = loc - p * uint32_t(D.nc[g]);
    dst[e] = src[D.fblk[g] + int64_t(rfull[D.roff[g] + p]) * D.fnc[g] + cfull[D.coff[g] + q]];
  }
}

// full element (R, C): entries kr = |inv_r| - 1, kc = |inv_c| - 1, sign = product of
// the inv signs (times coef); a p = q row or column has no packed entry
__global__ void __launch_bounds__(256) k_pack_scatter(cplx* __restrict__ dst, int64_t dis, const cplx* __restrict__ src,
                                                      int64_t sis, PackDims D, const int32_t* __restrict__ rinv,
                                                      const int32_t* __restrict__ cinv, int neg, int acc) {
  const int inst = blockIdx.y;
  dst += inst * dis;
  src += inst * sis;
  const int64_t total = D.fblk[D.G];
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int g = find_block(D.fblk, D.G, e);
    const uint32_t loc = uint32_t(e - D.fblk[g]);
    const uint32_t R = loc / uint32_t(D.fnc[g]), Cc = loc - R * uint32_t(D.fnc[g]);
    const int ir = rinv[D.froff[g] + R], ic = cinv[D.fcoff[g] + Cc];
    if (ir == 0 || ic == 0) {
      if (!acc) dst[e] = make_double2(0.0, 0.0);
      continue;
    }
    const int kr = (ir < 0 ? -ir : ir) - 1, kc = (ic < 0 ? -ic : ic) - 1;
    const long long sgn = (((ir < 0) ^ (ic < 0) ^ neg) != 0) ? (long long)0x8000000000000000ull : 0ll;
    const cplx v = src[D.blk[g] + int64_t(kr) * D.nc[g] + kc];
    const double vr = __longlong_as_double(__double_as_longlong(v.x) ^ sgn);
    const double vi = __longlong_as_double(__double_as_longlong(v.y) ^ sgn);
    if (acc) {
      const cplx o = dst[e];
      dst[e] = make_double2(o.x + vr, o.y + vi);
    } else {
      dst[e] = make_double2(vr, vi);
    }
  }
}

// dst[full] += sign * src[packed] at the canonical full positions only: entries whose
// row and column pairs are both p < q (a packed table's entries all are; an unpacked
// table's others are skipped), each written once, at its own position
__global__ void __launch_bounds__(256) k_pack_put_canon(cplx* __restrict__ dst, int64_t dis,
                                                        const cplx* __restrict__ src, int64_t sis, PackDims D,
                                                        const int32_t* __restrict__ rfull,
                                                        const int32_t* __restrict__ cfull,
                                                        const int32_t* __restrict__ rpair,
                                                        const int32_t* __restrict__ cpair, int neg) {
  const int inst = blockIdx.y;
  dst += inst * dis;
  src += inst * sis;
  const int64_t total = D.blk[D.G];
  const long long sgn = neg ? (long long)0x8000000000000000ull : 0ll;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int g = find_block(D.blk, D.G, e);
    const uint32_t loc = uint32_t(e - D.blk[g]);
    const uint32_t p = loc / uint32_t(D.nc[g]), q = loc - p * uint32_t(D.nc[g]);
    const int32_t pr = rpair[D.roff[g] + p], pc = cpair[D.coff[g] + q];
    if ((pr >> 16) >= (pr & 0xffff) || (pc >> 16) >= (pc & 0xffff)) continue;
    const cplx v = src[e];
    cplx& o = dst[D.fblk[g] + int64_t(rfull[D.roff[g] + p]) * D.fnc[g] + cfull[D.coff[g] + q]];
    o = make_double2(o.x + __longlong_as_double(__double_as_longlong(v.x) ^ sgn),
                     o.y + __longlong_as_double(__double_as_longlong(v.y) ^ sgn));
  }
}

static int pk_blocks(Ctx& c, int64_t n) {
  return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, int64_t(std::max(c.sm_count, 1)) * 8)));
}

void launch_pack_gather(Ctx& c, cplx* dst, int64_t dis, const cplx* src, int64_t sis, const PackDims& D,
                        const PairTable& R, const PairTable& C) {
  if (D.blk[D.G] == 0) return;
  k_pack_gather<<<dim3(pk_blocks(c, D.blk[D.G]), c.ninst), 256, 0, c.stream>>>(dst, dis, src, sis, D, R.d_full,
                                                                              C.d_full);
  KCHECK(c);
}

// into a pair_canon destination while Ctx::canon_pairs is set: canonical entries only
static void scatter_into(Ctx& c, Tensor& dst, const cplx* src, int64_t sis, const PackDims& D, const PairTable& R,
                         const PairTable& C) {
  if (!(dst.pair_canon && c.canon_pairs)) {
    launch_pack_scatter(c, dst.d, dst.is, src, sis, D, R, C, 1.0, true);
    return;
  }
  if (D.blk[D.G] == 0) return;
  k_pack_put_canon<<<dim3(pk_blocks(c, D.blk[D.G]), c.ninst), 256, 0, c.stream>>>(
      dst.d, dst.is, src, sis, D, R.d_full, C.d_full, R.d_pair, C.d_pair, 0);
  KCHECK(c);
}

void launch_pack_scatter(Ctx& c, cplx* dst, int64_t dis, const cplx* src, int64_t sis, const PackDims& D,
                         const PairTable& R, const PairTable& C, double coef, bool accumulate) {
  if (coef != 1.0 && coef != -1.0) throw ExpError{EXP_EINVAL, "packed scatter: coefficient must be +-1"};
  if (D.fblk[D.G] == 0) return;
  k_pack_scatter<<<dim3(pk_blocks(c, D.fblk[D.G]), c.ninst), 256, 0, c.stream>>>(
      dst, dis, src, sis, D, R.d_inv, C.d_inv, coef < 0 ? 1 : 0, accumulate ? 1 : 0);
  KCHECK(c);
}

// ---------------------------------------------------------------------------
// Packed contractions.  tau is gathered once per iteration into
//   T_P[g] = tau_ij^cd,  rows c<d, cols i<j,
// and serves every product that sums over a tau pair index:
//   R2pp   r2_ij^ab  += sum_{c<d} <ab||cd> T_P            (A = <ab||cd>, a<b, c<d)
//   Xamij  X_am,ij    = 2 sum_{e<f} <am||ef> T_P          (A = <am||ef>, e<f)
//   Wmnij2 W_mn,ij   += sum_{e<f} <mn||ef> T_P            (A = <mn||ef>, m<n, e<f)
//   R2hh   r2_ij^ab  += sum_{m<n} T_P(ab, mn) W_mn,ij      (B = W gathered to m<n)
// (each a sum over the full pair with factor 1/2 in Eq. (amplitudes) and the
// Stanton-Gauss intermediates).  Results are scattered into the blocked tensors
// with the signs of the pair swaps.
struct PackedOp {
  std::string site;
  Tensor A, B, C;             // packed operands (A or B may alias the shared T_P)
  int64_t offB = -1, offC = 0;  // operand-arena element offsets of B (-1: not there) and C
  PackDims dA{}, dB{}, dC{};  // with the full counterparts for generation / gather / scatter
  const PairTable *Ar = nullptr, *Ac = nullptr, *Br = nullptr, *Bc = nullptr, *Cr = nullptr, *Cc = nullptr;
  EinsumPlan* plan = nullptr;  // owned by c.plans
};

struct PackedState {
  std::map<std::string, std::unique_ptr<PairTable>> tables;
  Tensor TP;  // packed tau
  PackDims dT{};
  const PairTable *vv = nullptr, *oo = nullptr;
  std::map<std::string, std::unique_ptr<PackedOp>> ops;
};

static PackedState& PS(Ctx& c) {
  if (!c.packed_state) c.packed_state = new PackedState();
  return *(PackedState*)c.packed_state;
}

static const PairTable& table(Ctx& c, const Layout& L, bool rows, bool packed) {
  PackedState& s = PS(c);
  const std::string key = L.key() + (rows ? "|r" : "|c") + (packed ? "p" : "f");
  auto it = s.tables.find(key);
  if (it != s.tables.end()) return *it->second;
  PairTable* t = new PairTable();
  build_pair_table(c, L, rows, packed, *t);
  s.tables[key].reset(t);
  return *t;
}

static Layout packed_layout(const PairTable& R, const PairTable& C) {
  Layout L;
  L.rank = 2;
  L.nrow = 1;
  L.G = R.G;
  L.rows.assign(R.G, 0);
  L.cols.assign(R.G, 0);
  L.blk_off.assign(R.G, 0);
  int64_t o = 0;
  for (int g = 0; g < R.G; ++g) {
    L.rows[g] = R.n[g];
    L.cols[g] = C.n[g];
    L.blk_off[g] = o;
    o += int64_t(R.n[g]) * C.n[g];
  }
  L.size = o;
  return L;
}

static Tensor packed_tensor(Ctx& c, const PairTable& R, const PairTable& C) {
  Tensor* t = new_tensor(c, packed_layout(R, C), false);
  Tensor r = *t;
  delete t;
  return r;
}

// a packed matrix placed in the operand arena at run time
static Tensor arena_tensor(const PairTable& R, const PairTable& C) {
  Tensor t;
  t.L = packed_layout(R, C);
  t.is = std::max<int64_t>(t.L.size, 1);
  t.d = nullptr;
  return t;
}

const PackDims& packed_t2_space(Ctx& c, const Layout& L, const PairTable** vv, const PairTable** oo) {
  PackedState& s = PS(c);
  if (!s.vv) {
    s.vv = &table(c, L, true, true);   // (c, d), c < d
    s.oo = &table(c, L, false, true);  // (i, j), i < j
    s.dT = pack_dims(*s.vv, *s.oo);
    s.TP = packed_tensor(c, *s.vv, *s.oo);
  }
  if (vv) *vv = s.vv;
  if (oo) *oo = s.oo;
  return s.dT;
}

void packed_tau(Ctx& c, const Tensor& tau) {
  PackedState& s = PS(c);
  packed_t2_space(c, tau.L, nullptr, nullptr);
  launch_pack_gather(c, s.TP.d, s.TP.is, tau.d, tau.is, s.dT, *s.vv, *s.oo);
}

// C_P = A_P B_P through the emulated or FP64 grouped GEMM, registered in c.plans
// under `site` (so the work accounting and the top-contraction report see it)
static void finish_op(Ctx& c, PackedOp* op, bool a_const, double alpha = 1.0) {
  {
    int64_t off = 0;
    if (op->offB >= 0) { op->offB = off; off += op->B.is * c.ninst; }
    op->offC = off;
    off += op->C.is * c.ninst;
    arena_reserve(c, c.op_arena, size_t(off) * sizeof(cplx));
  }
  EinsumPlan* P = new EinsumPlan();
  c.plans[op->site].reset(P);
  op->plan = P;
  P->A = &op->A;
  P->B = &op->B;
  P->permC = true;
  P->C2 = op->C;
  P->alpha = make_double2(alpha, 0.0);
  P->gemm_beta = false;
  P->g = make_gemm_plan(c, op->A.L, op->B.L, op->C.L);
  P->emulate = emu_wanted(c, P->g, op->site);
  if (P->emulate) P->emu = emu_plan(c, P->g, &op->A, &op->B, a_const, false, op->offB < 0, op->site);
}

static void run_op(Ctx& c, PackedOp* op, const std::function<void()>& before, const std::function<void()>& after) {
  EinsumPlan* P = op->plan;
  cplx* ab = (cplx*)c.op_arena.base;
  if (op->offB >= 0) op->B.d = ab + op->offB;
  op->C.d = ab + op->offC;
  P->C2.d = op->C.d;
  const bool prof = c.profile;
  cudaEvent_t pe[2] = {nullptr, nullptr};
  if (prof) {
    for (auto& e : pe) CK(cudaEventCreate(&e));
    CK(cudaEventRecord(c.pev0, c.stream));
  }
  before();
  if (prof) CK(cudaEventRecord(pe[0], c.stream));
  if (P->emulate)
    emu_run(c, P->emu, P->g, op->A.d, op->B.d, op->C.d, op->A.is, op->B.is, op->C.is, P->alpha, false);
  else
    launch_gemm_fp64(c, P->g, op->A.d, op->B.d, op->C.d, op->A.is, op->B.is, op->C.is, P->alpha, false);
  if (prof) CK(cudaEventRecord(pe[1], c.stream));
  after();
  if (prof) {
    CK(cudaEventRecord(c.pev1, c.stream));
    CK(cudaEventSynchronize(c.pev1));
    float ms = 0.f, m_in = 0.f, m_g = 0.f, m_out = 0.f;
    CK(cudaEventElapsedTime(&ms, c.pev0, c.pev1));
    CK(cudaEventElapsedTime(&m_in, c.pev0, pe[0]));
    CK(cudaEventElapsedTime(&m_g, pe[0], pe[1]));
    CK(cudaEventElapsedTime(&m_out, pe[1], c.pev1));
    for (auto& e : pe) cudaEventDestroy(e);
    int64_t M = 0, N = 0, K = 0;
    for (auto& q : P->g.h_probs) { M = std::max<int64_t>(M, q.M); N = std::max<int64_t>(N, q.N); K = std::max<int64_t>(K, q.K); }
    fprintf(stderr, "[exp_phase] %-8s in %7.3f  gemm %7.3f  out %7.3f ms\n", op->site.c_str(), m_in, m_g, m_out);
    fprintf(stderr,
            "[exp_profile] %-8s %9.3f ms  %10.3g cMAC  %7.1f GF/s  probs=%d maxM=%lld maxN=%lld maxK=%lld perm=011 emu=%d "
            "packed\n",
            op->site.c_str(), ms, double(P->g.flops_mac) * c.ninst, 8.0 * double(P->g.flops_mac) * c.ninst / (ms * 1e6),
            P->g.n_probs, (long long)M, (long long)N, (long long)K, P->emulate);
  }
}

// A = integral <pq||rs> with (p, q) from table R and (r, s) from table K, made once:
// gathered from the full layout V(p q | r s) when it can be derived from a cached
// member of its family (src: the argument spaces; keep: cache that layout), drawn
// otherwise; B = T_P; C scattered into dst (rows Cr, cols oo)
static PackedOp* int_times_tau(Ctx& c, const std::string& site, const PairTable& R, const Tensor& dst, bool rows_packed,
                               double alpha, const IntRef* src = nullptr, bool keep = false) {
  PackedState& s = PS(c);
  auto it = s.ops.find(site);
  if (it != s.ops.end()) return it->second.get();
  PackedOp* op = new PackedOp();
  s.ops[site].reset(op);
  op->site = site;
  op->Ar = &R;
  op->Ac = s.vv;
  op->A = packed_tensor(c, R, *s.vv);
  op->dA = pack_dims(R, *s.vv);
  op->B = s.TP;
  op->Cr = &table(c, dst.L, true, rows_packed);
  op->Cc = &table(c, dst.L, false, true);
  op->C = arena_tensor(R, *s.oo);
  op->dC = pack_dims(*op->Cr, *op->Cc);
  bool made = false;
  if (src && &R != s.vv) {
    const int ident[4] = {0, 1, 2, 3};
    const Tensor* full = nullptr;
    Tensor* tmp = nullptr;
    if (keep) full = integral(c, *src, ident, 2);
    else full = tmp = integral_uncached(c, *src, ident, 2);
    if (full) {
      const PairTable& fr = table(c, full->L, true, rows_packed);
      const PairTable& fc = table(c, full->L, false, true);
      launch_pack_gather(c, op->A.d, op->A.is, full->d, full->is, pack_dims(fr, fc), fr, fc);
      made = true;
    }
    if (tmp) {
      CK(cudaStreamSynchronize(c.stream));
      c.dfree(tmp->d);
      delete tmp;
    }
  }
  if (!made) launch_generate_pairs(c, op->A.d, op->A.is, op->dA, R, *s.vv);
  finish_op(c, op, true, alpha);
  return op;
}

void packed_ladder(Ctx& c, Tensor& r2) {
  PackedState& s = PS(c);
  PackedOp* op = int_times_tau(c, "R2pp", *s.vv, r2, true, 1.0);
  run_op(c, op, [] {}, [&] { scatter_into(c, r2, op->C.d, op->C.is, op->dC, *op->Cr, *op->Cc); });
}

void packed_xamij(Ctx& c, Tensor& X) {
  const PairTable& am = table(c, X.L, true, false);
  static const IntRef VOVV{{SP_VIRT, SP_OCC, SP_VIRT, SP_VIRT}};
  PackedOp* op = int_times_tau(c, "Xamij", am, X, false, 2.0, &VOVV, false);  // sum_ef = 2 sum_{e<f}
  run_op(c, op, [] {}, [&] { launch_pack_scatter(c, X.d, X.is, op->C.d, op->C.is, op->dC, *op->Cr, *op->Cc, 1.0, false); });
}

void packed_wmnij(Ctx& c, Tensor& W) {
  const PairTable& mn = table(c, W.L, true, true);
  static const IntRef OOVV{{SP_OCC, SP_OCC, SP_VIRT, SP_VIRT}};
  PackedOp* op = int_times_tau(c, "Wmnij2", mn, W, true, 1.0, &OOVV, true);
  run_op(c, op, [] {}, [&] { launch_pack_scatter(c, W.d, W.is, op->C.d, op->C.is, op->dC, *op->Cr, *op->Cc, 1.0, true); });
}

// r2_ij^ab += sum_{m<n} T_P(ab, mn) W_mn,ij: A = T_P, B = W with rows m<n
void packed_hh(Ctx& c, const Tensor& W, Tensor& r2) {
  PackedState& s = PS(c);
  PackedOp* op;
  auto it = s.ops.find("R2hh");
  if (it == s.ops.end()) {
    op = new PackedOp();
    s.ops["R2hh"].reset(op);
    op->site = "R2hh";
    const PairTable& ijf = table(c, W.L, false, false);
    op->A = s.TP;
    op->Br = &table(c, W.L, true, true);  // (m, n), m < n: same enumeration as the tau columns
    op->Bc = &ijf;
    op->B = arena_tensor(*op->Br, ijf);
    op->offB = 0;
    op->dB = pack_dims(*op->Br, ijf);
    op->Cr = s.vv;
    op->Cc = &table(c, r2.L, false, false);
    op->C = arena_tensor(*s.vv, ijf);
    op->dC = pack_dims(*op->Cr, *op->Cc);
    finish_op(c, op, false);
  } else {
    op = it->second.get();
  }
  run_op(
      c, op, [&] { launch_pack_gather(c, op->B.d, op->B.is, W.d, W.is, op->dB, *op->Br, *op->Bc); },
      [&] { scatter_into(c, r2, op->C.d, op->C.is, op->dC, *op->Cr, *op->Cc); });
}

void packed_release(Ctx& c) {
  delete (PackedState*)c.packed_state;  // device memory belongs to the context's allocator
  c.packed_state = nullptr;
}
