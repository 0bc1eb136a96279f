// Host-side planning for symmetry-blocked tensors: layouts (DPD blocks,
// Sec. II.C), sub-block enumeration, permute plans and the TTGT einsum
// planner (Sec. II.B: permute operands into supermatrices, one grouped GEMM
// over all symmetry blocks (Fig. "mult"), permute the result back).
#include <algorithm>
#include <cstring>
#include <cstdio>
#include <sstream>

#include "engine.h"
#include "emu.h"
#include "packed.h"

static int64_t ipow(int G, int k) {
  int64_t r = 1;
  while (k-- > 0) r *= G;
  return r;
}
static inline int imod(int a, int G) { return ((a % G) + G) % G; }

std::string Layout::key() const {
  std::ostringstream s;
  s << rank << ":" << nrow << ":";
  for (int k = 0; k < rank; ++k) s << sp[k] << (sg[k] > 0 ? '+' : '-');
  return s.str();
}

void build_layout(Layout& L, const std::vector<Space>& S, int G) {
  L.G = G;
  const int nr = L.nrow, nc = L.rank - L.nrow;
  L.rows.assign(G, 0);
  L.cols.assign(G, 0);
  const int64_t NR = ipow(G, nr), NC = ipow(G, nc);
  L.rtup.assign(NR, 0);
  L.ctup.assign(NC, 0);
  for (int64_t code = 0; code < NR; ++code) {
    int64_t c = code;
    int irr[EXP_MAX_RANK] = {0, 0, 0, 0};
    for (int k = nr - 1; k >= 0; --k) { irr[k] = int(c % G); c /= G; }
    int sum = 0;
    int64_t sz = 1;
    for (int k = 0; k < nr; ++k) { sum += L.sg[k] * irr[k]; sz *= S[L.sp[k]].cnt[irr[k]]; }
    const int g = imod(sum, G);
    L.rtup[code] = L.rows[g];
    L.rows[g] += sz;
  }
  for (int64_t code = 0; code < NC; ++code) {
    int64_t c = code;
    int irr[EXP_MAX_RANK] = {0, 0, 0, 0};
    for (int k = nc - 1; k >= 0; --k) { irr[k] = int(c % G); c /= G; }
    int sum = 0;
    int64_t sz = 1;
    for (int k = 0; k < nc; ++k) { sum += L.sg[nr + k] * irr[k]; sz *= S[L.sp[nr + k]].cnt[irr[k]]; }
    const int g = imod(-sum, G);
    L.ctup[code] = L.cols[g];
    L.cols[g] += sz;
  }
  L.blk_off.assign(G, 0);
  int64_t off = 0;
  for (int g = 0; g < G; ++g) { L.blk_off[g] = off; off += L.rows[g] * L.cols[g]; }
  L.size = off;
}

Layout make_layout(const std::vector<Space>& S, int G, int rank, const int* sp, const int* sg,
                   int nrow) {
  Layout L;
  L.rank = rank;
  L.nrow = nrow;
  for (int k = 0; k < rank; ++k) { L.sp[k] = sp[k]; L.sg[k] = sg[k]; }
  build_layout(L, S, G);
  return L;
}

int64_t layout_count(const Layout& L, const std::vector<Space>&) { return L.size; }

// Every allowed sub-block, in tuple-code order.  Dims are padded to 4 with the
// padding in front (dim 3 is always the innermost storage slot).
void enumerate_blocks(const Layout& L, const std::vector<Space>& S, std::vector<SubBlock>& out) {
  const int G = L.G, r = L.rank, nr = L.nrow;
  out.clear();
  const int64_t NT = ipow(G, r);
  for (int64_t code = 0; code < NT; ++code) {
    int64_t c = code;
    int irr[EXP_MAX_RANK] = {0, 0, 0, 0};
    for (int k = r - 1; k >= 0; --k) { irr[k] = int(c % G); c /= G; }
    int sum = 0, rsum = 0;
    for (int k = 0; k < r; ++k) {
      sum += L.sg[k] * irr[k];
      if (k < nr) rsum += L.sg[k] * irr[k];
    }
    if (imod(sum, G) != 0) continue;
    SubBlock b;
    int64_t cnt = 1;
    for (int k = 0; k < r; ++k) { b.irr[k] = irr[k]; b.n[k] = S[L.sp[k]].cnt[irr[k]]; cnt *= b.n[k]; }
    for (int k = r; k < EXP_MAX_RANK; ++k) { b.irr[k] = 0; b.n[k] = 1; }
    b.count = cnt;
    const int g = imod(rsum, G);
    int64_t rcode = 0, ccode = 0;
    for (int k = 0; k < nr; ++k) rcode = rcode * G + irr[k];
    for (int k = nr; k < r; ++k) ccode = ccode * G + irr[k];
    b.base = L.blk_off[g] + L.rtup[rcode] * L.cols[g] + L.ctup[ccode];
    int64_t s = 1;
    for (int k = r - 1; k >= nr; --k) { b.st[k] = s; s *= b.n[k]; }
    s = L.cols[g];
    for (int k = nr - 1; k >= 0; --k) { b.st[k] = s; s *= b.n[k]; }
    for (int k = r; k < EXP_MAX_RANK; ++k) b.st[k] = 0;
    out.push_back(b);
  }
}

static const int64_t kChunk = EXP_CHUNK;

static void add_chunks(std::vector<ChunkRef>& chunks, int task, int64_t count) {
  for (int64_t s = 0; s < count; s += kChunk) chunks.push_back(ChunkRef{task, 0, s});
}

void* Ctx::dalloc(size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = alloc.alloc(bytes, alloc.user);
  if (!p) throw ExpError{EXP_ENOMEM, "allocator returned NULL for " + std::to_string(bytes) + " bytes"};
  owned.push_back(DevBuf{p, bytes});
  return p;
}

void Ctx::dfree(void* p) {
  for (size_t k = 0; k < owned.size(); ++k)
    if (owned[k].p == p) {
      alloc.free(p, alloc.user);
      owned.erase(owned.begin() + k);
      return;
    }
}

void* arena_reserve(Ctx& c, Arena& a, size_t bytes) {
  if (bytes <= a.bytes) return a.base;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(c.stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) throw ExpError{EXP_ESTATE, "scratch arena would grow during stream capture"};
  if (a.base) {
    CK(cudaStreamSynchronize(c.stream));  // work queued on the old region must finish first
    c.dfree(a.base);
    a.base = nullptr;
    a.bytes = 0;
  }
  a.base = c.dalloc(bytes);
  a.bytes = bytes;
  return a.base;
}

void Ctx::dfree_all() {
  for (auto& b : owned) alloc.free(b.p, alloc.user);
  owned.clear();
}

void upload(Ctx& c, void* dst, const void* src, size_t bytes) {
  if (!bytes) return;
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c.stream));
  // host buffers are temporaries: make the copy complete before they go away
  CK(cudaStreamSynchronize(c.stream));
}

void upload_async(Ctx& c, void* dst, const void* src, size_t bytes) {
  if (!bytes) return;
  Ctx::Staging& s = c.stg;
  if (!s.host[0]) {
    const size_t cap = size_t(32) << 20;
    for (int h = 0; h < 2; ++h) {
      CK(cudaMallocHost((void**)&s.host[h], cap));
      CK(cudaEventCreateWithFlags(&s.ev[h], cudaEventDisableTiming));
    }
    s.cap = cap;
  }
  if (bytes > s.cap / 4) {
    upload(c, dst, src, bytes);
    return;
  }
  if (s.used + bytes > s.cap) {  // this half is full: the other one, once its copies have run
    CK(cudaEventRecord(s.ev[s.cur], c.stream));
    s.pending[s.cur] = true;
    s.cur ^= 1;
    s.used = 0;
    if (s.pending[s.cur]) {
      CK(cudaEventSynchronize(s.ev[s.cur]));
      s.pending[s.cur] = false;
    }
  }
  uint8_t* h = s.host[s.cur] + s.used;
  memcpy(h, src, bytes);
  CK(cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, c.stream));
  s.used += (bytes + 255) & ~size_t(255);
}

void staging_release(Ctx& c) {
  Ctx::Staging& s = c.stg;
  for (int h = 0; h < 2; ++h) {
    if (s.host[h]) cudaFreeHost(s.host[h]);
    if (s.ev[h]) cudaEventDestroy(s.ev[h]);
    s.host[h] = nullptr;
    s.ev[h] = nullptr;
    s.pending[h] = false;
  }
  s.cap = s.used = 0;
}

Tensor* new_tensor(Ctx& c, const Layout& L, bool zero) {
  Tensor* t = new Tensor();
  t->L = L;
  const size_t bytes = sizeof(cplx) * size_t(std::max<int64_t>(L.size, 1)) * c.ninst;
  t->d = (cplx*)c.dalloc(bytes);
  t->is = std::max<int64_t>(L.size, 1);
  if (zero) CK(cudaMemsetAsync(t->d, 0, bytes, c.stream));
  return t;
}

Tensor* work_tensor(Ctx& c, const std::string& name, const Layout& L) {
  auto it = c.work.find(name);
  if (it != c.work.end()) return it->second.get();
  Tensor* t = new_tensor(c, L, true);
  c.work[name].reset(t);
  return t;
}

void gen_tasks(Ctx& c, const Layout& L, std::vector<GenTask>& tasks, std::vector<ChunkRef>& chunks) {
  std::vector<SubBlock> sb;
  enumerate_blocks(L, c.spaces, sb);
  const int r = L.rank, pad = EXP_MAX_RANK - r;
  for (auto& b : sb) {
    if (b.count == 0) continue;
    GenTask t;
    t.base = b.base;
    t.count = b.count;
    for (int d = 0; d < EXP_MAX_RANK; ++d) { t.n[d] = 1; t.st[d] = 0; t.g0[d] = 0; }
    for (int k = 0; k < r; ++k) {
      const Space& s = c.spaces[L.sp[k]];
      t.n[pad + k] = b.n[k];
      t.st[pad + k] = b.st[k];
      t.g0[pad + k] = s.gbase + s.off[b.irr[k]];
    }
    add_chunks(chunks, int(tasks.size()), t.count);
    tasks.push_back(t);
  }
}

// Integral tensors: V(p,q,r,s) generated directly in the requested storage
// order (slot k holds V argument arg[k]) and row/column split; cached.
static PermPlan make_perm_plan(Ctx& c, const Layout& D, const char* dl, const Layout& S, const char* sl,
                               const std::vector<std::string>& terms, bool check_signs = true,
                               bool canon = false);

// The exact symmetries of the integrals (the recipe antisymmetrises both pairs and
// Hermitises): V(x0 x1 x2 x3) = coef [conj] V(y) with y[pi[k]] = x_k.
struct VSym {
  int pi[4];
  double coef;
  bool conj;
};
static const VSym kVSym[8] = {
    {{0, 1, 2, 3}, 1.0, false},  {{1, 0, 2, 3}, -1.0, false}, {{0, 1, 3, 2}, -1.0, false},
    {{1, 0, 3, 2}, 1.0, false},  {{2, 3, 0, 1}, 1.0, true},   {{3, 2, 0, 1}, -1.0, true},
    {{2, 3, 1, 0}, -1.0, true},  {{3, 2, 1, 0}, 1.0, true}};

// A cached layout related by a symmetry of V: one permute instead of generating (the
// generator draws eight Gaussians per element; the values are the same).  nullptr when
// no member of the family is cached.
static Tensor* derive_integral(Ctx& c, const IntRef& v, const int arg[4], const Layout& L) {
  for (const auto& m : c.int_list) {
    for (const VSym& y : kVSym) {
      bool ok = true;
      for (int k = 0; k < 4; ++k) ok = ok && v.sp[k] == m.vsp[y.pi[k]];
      if (!ok) continue;
      const char* lab = "abcd";  // labels of the new V arguments
      char dl[5] = {0}, sl[5] = {0};
      for (int s2 = 0; s2 < 4; ++s2) {
        dl[s2] = lab[arg[s2]];
        for (int k = 0; k < 4; ++k)
          if (y.pi[k] == m.arg[s2]) sl[s2] = lab[k];
      }
      Tensor* t = new_tensor(c, L, false);
      PermPlan pp = make_perm_plan(c, L, dl, m.t->L, sl, {std::string(dl)}, !y.conj);
      const cplx coef = make_double2(y.coef, 0.0);
      launch_permute(c, pp, t->d, m.t->d, t->is, m.t->is, &coef, false, y.conj);
      return t;
    }
  }
  return nullptr;
}

Tensor* integral_uncached(Ctx& c, const IntRef& v, const int arg[4], int nrow) {
  int sp[4], sg[4];
  for (int k = 0; k < 4; ++k) {
    sp[k] = v.sp[arg[k]];
    sg[k] = arg[k] < 2 ? 1 : -1;
  }
  Layout L = make_layout(c.spaces, c.G, 4, sp, sg, nrow);
  return derive_integral(c, v, arg, L);
}

// V(p q | r s) in argument order with nrow 2, drawn with each same-space pair of one
// compound packed (p<q or r<s: the other half follows by antisymmetry) and scattered
// into the full layout with the swap signs
static Tensor* generate_packed_pairs(Ctx& c, const int cs[4]) {
  const int sg[4] = {1, 1, -1, -1};
  Layout L = make_layout(c.spaces, c.G, 4, cs, sg, 2);
  PairTable R, C;
  build_pair_table(c, L, true, cs[0] == cs[1], R);
  build_pair_table(c, L, false, cs[2] == cs[3], C);
  const PackDims D = pack_dims(R, C);
  const int64_t n = std::max<int64_t>(D.blk[D.G], 1);
  cplx* P = (cplx*)c.dalloc(sizeof(cplx) * n * c.ninst);
  launch_generate_pairs(c, P, n, D, R, C);
  Tensor* t = new_tensor(c, L, false);
  launch_pack_scatter(c, t->d, t->is, P, n, D, R, C, 1.0, false);
  CK(cudaStreamSynchronize(c.stream));  // the temporaries are released below
  c.dfree(P);
  for (PairTable* T : {&R, &C}) {
    c.dfree(T->d_pair);
    c.dfree(T->d_full);
    c.dfree(T->d_inv);
  }
  return t;
}

static std::string int_key(const int sp[4], const int arg[4], int nrow) {
  std::ostringstream key;
  key << sp[0] << sp[1] << sp[2] << sp[3] << "|" << arg[0] << arg[1] << arg[2] << arg[3] << "|" << nrow;
  return key.str();
}

const Tensor* integral(Ctx& c, const IntRef& v, const int arg[4], int nrow) {
  std::ostringstream key;
  key << int_key(v.sp, arg, nrow);
  auto it = c.int_cache.find(key.str());
  if (it != c.int_cache.end()) return it->second.get();
  if (!c.have_integrals) throw ExpError{EXP_ESTATE, "integrals requested before exp_init_integrals"};
  // the first layout of a symmetry family: when an orientation V(p q | r s) of the
  // family has a same-space pair in one compound, draw that one packed and derive
  // the requested layout from it (below).  Before the scale is final only a request
  // that is itself that orientation is drawn this way (it gets rescaled in place).
  {
    bool family = false;
    for (const auto& m : c.int_list)
      for (const VSym& y : kVSym) {
        bool ok = true;
        for (int k = 0; k < 4; ++k) ok = ok && v.sp[k] == m.vsp[y.pi[k]];
        family = family || ok;
      }
    if (!family) {
      int best = -1, best_score = 0, cs[4] = {0, 0, 0, 0};
      for (int y = 0; y < 8; ++y) {
        int img[4];
        for (int k = 0; k < 4; ++k) img[kVSym[y].pi[k]] = v.sp[k];
        const int score = (img[0] == img[1]) + (img[2] == img[3]);
        if (score > best_score) {
          best_score = score;
          best = y;
          for (int k = 0; k < 4; ++k) cs[k] = img[k];
        }
      }
      const int ident[4] = {0, 1, 2, 3};
      const bool is_canon = best == 0 && nrow == 2 && arg[0] == 0 && arg[1] == 1 && arg[2] == 2 && arg[3] == 3;
      if (best >= 0 && (c.integrals_scaled || is_canon)) {
        Tensor* t = generate_packed_pairs(c, cs);
        c.int_cache[int_key(cs, ident, 2)].reset(t);
        c.int_list.push_back({{cs[0], cs[1], cs[2], cs[3]}, {0, 1, 2, 3}, t});
        if (is_canon) return t;
      }
    }
  }
  int sp[4], sg[4], map[4];
  for (int k = 0; k < 4; ++k) {
    sp[k] = v.sp[arg[k]];
    sg[k] = arg[k] < 2 ? 1 : -1;
    map[arg[k]] = k;
  }
  Layout L = make_layout(c.spaces, c.G, 4, sp, sg, nrow);
  if (Tensor* t = derive_integral(c, v, arg, L)) {
    c.int_cache[key.str()].reset(t);
    c.int_list.push_back({{v.sp[0], v.sp[1], v.sp[2], v.sp[3]}, {arg[0], arg[1], arg[2], arg[3]}, t});
    return t;
  }
  Tensor* t = new_tensor(c, L, true);
  std::vector<GenTask> tasks;
  std::vector<ChunkRef> chunks;
  gen_tasks(c, L, tasks, chunks);
  if (!chunks.empty()) {
    GenTask* dt = (GenTask*)c.dalloc(tasks.size() * sizeof(GenTask));
    ChunkRef* dc = (ChunkRef*)c.dalloc(chunks.size() * sizeof(ChunkRef));
    upload(c, dt, tasks.data(), tasks.size() * sizeof(GenTask));
    upload(c, dc, chunks.data(), chunks.size() * sizeof(ChunkRef));
    launch_generate(c, t->d, t->is, dt, dc, int(chunks.size()), map);
  }
  c.int_cache[key.str()].reset(t);
  c.int_list.push_back({{v.sp[0], v.sp[1], v.sp[2], v.sp[3]}, {arg[0], arg[1], arg[2], arg[3]}, t});
  return t;
}

// ---------------------------------------------------------------------------
// Permute plans.  dst[dl] (+)= sum_t coef_t * src[sigma_t], where term t is a
// relabelling string ts (a permutation of dl): the src slot labelled l takes
// the value of the dst slot labelled sigma_t(l), sigma_t(dl[k]) = ts[k].
// canon: the destination is antisymmetric in slots (0, 1) and (2, 3) and only its
// canonical entries are written -- sub-blocks with irreps g0 <= g1 and g2 <= g3, and
// inside a block with g0 = g1 (g2 = g3) the elements with local index i0 < i1 (i2 < i3)
static PermPlan make_perm_plan(Ctx& c, const Layout& D, const char* dl, const Layout& S,
                               const char* sl, const std::vector<std::string>& terms, bool check_signs,
                               bool canon) {
  const int r = D.rank;
  if (S.rank != r) throw ExpError{EXP_EINVAL, "permute rank mismatch"};
  if (canon && (r != 4 || D.sp[0] != D.sp[1] || D.sg[0] != D.sg[1] || D.sp[2] != D.sp[3] || D.sg[2] != D.sg[3]))
    throw ExpError{EXP_EINVAL, "canonical-pairs permute: destination without two same-space pairs"};
  std::vector<SubBlock> db, sb;
  enumerate_blocks(D, c.spaces, db);
  enumerate_blocks(S, c.spaces, sb);
  const int G = c.G;
  std::vector<int> sidx(size_t(ipow(G, r)), -1);
  for (size_t k = 0; k < sb.size(); ++k) {
    int64_t code = 0;
    for (int s = 0; s < r; ++s) code = code * G + sb[k].irr[s];
    sidx[code] = int(k);
  }
  const int nt = int(terms.size());
  // pos[t][k]: dst position feeding src slot k under term t
  int pos[EXP_MAX_TERMS][EXP_MAX_RANK];
  for (int t = 0; t < nt; ++t) {
    const std::string& ts = terms[t];
    for (int k = 0; k < r; ++k) {
      // sigma(l) = ts[j] where dl[j] == l
      const char* pl = strchr(dl, sl[k]);
      if (!pl) throw ExpError{EXP_EINVAL, std::string("permute label missing: ") + sl[k]};
      const char target = ts[pl - dl];
      const char* pd = strchr(dl, target);
      if (!pd) throw ExpError{EXP_EINVAL, "bad permute term"};
      pos[t][k] = int(pd - dl);
      if ((check_signs && S.sg[k] != D.sg[pos[t][k]]) || S.sp[k] != D.sp[pos[t][k]])
        throw ExpError{EXP_EINVAL, "permute space/sign mismatch"};
    }
  }
  const int pad = EXP_MAX_RANK - r;
  std::vector<PermTask> tasks;
  std::vector<ChunkRef> chunks;
  for (auto& b : db) {
    if (b.count == 0) continue;
    if (canon && (b.irr[0] > b.irr[1] || b.irr[2] > b.irr[3])) continue;
    PermTask T;
    memset(&T, 0, sizeof(T));
    T.dst = b.base;
    T.count = b.count;
    if (canon) T.tri = (b.irr[0] == b.irr[1] ? 1 : 0) | (b.irr[2] == b.irr[3] ? 2 : 0);
    for (int d = 0; d < 4; ++d) { T.n[d] = 1; T.dst_st[d] = 0; }
    for (int k = 0; k < r; ++k) { T.n[pad + k] = b.n[k]; T.dst_st[pad + k] = b.st[k]; }
    for (int t = 0; t < nt; ++t) {
      int64_t code = 0;
      for (int k = 0; k < r; ++k) code = code * G + b.irr[pos[t][k]];
      const int si = sidx[code];
      if (si < 0) throw ExpError{EXP_EINVAL, "permute source block missing"};
      const SubBlock& s = sb[si];
      T.src[t] = s.base;
      for (int d = 0; d < 4; ++d) T.src_st[t][d] = 0;
      for (int k = 0; k < r; ++k) T.src_st[t][pad + pos[t][k]] = s.st[k];
    }
    if (T.count >= (int64_t(1) << 31)) throw ExpError{EXP_EINVAL, "permute sub-block above 2^31 elements"};
    for (int d = 0; d < 4; ++d) udiv_magic(uint32_t(T.n[d]), T.mg[d], T.ml[d]);
    add_chunks(chunks, int(tasks.size()), T.count);
    tasks.push_back(T);
  }
  PermPlan p;
  p.n_terms = nt;
  p.n_chunks = int(chunks.size());
  if (!tasks.empty()) {
    p.d_tasks = (PermTask*)c.dalloc(tasks.size() * sizeof(PermTask));
    p.d_chunks = (ChunkRef*)c.dalloc(chunks.size() * sizeof(ChunkRef));
    upload(c, p.d_tasks, tasks.data(), tasks.size() * sizeof(PermTask));
    upload(c, p.d_chunks, chunks.data(), chunks.size() * sizeof(ChunkRef));
  }
  return p;
}

static Layout relayout(Ctx& c, const Layout& S, const char* sl, const std::string& order, int nrow) {
  int sp[4], sg[4];
  const int r = int(order.size());
  for (int k = 0; k < r; ++k) {
    const char* p = strchr(sl, order[k]);
    sp[k] = S.sp[p - sl];
    sg[k] = S.sg[p - sl];
  }
  return make_layout(c.spaces, c.G, r, sp, sg, nrow);
}

static std::vector<std::string> term_strings(const char* dl,
                                             const std::vector<std::pair<double, std::string>>& terms,
                                             std::vector<double>& coefs) {
  std::vector<std::string> ts;
  coefs.clear();
  if (terms.empty()) {
    ts.push_back(dl);
    coefs.push_back(1.0);
  } else {
    for (auto& t : terms) { ts.push_back(t.second); coefs.push_back(t.first); }
  }
  if (ts.size() > EXP_MAX_TERMS) throw ExpError{EXP_EINVAL, "too many permute terms"};
  return ts;
}

void permute_into(Ctx& c, const std::string& site, Tensor& dst, const char* dl, const Tensor& src,
                  const char* sl, bool accumulate, std::vector<std::pair<double, std::string>> terms) {
  const bool canon = dst.pair_canon && c.canon_pairs;
  const std::string key = "P:" + site + (canon ? "|canon" : "");
  auto it = c.perm_cache.find(key);
  std::vector<double> coefs;
  auto ts = term_strings(dl, terms, coefs);
  if (it == c.perm_cache.end()) {
    PermPlan p = make_perm_plan(c, dst.L, dl, src.L, sl, ts, true, canon);
    it = c.perm_cache.emplace(key, p).first;
  }
  cplx co[EXP_MAX_TERMS];
  for (size_t k = 0; k < coefs.size(); ++k) co[k] = make_double2(coefs[k], 0.0);
  launch_permute(c, it->second, dst.d, src.d, dst.is, src.is, co, accumulate, false);
}

// ---------------------------------------------------------------------------
// TTGT einsum: C[cl] (+)= alpha * sum_K A[al] B[bl], optionally antisymmetrised
// on output by the relabelling terms.  Operands are permuted into the
// supermatrices A'(FA|K), B'(K|FB) unless they already are, integrals are
// generated in the needed layout once, and the product runs as one grouped GEMM
// over the symmetry blocks (all instances).
GemmPlan make_gemm_plan(Ctx& c, const Layout& A, const Layout& B, const Layout& C) {
  GemmPlan g;
  int64_t tiles_mn = 0;
  int64_t maxM = 0, maxN = 0;
  for (int q = 0; q < c.G; ++q) {
    if (A.rows[q] && B.cols[q]) { maxM = std::max<int64_t>(maxM, A.rows[q]); maxN = std::max<int64_t>(maxN, B.cols[q]); }
  }
  g.tm = maxM <= 16 ? 16 : 64;
  g.tn = maxN <= 16 ? 16 : 64;
  for (int q = 0; q < c.G; ++q) {
    const int64_t M = A.rows[q], K = A.cols[q], N = B.cols[q];
    if (B.rows[q] != K || C.rows[q] != M || C.cols[q] != N)
      throw ExpError{EXP_EINVAL, "gemm block shape mismatch"};
    if (M == 0 || N == 0) continue;
    GemmProb p{};
    p.a = A.blk_off[q];
    p.b = B.blk_off[q];
    p.c = C.blk_off[q];
    p.M = int32_t(M);
    p.N = int32_t(N);
    p.K = int32_t(K);
    p.tiles_n = int32_t((N + g.tn - 1) / g.tn);
    p.tiles_m = int32_t((M + g.tm - 1) / g.tm);
    p.ksplit = 1;
    p.kchunk = int32_t(((K + 7) / 8) * 8);
    tiles_mn += int64_t(p.tiles_m) * p.tiles_n;
    g.flops_mac += M * N * K;
    g.h_probs.push_back(p);
  }
  // matrix-vector products, and small ones whose K is long enough for the warp's lanes
  // to share or whose outputs are few: one warp per output element (a short K leaves
  // most lanes idle, which a batch of instances multiplies: those take the tiles)
  int64_t maxK = 0, outs = 0;
  for (const GemmProb& p : g.h_probs) {
    maxK = std::max<int64_t>(maxK, p.K);
    outs += int64_t(p.M) * p.N;
  }
  if (maxN <= 2 ||
      (g.flops_mac * c.ninst < (int64_t(1) << 22) && (maxK >= 32 || outs * c.ninst <= (int64_t(1) << 18)))) {
    int64_t o = 0;
    for (auto& p : g.h_probs) { p.ws = o; o += int64_t(p.M) * p.N; }
    g.dot_outputs = o;
    g.n_probs = int(g.h_probs.size());
    if (g.n_probs) {
      g.d_probs = (GemmProb*)c.dalloc(g.h_probs.size() * sizeof(GemmProb));
      upload(c, g.d_probs, g.h_probs.data(), g.h_probs.size() * sizeof(GemmProb));
    }
    return g;
  }
  // split K when the output tiles cannot fill the GPU (long-K, small-MN blocks)
  const int64_t want = 8LL * std::max(c.sm_count, 1);
  const int64_t have = tiles_mn * c.ninst;
  int tile0 = 0;
  int64_t ws = 0;
  for (auto& p : g.h_probs) {
    if (have < 2LL * std::max(c.sm_count, 1) && p.K >= 512) {
      int64_t ks = std::min<int64_t>((p.K + 255) / 256, (want + have - 1) / std::max<int64_t>(have, 1));
      ks = std::max<int64_t>(1, std::min<int64_t>(ks, 256));
      if (ks > 1) {
        p.kchunk = int32_t((((p.K + ks - 1) / ks) + 7) / 8 * 8);
        p.ksplit = int32_t((p.K + p.kchunk - 1) / p.kchunk);
      }
    }
    if (p.ksplit > 1) {
      p.ws = ws;
      ws += int64_t(p.ksplit) * p.M * p.N;
      g.red_elems += int64_t(p.M) * p.N;
    }
    p.tile0 = tile0;
    tile0 += p.tiles_m * p.tiles_n * p.ksplit;
  }
  g.n_probs = int(g.h_probs.size());
  g.n_tiles = tile0;
  if (ws) {
    g.ws_is = ws;
    g.d_ws = (cplx*)c.dalloc(sizeof(cplx) * ws * c.ninst);
  }
  if (g.n_probs) {
    g.d_probs = (GemmProb*)c.dalloc(g.h_probs.size() * sizeof(GemmProb));
    upload(c, g.d_probs, g.h_probs.data(), g.h_probs.size() * sizeof(GemmProb));
  }
  return g;
}

static const Tensor* prepare_operand(Ctx& c, const std::string& site, const Operand& op,
                                     const std::string& order, int nrow, Tensor& scratch,
                                     PermPlan& plan, bool& permuted) {
  permuted = false;
  if (op.v) {
    int arg[4];
    for (int k = 0; k < 4; ++k) {
      const char* p = strchr(op.labels, order[k]);
      arg[k] = int(p - op.labels);
    }
    return integral(c, *op.v, arg, nrow);
  }
  const Tensor* t = op.t;
  if (order == op.labels && t->L.nrow == nrow) return t;
  Layout L = relayout(c, t->L, op.labels, order, nrow);
  scratch.L = L;  // storage: the operand arena, placed by the caller
  scratch.is = std::max<int64_t>(L.size, 1);
  scratch.d = nullptr;
  std::vector<std::string> ts{order};
  plan = make_perm_plan(c, L, order.c_str(), t->L, op.labels, ts);
  permuted = true;
  return &scratch;
}

// product of the full space sizes of an operand's labels in F
static double free_extent(const Ctx& c, const Operand& op, const std::string& F) {
  double d = 1.0;
  for (char x : F) {
    const char* p = strchr(op.labels, x);
    if (!p) continue;
    const int k = int(p - op.labels);
    const int sp = op.v ? op.v->sp[k] : op.t->L.sp[k];
    d *= double(c.spaces[sp].n);
  }
  return d;
}

void einsum(Ctx& c, const std::string& site, cplx alpha, Operand A, Operand B, Tensor& C,
            const char* cl, bool accumulate, std::vector<std::pair<double, std::string>> terms) {
  auto it = c.plans.find(site);
  EinsumPlan* P;
  if (it == c.plans.end()) {
    P = new EinsumPlan();
    c.plans[site].reset(P);
    const std::string clab = cl;
    std::string K, FA, FB;
    auto split_labels = [&]() {
      const std::string al = A.labels, bl = B.labels;
      K.clear();
      FA.clear();
      FB.clear();
      for (char x : al)
        if (bl.find(x) != std::string::npos && clab.find(x) == std::string::npos) K += x;
      for (char x : al)
        if (K.find(x) == std::string::npos) FA += x;
      for (char x : bl)
        if (K.find(x) == std::string::npos) FB += x;
      // when each operand holds exactly one side of the output compound, take its free
      // labels in the output's order: the GEMM then writes the destination directly.
      // Only where that adds no operand permute: an integral is generated in any
      // layout, a tensor only if it is permuted anyway.
      auto same_set = [](std::string a, std::string b) {
        std::sort(a.begin(), a.end());
        std::sort(b.begin(), b.end());
        return a == b;
      };
      auto in_place = [](const Operand& op, const std::string& ord, int nrow) {
        return op.t && std::string(op.labels) == ord && op.t->L.nrow == nrow;
      };
      if (terms.empty() && FA.size() + FB.size() == clab.size() && C.L.nrow == int(FA.size()) &&
          same_set(FA, clab.substr(0, FA.size())) && same_set(FB, clab.substr(FA.size()))) {
        const std::string FA2 = clab.substr(0, FA.size()), FB2 = clab.substr(FA.size());
        const bool okA = FA2 == FA || A.v || !in_place(A, FA + K, int(FA.size()));
        const bool okB = FB2 == FB || B.v || !in_place(B, K + FB, int(K.size()));
        if (okA && okB) {
          FA = FA2;
          FB = FB2;
        }
      }
    };
    split_labels();
    if (FA.size() + FB.size() != clab.size()) throw ExpError{EXP_EINVAL, "einsum labels: " + site};
    // The emulated GEMM slices its A operand into half the bytes of B (B'' holds
    // every element twice), so when the output goes through a permute anyway the
    // operand with the larger free extent takes the A role (C^T = B^T A^T).
    if (c.cfg.precision == EXP_EMU_BF16) {
      const bool identity0 = terms.empty() && FA + FB == clab && C.L.nrow == int(FA.size());
      const double ea = free_extent(c, A, FA), eb = free_extent(c, B, FB);
      // a small output over a long contraction, integral times amplitudes: the
      // amplitudes (sliced every iteration) go to A, the integral (sliced once) to B
      const bool small_out = A.v && B.t && ea <= 64.0 && eb <= 64.0;
      // (a direct write is given up only for a tiny output, where the permute is free)
      if ((!identity0 && eb > 2.0 * ea) || (small_out && (!identity0 || C.L.size <= (1 << 16)))) {
        std::swap(A, B);
        split_labels();
        P->swapped = true;
      }
    }
    // contracted labels must meet with opposite signs
    const std::string ordA = FA + K, ordB = K + FB;
    const Tensor* Ap = prepare_operand(c, site, A, ordA, int(FA.size()), P->A2, P->pA, P->permA);
    const Tensor* Bp = prepare_operand(c, site, B, ordB, int(K.size()), P->B2, P->pB, P->permB);
    for (size_t k = 0; k < K.size(); ++k) {
      if (Ap->L.sg[FA.size() + k] != -Bp->L.sg[k] || Ap->L.sp[FA.size() + k] != Bp->L.sp[k])
        throw ExpError{EXP_EINVAL, "einsum contracted label sign/space mismatch: " + site};
    }
    P->A = A.v ? Ap : (P->permA ? &P->A2 : A.t);
    P->B = B.v ? Bp : (P->permB ? &P->B2 : B.t);
    // result supermatrix C'(FA|FB)
    const std::string ordC = FA + FB;
    std::vector<double> coefs;
    auto ts = term_strings(cl, terms, coefs);
    const bool identity = terms.empty() && ordC == clab && C.L.nrow == int(FA.size());
    if (identity) {
      P->permC = false;
      P->gemm_beta = accumulate;
      P->g = make_gemm_plan(c, P->A->L, P->B->L, C.L);
    } else {
      int sp[4], sg[4];
      for (size_t k = 0; k < FA.size(); ++k) { sp[k] = P->A->L.sp[k]; sg[k] = P->A->L.sg[k]; }
      for (size_t k = 0; k < FB.size(); ++k) {
        sp[FA.size() + k] = P->B->L.sp[K.size() + k];
        sg[FA.size() + k] = P->B->L.sg[K.size() + k];
      }
      Layout LC = make_layout(c.spaces, c.G, int(ordC.size()), sp, sg, int(FA.size()));
      P->C2.L = LC;  // storage: the operand arena
      P->C2.is = std::max<int64_t>(LC.size, 1);
      P->C2.d = nullptr;
      P->permC = true;
      P->gemm_beta = false;
      P->g = make_gemm_plan(c, P->A->L, P->B->L, LC);
      // output permute: C[cl] (+)= sum coef * C'[ordC relabelled]
      P->pC = make_perm_plan(c, C.L, cl, LC, ordC.c_str(), ts);
      if (C.pair_canon) P->pCc = make_perm_plan(c, C.L, cl, LC, ordC.c_str(), ts, true, true);
    }
    for (size_t k = 0; k < coefs.size(); ++k) P->cterms[k] = make_double2(coefs[k], 0.0);
    P->alpha = alpha;
    {  // A2 | B2 | C2 side by side in the operand arena
      int64_t off = 0;
      if (P->permA) { P->offA2 = off; off += P->A2.is * c.ninst; }
      if (P->permB) { P->offB2 = off; off += P->B2.is * c.ninst; }
      if (P->permC) { P->offC2 = off; off += P->C2.is * c.ninst; }
      arena_reserve(c, c.op_arena, size_t(off) * sizeof(cplx));
    }
    P->emulate = emu_wanted(c, P->g, site);
    if (P->emulate && ds_wanted(c, P->g)) {  // short K: double-single SIMT instead of slices
      P->emulate = false;
      P->ds = true;
      ds_prepare(c, P->g);
    }
    // a B operand in the arena is not a tensor other contractions could share slices of
    if (P->emulate) P->emu = emu_plan(c, P->g, P->A, P->B, A.v != nullptr, B.v != nullptr, !P->permB, site);
  } else {
    P = it->second.get();
    if (P->swapped) std::swap(A, B);
  }
  // execute
  const bool prof = c.profile;
  cudaEvent_t pe[4] = {nullptr, nullptr, nullptr, nullptr};
  if (prof) {
    for (auto& e : pe) CK(cudaEventCreate(&e));
    CK(cudaEventRecord(c.pev0, c.stream));
  }
  {
    cplx* ab = (cplx*)c.op_arena.base;
    if (P->permA) P->A2.d = ab + P->offA2;
    if (P->permB) P->B2.d = ab + P->offB2;
    if (P->permC) P->C2.d = ab + P->offC2;
  }
  if (P->permA) {
    cplx one = make_double2(1, 0);
    launch_permute(c, P->pA, P->A2.d, A.t->d, P->A2.is, A.t->is, &one, false, false);
  }
  if (P->permB) {
    cplx one = make_double2(1, 0);
    launch_permute(c, P->pB, P->B2.d, B.t->d, P->B2.is, B.t->is, &one, false, false);
  }
  Tensor* Cg = P->permC ? &P->C2 : &C;
  P->gemm_out = Cg->d;
  P->gemm_out_is = Cg->is;
  if (prof) CK(cudaEventRecord(pe[0], c.stream));
  if (P->emulate)
    emu_run(c, P->emu, P->g, P->A->d, P->B->d, Cg->d, P->A->is, P->B->is, Cg->is, alpha,
            P->gemm_beta);
  else if (P->ds)
    launch_gemm_ds(c, P->g, P->A->d, P->B->d, Cg->d, P->A->is, P->B->is, Cg->is, alpha, P->gemm_beta);
  else
    launch_gemm_fp64(c, P->g, P->A->d, P->B->d, Cg->d, P->A->is, P->B->is, Cg->is, alpha,
                     P->gemm_beta);
  if (prof) CK(cudaEventRecord(pe[1], c.stream));
  if (P->permC)
    launch_permute(c, (C.pair_canon && c.canon_pairs) ? P->pCc : P->pC, C.d, P->C2.d, C.is, P->C2.is, P->cterms,
                   accumulate, false);
  if (prof) {
    CK(cudaEventRecord(c.pev1, c.stream));
    CK(cudaEventSynchronize(c.pev1));
    float ms = 0.f, m_in = 0.f, m_g = 0.f, m_out = 0.f;
    CK(cudaEventElapsedTime(&ms, c.pev0, c.pev1));
    CK(cudaEventElapsedTime(&m_in, c.pev0, pe[0]));
    CK(cudaEventElapsedTime(&m_g, pe[0], pe[1]));
    CK(cudaEventElapsedTime(&m_out, pe[1], c.pev1));
    for (auto& e : pe)
      if (e) cudaEventDestroy(e);
    fprintf(stderr, "[exp_phase] %-8s in %7.3f  gemm %7.3f  out %7.3f ms\n", site.c_str(), m_in, m_g, m_out);
    int64_t M = 0, N = 0, K = 0;
    for (auto& q : P->g.h_probs) { M = std::max<int64_t>(M, q.M); N = std::max<int64_t>(N, q.N); K = std::max<int64_t>(K, q.K); }
    fprintf(stderr, "[exp_profile] %-8s %9.3f ms  %10.3g cMAC  %7.1f GF/s  probs=%d maxM=%lld maxN=%lld maxK=%lld perm=%d%d%d emu=%d%s\n",
            site.c_str(), ms, double(P->g.flops_mac) * c.ninst,
            8.0 * double(P->g.flops_mac) * c.ninst / (ms * 1e6), P->g.n_probs, (long long)M, (long long)N,
            (long long)K, P->permA, P->permB, P->permC, P->emulate, P->ds ? " ds" : "");
  }
}
