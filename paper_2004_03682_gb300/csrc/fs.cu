// The (0h,1p) Fock-space sector (Eq. (sectors); H_eff = (H Omega)_Cl, Sec. II.A;
// flowchart steps II-V, Sec. II.B).  With T converged, the Bloch equation
//     Q Hbar (P + S) = S H_eff,   H_eff = P Hbar (P + S)
// is iterated as s <- s + (Q Hbar (P+S) - S H_eff)/D.  Hbar (P+S) for all active
// spinors is one CCSD residual evaluation: every active x owns a ghost occupied
// spinor g_x (orbital energy 0, no integrals) whose amplitudes t_{g_x}^a,
// t_{g_x j}^{ab} hold the column (P+S)_x, and the residual's ghost projections
// are (Hbar_N - E_CC)(P+S)_x.  S H_eff is two small contractions over the ghost
// index (the same TTGT engine).  H_eff is diagonalised per irrep block on the
// device (Hessenberg reduction + Wilkinson-shifted QR, complex FP64).
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <map>

#include "ccsd.h"
#include "fs.h"

// ROLE_MIRROR: a copy of an unknown under the antisymmetry of t2, written from its canonical
// element after every step
enum : int8_t { ROLE_REAL = 0, ROLE_Q = 1, ROLE_P = 2, ROLE_ZERO = 3, ROLE_MIRROR = 4 };

struct HPair {
  int64_t src;   // offset of t1(a = act[y], i = g_x) in the amplitude vector
  int64_t dst;   // offset of Hg(m = g_y, i = g_x)
  int32_t dense; // y * nact + x
  int32_t pad;
};

struct FsState {
  int8_t* d_role = nullptr;   // [namp]
  double* d_Dfs = nullptr;    // [ninst][namp]
  cplx* d_XV = nullptr;       // [ninst][namp]: S H_eff, t1 then t2 part
  Tensor Hg, X1, X2;
  HPair* d_pairs = nullptr;
  int n_pairs = 0;
  cplx* d_heff = nullptr;     // [ninst][nact][nact]
  cplx* d_eig = nullptr;      // [ninst][nact]
  int* d_blk = nullptr;       // active slots grouped by irrep
  int* d_blk_off = nullptr;   // [G + 1]
  bool done = false;
  bool converged = false;
  int n_iter = 0;
  std::vector<cplx> h_heff, h_eig;
  void* fs2 = nullptr;  // the (0h,2p) sector's state (Fs2State, below)
  int64_t* d_mir = nullptr;  // mirrored copies of the one-ghost doubles
  int64_t n_mir = 0;
};

static FsState& F(Ctx& c) { return *reinterpret_cast<FsState*>(c.fs_state); }

static void fs2_release(FsState& s);

void fs_release(Ctx& c) {
  FsState* s = reinterpret_cast<FsState*>(c.fs_state);
  if (s) fs2_release(*s);
  delete s;
  c.fs_state = nullptr;
}

// roles over the t1 (a|i) and t2 (ab|ij) layouts
__global__ void k_fs_roles(int8_t* __restrict__ role, int64_t off, const GenTask* __restrict__ tasks,
                           const ChunkRef* __restrict__ chunks, int rank, int no, const int* __restrict__ ghost,
                           const int* __restrict__ actslot) {
  const ChunkRef ch = chunks[blockIdx.x];
  const GenTask T = tasks[ch.task];
  const int64_t end = min(ch.start + (int64_t)4096, T.count);
  for (int64_t e = ch.start + threadIdx.x; e < end; e += blockDim.x) {
    int64_t r = e;
    int i[4];
    i[3] = int(r % T.n[3]); r /= T.n[3];
    i[2] = int(r % T.n[2]); r /= T.n[2];
    i[1] = int(r % T.n[1]);
    i[0] = int(r / T.n[1]);
    const int64_t p = off + T.base + i[0] * T.st[0] + i[1] * T.st[1] + i[2] * T.st[2] + i[3] * T.st[3];
    int8_t ro;
    if (rank == 2) {  // (a, i) in dims 2, 3
      const int a = T.g0[2] + i[2] - no, k = ghost[T.g0[3] + i[3]];
      if (k < 0) ro = ROLE_REAL;
      else if (actslot[a] == k) ro = ROLE_P;
      else if (actslot[a] >= 0) ro = ROLE_ZERO;  // intermediate normalisation: s_x^y = 0
      else ro = ROLE_Q;
    } else {
      const int ki = ghost[T.g0[2] + i[2]], kj = ghost[T.g0[3] + i[3]];
      if (ki >= 0 && kj >= 0) ro = ROLE_ZERO;
      else if (ki >= 0 || kj >= 0) ro = ROLE_Q;
      else ro = ROLE_REAL;
    }
    role[p] = ro;
  }
}

// ghost amplitudes <- P (1 at t1(act[x], g_x)), 0 elsewhere
__global__ void k_fs_init(cplx* __restrict__ T, const int8_t* __restrict__ role, int64_t namp) {
  const int inst = blockIdx.y;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < namp; k += int64_t(gridDim.x) * blockDim.x) {
    const int8_t r = role[k];
    if (r == ROLE_P) T[inst * namp + k] = make_double2(1.0, 0.0);
    else if (r != ROLE_REAL) T[inst * namp + k] = make_double2(0.0, 0.0);
  }
}

// H_eff[y, x] = (Hbar (P+S))_x at active y = R - D0 t at t1(act[y], g_x)
__global__ void k_fs_heff(const HPair* __restrict__ pairs, int np, const cplx* __restrict__ R,
                          const double* __restrict__ D, const cplx* __restrict__ T, int64_t namp, cplx* __restrict__ Hg,
                          int64_t hg_is, cplx* __restrict__ heff, int nact, const int* __restrict__ state) {
  const int inst = blockIdx.y;
  if (state[inst * 4 + 2]) return;
  for (int k = threadIdx.x; k < np; k += blockDim.x) {
    const HPair P = pairs[k];
    const cplx r = R[inst * namp + P.src], t = T[inst * namp + P.src];
    const double d = D[inst * namp + P.src];
    const cplx s = make_double2(r.x - d * t.x, r.y - d * t.y);
    Hg[inst * hg_is + P.dst] = s;
    heff[int64_t(inst) * nact * nact + P.dense] = s;
  }
}

// Q elements: rho = (R - D0 t) - (S H_eff); t_new = t + rho / D_fs; error = rho / D_fs.
// Other elements keep their value (error 0).
__global__ void __launch_bounds__(256) k_fs_update(const cplx* __restrict__ R, const double* __restrict__ D0,
                                                   const double* __restrict__ Dfs, const cplx* __restrict__ X,
                                                   const int8_t* __restrict__ role, const cplx* __restrict__ T,
                                                   cplx* __restrict__ Tn, cplx* __restrict__ En, int64_t namp, int dim,
                                                   const int* __restrict__ state, double* __restrict__ part,
                                                   double shift, double ds, int dn) {
  __shared__ double sh[32];
  const int inst = blockIdx.y;
  const int* st = state + inst * 4;
  const int slot = dim > 0 ? (st[1] + 1) % dim : 0;
  const int64_t off = int64_t(inst) * namp;
  const int64_t soff = (int64_t(inst) * (dim > 0 ? dim : 1) + slot) * namp;
  double m = 0.0;
  if (!st[2]) {
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < namp; k += int64_t(gridDim.x) * blockDim.x) {
      const cplx t = T[off + k];
      cplx tn = t, e = make_double2(0.0, 0.0);
      if (role[k] == ROLE_Q) {
        const cplx r = R[off + k], x = X[off + k];
        const double d0 = D0[off + k], df0 = Dfs[off + k];
        // intruder-state shift (ds > 0): the shifted equations rho + (D - D~) s = 0,
        // stepped with 1/D~ (ds = 0: D~ = D, the plain Bloch equation)
        const double df = dyn_shift(df0, ds, dn), dd = df0 - df;
        const double rr = r.x - d0 * t.x - x.x + dd * t.x, ri = r.y - d0 * t.y - x.y + dd * t.y;
        // level shift away from zero in the denominator's sign: |D| grows by sigma,
        // the step shrinks, the fixed point (zero residual) stays
        const double q = 1.0 / (df < 0.0 ? df - shift : df + shift);
        e = make_double2(rr * q, ri * q);
        tn = make_double2(t.x + e.x, t.y + e.y);
        const double ae = fma(e.x, e.x, e.y * e.y);  // |e|^2: k_finalize_update takes the root
        m = (ae != ae || ae > m) ? ae : m;  // NaN-propagating max
      }
      Tn[soff + k] = tn;
      En[soff + k] = e;
    }
  }
  for (int o = 16; o; o >>= 1) {
    const double v = __shfl_xor_sync(0xffffffffu, m, o);
    m = (v != v || v > m) ? v : m;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (blockDim.x >> 5); ++k) m = (sh[k] != sh[k] || sh[k] > m) ? sh[k] : m;
    part[(inst * gridDim.x + blockIdx.x) * 8] = m;
  }
}

// ---------------------------------------------------------------------------
// Eigenvalues of the per-irrep blocks of H_eff: complex Hessenberg reduction by
// Givens rotations, then explicitly shifted QR steps (Wilkinson shift from the
// trailing 2x2 block) with deflation.  One thread per (instance, irrep block);
// blocks have at most EXP_FS_MAXB rows.
#define EXP_FS_MAXB 32
struct Cd {
  double re, im;
};
__device__ __forceinline__ Cd cadd(Cd a, Cd b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Cd csub(Cd a, Cd b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ Cd cmul(Cd a, Cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Cd cconj(Cd a) { return {a.re, -a.im}; }
__device__ __forceinline__ double cabs_(Cd a) { return hypot(a.re, a.im); }
__device__ __forceinline__ Cd cdiv(Cd a, Cd b) {
  const double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__device__ Cd csqrt_(Cd a) {
  const double r = cabs_(a);
  double x = sqrt(0.5 * (r + a.re)), y = sqrt(fmax(0.0, 0.5 * (r - a.re)));
  if (a.im < 0) y = -y;
  return {x, y};
}
// Givens rotation [c s; -conj(s) c] (c real) zeroing b in (a, b)
__device__ void givens(Cd a, Cd b, double& c, Cd& s) {
  const double na = cabs_(a), nb = cabs_(b);
  if (nb == 0.0) { c = 1.0; s = {0.0, 0.0}; return; }
  if (na == 0.0) { c = 0.0; s = cdiv(cconj(b), Cd{nb, 0.0}); return; }
  const double r = hypot(na, nb);
  c = na / r;
  const Cd ph = {a.re / na, a.im / na};  // a / |a|
  s = cmul(ph, cconj(Cd{b.re / r, b.im / r}));
}

__global__ void k_fs_eig(const cplx* __restrict__ heff, int nact, const int* __restrict__ blk,
                         const int* __restrict__ blk_off, int G, cplx* __restrict__ eig, int* __restrict__ err) {
  const int inst = blockIdx.x;
  const int g = threadIdx.x;
  if (g >= G) return;
  const int b0 = blk_off[g], n = blk_off[g + 1] - b0;
  if (n == 0) return;
  if (n > EXP_FS_MAXB) { atomicExch(err, 1); return; }
  Cd H[EXP_FS_MAXB][EXP_FS_MAXB];
  for (int r = 0; r < n; ++r)
    for (int q = 0; q < n; ++q) {
      const cplx v = heff[int64_t(inst) * nact * nact + blk[b0 + r] * nact + blk[b0 + q]];
      H[r][q] = {v.x, v.y};
    }
  // Hessenberg: zero H[r][k] for r > k + 1 with rotations in rows/cols (r-1, r)
  for (int k = 0; k < n - 2; ++k)
    for (int r = n - 1; r > k + 1; --r) {
      double c;
      Cd s;
      givens(H[r - 1][k], H[r][k], c, s);
      for (int q = 0; q < n; ++q) {  // rows: [c s; -conj(s) c]
        const Cd x = H[r - 1][q], y = H[r][q];
        H[r - 1][q] = cadd(Cd{c * x.re, c * x.im}, cmul(s, y));
        H[r][q] = csub(Cd{c * y.re, c * y.im}, cmul(cconj(s), x));
      }
      for (int q = 0; q < n; ++q) {  // columns: multiply by the adjoint
        const Cd x = H[q][r - 1], y = H[q][r];
        H[q][r - 1] = cadd(Cd{c * x.re, c * x.im}, cmul(cconj(s), y));
        H[q][r] = csub(Cd{c * y.re, c * y.im}, cmul(s, x));
      }
    }
  int hi = n - 1, iter = 0;
  double cs[EXP_FS_MAXB];
  Cd sn[EXP_FS_MAXB];
  while (hi > 0) {
    if (++iter > 100 * n) { atomicExch(err, 2); break; }
    const double tiny = 1e-15 * (cabs_(H[hi][hi]) + cabs_(H[hi - 1][hi - 1]));
    if (cabs_(H[hi][hi - 1]) <= tiny) { H[hi][hi - 1] = {0, 0}; --hi; iter = 0; continue; }
    int lo = hi - 1;
    while (lo > 0 && cabs_(H[lo][lo - 1]) > 1e-15 * (cabs_(H[lo][lo]) + cabs_(H[lo - 1][lo - 1]))) --lo;
    // Wilkinson shift: eigenvalue of the trailing 2x2 closer to H[hi][hi]
    const Cd a = H[hi - 1][hi - 1], b = H[hi - 1][hi], cc = H[hi][hi - 1], d = H[hi][hi];
    const Cd tr = cadd(a, d), det = csub(cmul(a, d), cmul(b, cc));
    const Cd half = {0.5 * tr.re, 0.5 * tr.im};
    const Cd disc = csqrt_(csub(cmul(half, half), det));
    const Cd l1 = cadd(half, disc), l2 = csub(half, disc);
    Cd mu = cabs_(csub(l1, d)) < cabs_(csub(l2, d)) ? l1 : l2;
    if (iter % 11 == 10) mu = cadd(mu, Cd{cabs_(H[hi][hi - 1]), 0.0});  // exceptional shift
    for (int k = lo; k <= hi; ++k) H[k][k] = csub(H[k][k], mu);
    for (int k = lo; k < hi; ++k) {  // QR: rotations on rows k, k+1
      givens(H[k][k], H[k + 1][k], cs[k], sn[k]);
      for (int q = k; q < n; ++q) {
        const Cd x = H[k][q], y = H[k + 1][q];
        H[k][q] = cadd(Cd{cs[k] * x.re, cs[k] * x.im}, cmul(sn[k], y));
        H[k + 1][q] = csub(Cd{cs[k] * y.re, cs[k] * y.im}, cmul(cconj(sn[k]), x));
      }
    }
    for (int k = lo; k < hi; ++k)  // RQ: the adjoint rotations on columns k, k+1
      for (int q = 0; q <= min(k + 2, hi); ++q) {
        const Cd x = H[q][k], y = H[q][k + 1];
        H[q][k] = cadd(Cd{cs[k] * x.re, cs[k] * x.im}, cmul(cconj(sn[k]), y));
        H[q][k + 1] = csub(Cd{cs[k] * y.re, cs[k] * y.im}, cmul(sn[k], x));
      }
    for (int k = lo; k <= hi; ++k) H[k][k] = cadd(H[k][k], mu);
  }
  for (int r = 0; r < n; ++r) eig[int64_t(inst) * nact + b0 + r] = make_double2(H[r][r].re, H[r][r].im);
}

// copies of the canonical unknowns: Tn[dst] = +-Tn[src] in the slot k_fs_update wrote
__global__ void k_fs_mirror(const int64_t* __restrict__ mir, int64_t n, cplx* __restrict__ Tn, int64_t namp, int dim,
                            const int* __restrict__ state) {
  const int inst = blockIdx.y;
  const int* st = state + inst * 4;
  if (st[2]) return;
  const int slot = dim > 0 ? (st[1] + 1) % dim : 0;
  cplx* T = Tn + (int64_t(inst) * (dim > 0 ? dim : 1) + slot) * namp;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
    const int64_t d = mir[2 * k], sw = mir[2 * k + 1];
    const int64_t s = sw & 0x7FFFFFFFFFFFFFFFll;
    const cplx v = T[s];
    T[d] = sw < 0 ? make_double2(-v.x, -v.y) : v;
  }
}

__global__ void k_set_roles(int8_t* __restrict__ role, const int64_t* __restrict__ idx, int64_t n, int stride,
                            int8_t value) {
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
    role[idx[k * stride]] = value;
}

// Element offsets in a blocked rank-4 layout from a table of its sub-blocks per irrep tuple.
struct BlockAddr {
  int G = 1;
  int sp[4] = {0, 0, 0, 0};
  int64_t base_off = 0;  // added to every offset (the t2 part of the amplitude vector)
  std::vector<SubBlock> sb;
  std::vector<const SubBlock*> tab;
  std::vector<int> irr[SP_COUNT], off[SP_COUNT];
  BlockAddr(const Ctx& c, const Layout& L, int64_t base) : G(c.G), base_off(base) {
    for (int k = 0; k < 4; ++k) sp[k] = L.sp[k];
    enumerate_blocks(L, c.spaces, sb);
    tab.assign(size_t(G) * G * G * G, nullptr);
    for (auto& b : sb) tab[((size_t(b.irr[0]) * G + b.irr[1]) * G + b.irr[2]) * G + b.irr[3]] = &b;
    for (int s = 0; s < SP_COUNT; ++s) {
      const Space& S = c.spaces[s];
      irr[s].assign(S.n, 0);
      off[s] = S.off;
      for (int g = 0; g < G; ++g)
        for (int k = 0; k < S.cnt[g]; ++k) irr[s][S.off[g] + k] = g;
    }
  }
  int64_t at(int i0, int i1, int i2, int i3) const {
    const int i[4] = {i0, i1, i2, i3};
    int g[4];
    for (int k = 0; k < 4; ++k) g[k] = irr[sp[k]][i[k]];
    const SubBlock* B = tab[((size_t(g[0]) * G + g[1]) * G + g[2]) * G + g[3]];
    if (!B) return -1;
    int64_t o = B->base;
    for (int k = 0; k < 4; ++k) o += (i[k] - off[sp[k]][g[k]]) * B->st[k];
    return base_off + o;
  }
};

// mirror entry: destination, source with the sign in bit 63
static void add_mirror(std::vector<int64_t>& m, int64_t dst, int64_t src, bool neg) {
  if (dst < 0 || src < 0) return;
  m.push_back(dst);
  m.push_back(neg ? int64_t(uint64_t(src) | (uint64_t(1) << 63)) : src);
}

// ---------------------------------------------------------------------------
static void fs_setup(Ctx& c) {
  FsState* s = new FsState();
  c.fs_state = s;
  const int na = c.nact;
  s->d_role = (int8_t*)c.dalloc(c.namp);
  s->d_Dfs = (double*)c.dalloc(sizeof(double) * c.namp * c.ninst);
  s->d_XV = (cplx*)c.dalloc(sizeof(cplx) * c.namp * c.ninst);
  CK(cudaMemsetAsync(s->d_XV, 0, sizeof(cplx) * c.namp * c.ninst, c.stream));
  s->X1 = c.t1;
  s->X1.d = s->d_XV;
  s->X2 = c.t2;
  s->X2.d = s->d_XV + c.n1;
  // roles and D_fs over both layouts
  std::vector<int> actslot(c.nv, -1);
  for (int k = 0; k < na; ++k) actslot[c.act[k]] = k;
  int* d_ghost = (int*)c.dalloc(sizeof(int) * c.no);
  int* d_actslot = (int*)c.dalloc(sizeof(int) * c.nv);
  upload(c, d_ghost, c.occ_ghost.data(), sizeof(int) * c.no);
  upload(c, d_actslot, actslot.data(), sizeof(int) * c.nv);
  for (int rank : {2, 4}) {
    const Layout& L = rank == 2 ? c.t1.L : c.t2.L;
    std::vector<GenTask> tk;
    std::vector<ChunkRef> ch;
    gen_tasks(c, L, tk, ch);
    if (ch.empty()) continue;
    GenTask* dt = (GenTask*)c.dalloc(tk.size() * sizeof(GenTask));
    ChunkRef* dc = (ChunkRef*)c.dalloc(ch.size() * sizeof(ChunkRef));
    upload(c, dt, tk.data(), tk.size() * sizeof(GenTask));
    upload(c, dc, ch.data(), ch.size() * sizeof(ChunkRef));
    const int64_t off = rank == 2 ? 0 : c.n1;
    k_fs_roles<<<int(ch.size()), 256, 0, c.stream>>>(s->d_role, off, dt, dc, rank, c.no, d_ghost, d_actslot);
    KCHECK(c);
    const int sg2[2] = {+1, -1}, sg4[4] = {+1, +1, -1, -1};
    launch_fill_denom(c, s->d_Dfs + off, c.namp, dt, dc, int(ch.size()), rank, rank == 2 ? sg2 : sg4, c.d_eps_fs);
  }
  // one-ghost doubles: the unknown is t2(a, b, g_x, j) with a < b; (b, a, g_x, j),
  // (a, b, j, g_x) and (b, a, j, g_x) are its signed copies
  {
    const BlockAddr A(c, c.t2.L, c.n1);
    std::vector<int64_t> mir;
    for (int gx = 0; gx < c.no; ++gx) {
      if (c.occ_ghost[gx] < 0) continue;
      for (int j = 0; j < c.no; ++j) {
        if (c.occ_ghost[j] >= 0) continue;
        for (int a = 0; a < c.nv; ++a)
          for (int b = a + 1; b < c.nv; ++b) {
            const int64_t p = A.at(a, b, gx, j);
            if (p < 0) continue;  // symmetry-forbidden
            add_mirror(mir, A.at(b, a, gx, j), p, true);
            add_mirror(mir, A.at(a, b, j, gx), p, true);
            add_mirror(mir, A.at(b, a, j, gx), p, false);
          }
      }
    }
    s->n_mir = int64_t(mir.size() / 2);
    s->d_mir = (int64_t*)c.dalloc(sizeof(int64_t) * std::max<size_t>(mir.size(), 2));
    upload(c, s->d_mir, mir.data(), sizeof(int64_t) * mir.size());
    if (s->n_mir) {
      k_set_roles<<<int(std::min<int64_t>((s->n_mir + 255) / 256, 4096)), 256, 0, c.stream>>>(s->d_role, s->d_mir,
                                                                                           s->n_mir, 2, ROLE_MIRROR);
      KCHECK(c);
    }
  }
  // H_eff gather list: t1(a = act[y], i = g_x) -> Hg(m = g_y, i = g_x), irreps equal
  s->Hg = *new_tensor(c, L2(c, SP_OCC, +1, SP_OCC, -1), true);
  std::vector<int> ghost_local(na, -1);
  for (int l = 0; l < c.no; ++l)
    if (c.occ_ghost[l] >= 0) ghost_local[c.occ_ghost[l]] = l;
  auto addr2 = [&](const Layout& L, int sp0, int l0, int sp1, int l1) -> int64_t {
    std::vector<SubBlock> sb;
    enumerate_blocks(L, c.spaces, sb);
    const Space& S0 = c.spaces[sp0];
    const Space& S1 = c.spaces[sp1];
    int g0 = 0, g1 = 0;
    while (g0 + 1 < c.G && S0.off[g0 + 1] <= l0) ++g0;
    while (g1 + 1 < c.G && S1.off[g1 + 1] <= l1) ++g1;
    for (auto& b : sb)
      if (b.irr[0] == g0 && b.irr[1] == g1) return b.base + (l0 - S0.off[g0]) * b.st[0] + (l1 - S1.off[g1]) * b.st[1];
    return -1;
  };
  std::vector<HPair> pairs;
  for (int y = 0; y < na; ++y)
    for (int x = 0; x < na; ++x) {
      const int64_t src = addr2(c.t1.L, SP_VIRT, c.act[y], SP_OCC, ghost_local[x]);
      const int64_t dst = addr2(s->Hg.L, SP_OCC, ghost_local[y], SP_OCC, ghost_local[x]);
      if (src < 0 || dst < 0) continue;  // different irreps: H_eff[y, x] = 0
      pairs.push_back(HPair{src, dst, y * na + x, 0});
    }
  s->n_pairs = int(pairs.size());
  s->d_pairs = (HPair*)c.dalloc(sizeof(HPair) * std::max<size_t>(pairs.size(), 1));
  upload(c, s->d_pairs, pairs.data(), sizeof(HPair) * pairs.size());
  s->d_heff = (cplx*)c.dalloc(sizeof(cplx) * na * na * c.ninst);
  CK(cudaMemsetAsync(s->d_heff, 0, sizeof(cplx) * na * na * c.ninst, c.stream));
  s->d_eig = (cplx*)c.dalloc(sizeof(cplx) * na * c.ninst);
  // active slots grouped by irrep for the eigensolver
  std::vector<int> blk, blk_off(c.G + 1, 0);
  std::vector<int> virt_irrep(c.nv);
  for (int g = 0; g < c.G; ++g)
    for (int a = 0; a < c.spaces[SP_VIRT].cnt[g]; ++a) virt_irrep[c.spaces[SP_VIRT].off[g] + a] = g;
  for (int g = 0; g < c.G; ++g) {
    blk_off[g] = int(blk.size());
    for (int k = 0; k < na; ++k)
      if (virt_irrep[c.act[k]] == g) blk.push_back(k);
  }
  blk_off[c.G] = int(blk.size());
  s->d_blk = (int*)c.dalloc(sizeof(int) * std::max(na, 1));
  s->d_blk_off = (int*)c.dalloc(sizeof(int) * (c.G + 1));
  upload(c, s->d_blk, blk.data(), sizeof(int) * na);
  upload(c, s->d_blk_off, blk_off.data(), sizeof(int) * (c.G + 1));
}

static void fs_run(Ctx& c) {
  FsState& s = F(c);
  const int64_t na = c.namp;
  const int dim = c.cfg.diis_dim;
  // start from P: ghost amplitudes = unit vectors; fresh DIIS
  k_fs_init<<<dim3(std::min<int64_t>((na + 255) / 256, 1216), c.ninst), 256, 0, c.stream>>>(c.d_T, s.d_role, na);
  KCHECK(c);
  ccsd_reset_diis(c);
  s.n_iter = 0;
  s.converged = false;
  for (int it = 1; it <= c.cfg.max_iter; ++it) {
    ccsd_rhs(c);
    k_fs_heff<<<dim3(1, c.ninst), 256, 0, c.stream>>>(s.d_pairs, s.n_pairs, c.d_R, c.d_D, c.d_T, na, s.Hg.d, s.Hg.is,
                                                      s.d_heff, c.nact, c.d_diis_state);
    KCHECK(c);
    // S H_eff:  X_ai = sum_m t_am Hg_mi ;  X_abij = P(ij) sum_m t_abmj Hg_mi  (m runs over ghosts)
    einsum(c, "FSx1", make_double2(1, 0), {&c.t1, nullptr, "am"}, {&s.Hg, nullptr, "mi"}, s.X1, "ai", false);
    einsum(c, "FSx2", make_double2(1, 0), {&c.t2, nullptr, "abmj"}, {&s.Hg, nullptr, "mi"}, s.X2, "abij", false,
           {{1.0, "abij"}, {-1.0, "abji"}});
    fs_step(c, s.d_Dfs, s.d_role, s.d_XV, s.d_mir, s.n_mir);
    s.n_iter = it;
    const int nconv = ccsd_count_converged(c);
    if (nconv < 0) throw ExpError{EXP_ENUMERIC, "NaN/Inf in the (0h,1p) amplitudes"};
    if (nconv == c.ninst) { s.converged = true; break; }
  }
  // eigenvalues per irrep block
  int* d_err = (int*)c.dalloc(sizeof(int));
  CK(cudaMemsetAsync(d_err, 0, sizeof(int), c.stream));
  k_fs_eig<<<c.ninst, 32, 0, c.stream>>>(s.d_heff, c.nact, s.d_blk, s.d_blk_off, c.G, s.d_eig, d_err);
  KCHECK(c);
  int err = 0;
  CK(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  s.h_heff.resize(size_t(c.nact) * c.nact * c.ninst);
  s.h_eig.resize(size_t(c.nact) * c.ninst);
  CK(cudaMemcpyAsync(s.h_heff.data(), s.d_heff, sizeof(cplx) * s.h_heff.size(), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaMemcpyAsync(s.h_eig.data(), s.d_eig, sizeof(cplx) * s.h_eig.size(), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  if (err == 1) throw ExpError{EXP_EINVAL, "an irrep block of H_eff is larger than 32"};
  if (err == 2) throw ExpError{EXP_ENUMERIC, "H_eff eigensolver did not converge"};
  s.done = true;
}

exp_status fs_entry(Ctx& c, int inst, double* heff, double* eig_re, double* eig_im, int* n_iter) {
  if (c.nact <= 0) throw ExpError{EXP_ESTATE, "no active spinors configured (n_active = 0)"};
  if (inst < 0 || inst >= c.ninst) throw ExpError{EXP_EINVAL, "instance out of range"};
  if (!c.fs_state) {
    if (ccsd_count_converged(c) != c.ninst)
      throw ExpError{EXP_ESTATE, "the (0h,0p) iteration has not converged for every instance"};
    fs_setup(c);
    fs_run(c);
  }
  FsState& s = F(c);
  const int na = c.nact;
  if (heff)
    for (int k = 0; k < na * na; ++k) {
      heff[2 * k] = s.h_heff[size_t(inst) * na * na + k].x;
      heff[2 * k + 1] = s.h_heff[size_t(inst) * na * na + k].y;
    }
  std::vector<std::complex<double>> w(na);
  for (int k = 0; k < na; ++k) w[k] = {s.h_eig[size_t(inst) * na + k].x, s.h_eig[size_t(inst) * na + k].y};
  std::sort(w.begin(), w.end(), [](const std::complex<double>& a, const std::complex<double>& b) {
    return a.real() != b.real() ? a.real() < b.real() : a.imag() < b.imag();
  });
  for (int k = 0; k < na; ++k) {
    if (eig_re) eig_re[k] = w[k].real();
    if (eig_im) eig_im[k] = w[k].imag();
  }
  if (n_iter) *n_iter = s.n_iter;
  return s.converged ? EXP_OK : EXP_ENOTCONV;
}

// one Bloch update + DIIS for every instance (kernels shared with the (0h,0p) path)
void fs_step(Ctx& c, const double* Dfs, const int8_t* role, const cplx* XV, const int64_t* mir, int64_t n_mir) {
  ccsd_update_step(c, [&](double* part, int nb) {
    k_fs_update<<<dim3(nb, c.ninst), 256, 0, c.stream>>>(c.d_R, c.d_D, Dfs, XV, role, c.d_T, c.d_diis_t, c.d_diis_e,
                                                         c.namp, c.cfg.diis_dim, c.d_diis_state, part,
                                                         c.cfg.level_shift, c.cfg.denom_shift, c.cfg.denom_shift_n);
    KCHECK(c);
    if (n_mir) {  // the signed copies follow their canonical element before DIIS sees the vector
      k_fs_mirror<<<dim3(int(std::min<int64_t>((n_mir + 255) / 256, 2048)), c.ninst), 256, 0, c.stream>>>(
          mir, n_mir, c.d_diis_t, c.namp, c.cfg.diis_dim, c.d_diis_state);
      KCHECK(c);
    }
  }, false);
}

// ---------------------------------------------------------------------------
// The (0h,2p) sector (Eq. (sectors): after (0h,0p) and (0h,1p), whose amplitudes stay
// fixed).  In the ghost picture the two-valence-particle amplitudes s_xy^ab are the
// doubles t_{g_x g_y}^{ab} (both occupied indices ghosts), zero until now.  The
// Bloch equation of the sector, projected on the two-particle determinants, is the
// CCSD residual at those elements minus the terms of Omega H_eff,
//     rho_xy^ab = R_{g_x g_y}^{ab} - sum_z s_zy^ab H1_zx - sum_w s_xw^ab H1_wy
//                 - 1/2 sum_zw tau_{g_z g_w}^{ab} H2_zw,xy,
// with H1 the converged (0h,1p) H_eff and H2_zw,xy the residual at the active-active
// elements (a = z, b = w): the connected two-particle part of the (0h,2p) H_eff, which
// is H1 (x) 1 + 1 (x) H1 + H2 on the pairs x < y.  The first two terms are the (0h,1p)
// S H_eff contraction over the ghost index; the last is the hole-hole ladder with H2
// in place of W_mnij.  Updated: the canonical elements (g_x before g_y, a < b, not both
// active) by rho / (e_x + e_y - e_a - e_b); the other three copies are written from
// them with the antisymmetry signs (steps taken on every copy separately let rounding
// grow a symmetric part the equations do not damp).

struct Fs2State {
  int8_t* d_role = nullptr;      // [namp]
  int64_t* d_mir = nullptr;      // [n_mir][2]: destination, source | sign in bit 63
  int64_t n_mir = 0;
  Tensor H2;                     // (m n | i j), ghost entries only
  HPair* d_pairs = nullptr;      // residual at t2(act z, act w, g_x, g_y) -> H2(g_z, g_w, g_x, g_y)
  int n_pairs = 0;
  cplx* d_h2 = nullptr;          // [ninst][na^4]: H2[z, w, x, y]
  cplx* d_heff = nullptr;        // [ninst][np^2]: pair H_eff
  cplx* d_eig = nullptr;         // [ninst][np]
  int* d_blk = nullptr;
  int* d_blk_off = nullptr;
  int npair = 0;
  bool done = false, converged = false;
  int n_iter = 0;
  std::vector<cplx> h_heff, h_eig;
};

static Fs2State& F2(Ctx& c) { return *reinterpret_cast<Fs2State*>(F(c).fs2); }
static void fs2_release(FsState& s) {
  delete reinterpret_cast<Fs2State*>(s.fs2);
  s.fs2 = nullptr;
}

static void fs2_setup(Ctx& c) {
  FsState& s1 = F(c);
  Fs2State* s = new Fs2State();
  s1.fs2 = s;
  const int na = c.nact;
  const Layout& L = c.t2.L;
  std::vector<SubBlock> sb;
  enumerate_blocks(L, c.spaces, sb);
  const Space& SO = c.spaces[SP_OCC];
  const Space& SV = c.spaces[SP_VIRT];
  auto irr = [&](const Space& S, int l) {
    int g = 0;
    while (g + 1 < c.G && S.off[g + 1] <= l) ++g;
    return g;
  };
  // sub-block of each (G_a, G_b, G_i, G_j) tuple of the t2 layout (a, b | i, j)
  std::map<std::array<int, 4>, const SubBlock*> blk;
  for (auto& b : sb) blk[{b.irr[0], b.irr[1], b.irr[2], b.irr[3]}] = &b;
  auto addr = [&](int a, int b, int i, int j) -> int64_t {
    const int ga = irr(SV, a), gb = irr(SV, b), gi = irr(SO, i), gj = irr(SO, j);
    auto it = blk.find({ga, gb, gi, gj});
    if (it == blk.end()) return -1;
    const SubBlock& B = *it->second;
    return c.n1 + B.base + (a - SV.off[ga]) * B.st[0] + (b - SV.off[gb]) * B.st[1] + (i - SO.off[gi]) * B.st[2] +
           (j - SO.off[gj]) * B.st[3];
  };
  std::vector<int> gl(na, -1);  // ghost local occupied index of each active slot
  for (int l = 0; l < c.no; ++l)
    if (c.occ_ghost[l] >= 0) gl[c.occ_ghost[l]] = l;
  std::vector<int> slot_of(c.nv, -1);
  for (int k = 0; k < na; ++k) slot_of[c.act[k]] = k;
  std::vector<int64_t> canon, mir;
  for (int x = 0; x < na; ++x)
    for (int y = 0; y < na; ++y) {
      if (x == y) continue;
      for (int a = 0; a < c.nv; ++a)
        for (int b = 0; b < c.nv; ++b) {
          if (a == b || (slot_of[a] >= 0 && slot_of[b] >= 0)) continue;
          const int64_t p = addr(a, b, gl[x], gl[y]);
          if (p < 0) continue;  // symmetry-forbidden
          const bool gx_first = gl[x] < gl[y];
          if (gx_first && a < b) {
            canon.push_back(p);
            continue;
          }
          // source: the canonical copy, sign = (-1)^(number of swaps)
          const int i0 = gx_first ? x : y, j0 = gx_first ? y : x;
          const int a0 = a < b ? a : b, b0 = a < b ? b : a;
          const int64_t src = addr(a0, b0, gl[i0], gl[j0]);
          const bool neg = (gx_first != (a < b));  // exactly one swap
          mir.push_back(p);
          mir.push_back(neg ? int64_t(uint64_t(src) | (uint64_t(1) << 63)) : src);
        }
    }
  s->n_mir = int64_t(mir.size() / 2);
  s->d_role = (int8_t*)c.dalloc(c.namp);
  CK(cudaMemsetAsync(s->d_role, ROLE_REAL, c.namp, c.stream));
  int64_t* d_canon = (int64_t*)c.dalloc(sizeof(int64_t) * std::max<size_t>(canon.size(), 1));
  upload(c, d_canon, canon.data(), sizeof(int64_t) * canon.size());
  s->d_mir = (int64_t*)c.dalloc(sizeof(int64_t) * std::max<size_t>(mir.size(), 2));
  upload(c, s->d_mir, mir.data(), sizeof(int64_t) * mir.size());
  if (!canon.empty()) {
    k_set_roles<<<int(std::min<int64_t>((int64_t(canon.size()) + 255) / 256, 4096)), 256, 0, c.stream>>>(
        s->d_role, d_canon, int64_t(canon.size()), 1, ROLE_Q);
    KCHECK(c);
  }
  if (s->n_mir) {
    k_set_roles<<<int(std::min<int64_t>((s->n_mir + 255) / 256, 4096)), 256, 0, c.stream>>>(s->d_role, s->d_mir,
                                                                                         s->n_mir, 2, ROLE_MIRROR);
    KCHECK(c);
  }
  // H2 gather: residual at t2(a = act z, b = act w, i = g_x, j = g_y) -> H2(g_z, g_w, g_x, g_y)
  s->H2 = *new_tensor(c, L4(c, SP_OCC, +1, SP_OCC, +1, SP_OCC, -1, SP_OCC, -1, 2), true);
  std::vector<SubBlock> hb;
  enumerate_blocks(s->H2.L, c.spaces, hb);
  std::map<std::array<int, 4>, const SubBlock*> hblk;
  for (auto& b : hb) hblk[{b.irr[0], b.irr[1], b.irr[2], b.irr[3]}] = &b;
  auto haddr = [&](int m, int n, int i, int j) -> int64_t {
    const int g[4] = {irr(SO, m), irr(SO, n), irr(SO, i), irr(SO, j)};
    auto it = hblk.find({g[0], g[1], g[2], g[3]});
    if (it == hblk.end()) return -1;
    const SubBlock& B = *it->second;
    return B.base + (m - SO.off[g[0]]) * B.st[0] + (n - SO.off[g[1]]) * B.st[1] + (i - SO.off[g[2]]) * B.st[2] +
           (j - SO.off[g[3]]) * B.st[3];
  };
  std::vector<HPair> hp;
  for (int z = 0; z < na; ++z)
    for (int w = 0; w < na; ++w)
      for (int x = 0; x < na; ++x)
        for (int y = 0; y < na; ++y) {
          if (z == w || x == y) continue;
          const int64_t src = addr(c.act[z], c.act[w], gl[x], gl[y]);
          const int64_t dst = haddr(gl[z], gl[w], gl[x], gl[y]);
          if (src < 0 || dst < 0) continue;
          hp.push_back(HPair{src, dst, ((z * na + w) * na + x) * na + y, 0});
        }
  s->n_pairs = int(hp.size());
  s->d_pairs = (HPair*)c.dalloc(sizeof(HPair) * std::max<size_t>(hp.size(), 1));
  upload(c, s->d_pairs, hp.data(), sizeof(HPair) * hp.size());
  const int64_t na4 = int64_t(na) * na * na * na;
  s->d_h2 = (cplx*)c.dalloc(sizeof(cplx) * std::max<int64_t>(na4, 1) * c.ninst);
  CK(cudaMemsetAsync(s->d_h2, 0, sizeof(cplx) * std::max<int64_t>(na4, 1) * c.ninst, c.stream));
  // pairs x < y grouped by pair irrep for the eigensolver
  s->npair = na * (na - 1) / 2;
  std::vector<int> pblk, pblk_off(c.G + 1, 0);
  for (int g = 0; g < c.G; ++g) {
    pblk_off[g] = int(pblk.size());
    int k = 0;
    for (int x = 0; x < na; ++x)
      for (int y = x + 1; y < na; ++y, ++k)
        if ((irr(SV, c.act[x]) + irr(SV, c.act[y])) % c.G == g) pblk.push_back(k);
  }
  pblk_off[c.G] = int(pblk.size());
  s->d_blk = (int*)c.dalloc(sizeof(int) * std::max(s->npair, 1));
  s->d_blk_off = (int*)c.dalloc(sizeof(int) * (c.G + 1));
  upload(c, s->d_blk, pblk.data(), sizeof(int) * pblk.size());
  upload(c, s->d_blk_off, pblk_off.data(), sizeof(int) * (c.G + 1));
  s->d_heff = (cplx*)c.dalloc(sizeof(cplx) * std::max(s->npair * s->npair, 1) * c.ninst);
  s->d_eig = (cplx*)c.dalloc(sizeof(cplx) * std::max(s->npair, 1) * c.ninst);
}

static void fs2_run(Ctx& c) {
  FsState& s1 = F(c);
  Fs2State& s = F2(c);
  const int na = c.nact;
  const int64_t nam = c.namp;
  ccsd_reset_diis(c);
  s.n_iter = 0;
  s.converged = false;
  Tensor* tau = work_tensor(c, "tau", c.t2.L);
  for (int it = 1; it <= c.cfg.max_iter; ++it) {
    ccsd_rhs(c);
    // H2 from the residual at the active-active elements (t = 0 there)
    k_fs_heff<<<dim3(1, c.ninst), 256, 0, c.stream>>>(s.d_pairs, s.n_pairs, c.d_R, c.d_D, c.d_T, nam, s.H2.d, s.H2.is,
                                                      s.d_h2, na * na, c.d_diis_state);
    KCHECK(c);
    // Omega H_eff terms: P(ij) sum_m t_abmj H1_mi (ghost m) + 1/2 sum_mn tau_abmn H2_mnij
    einsum(c, "FSx2", make_double2(1, 0), {&c.t2, nullptr, "abmj"}, {&s1.Hg, nullptr, "mi"}, s1.X2, "abij", false,
           {{1.0, "abij"}, {-1.0, "abji"}});
    einsum(c, "FS2hh", make_double2(0.5, 0), {tau, nullptr, "abmn"}, {&s.H2, nullptr, "mnij"}, s1.X2, "abij", true);
    fs_step(c, s1.d_Dfs, s.d_role, s1.d_XV, s.d_mir, s.n_mir);
    s.n_iter = it;
    const int nconv = ccsd_count_converged(c);
    if (nconv < 0) throw ExpError{EXP_ENUMERIC, "NaN/Inf in the (0h,2p) amplitudes"};
    if (nconv == c.ninst) { s.converged = true; break; }
  }
  // the (0h,2p) H_eff on the pairs x < y: H1 (x) 1 + 1 (x) H1 + H2, then its eigenvalues
  const int np = s.npair;
  const int64_t na4 = int64_t(na) * na * na * na;
  std::vector<cplx> h2(size_t(std::max<int64_t>(na4, 1)) * c.ninst);
  CK(cudaMemcpyAsync(h2.data(), s.d_h2, sizeof(cplx) * h2.size(), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  std::vector<std::pair<int, int>> pr;
  for (int x = 0; x < na; ++x)
    for (int y = x + 1; y < na; ++y) pr.push_back({x, y});
  s.h_heff.assign(size_t(np) * np * c.ninst, make_double2(0.0, 0.0));
  for (int k = 0; k < c.ninst; ++k) {
    const cplx* H1 = s1.h_heff.data() + size_t(k) * na * na;  // H1[y * na + x]
    const cplx* H2 = h2.data() + size_t(k) * na4;
    for (int r = 0; r < np; ++r)
      for (int q = 0; q < np; ++q) {
        const int z = pr[r].first, w = pr[r].second, x = pr[q].first, y = pr[q].second;
        cplx v = H2[((z * na + w) * na + x) * na + y];
        auto add = [&](double sg, cplx h) { v.x += sg * h.x; v.y += sg * h.y; };
        if (w == y) add(1.0, H1[z * na + x]);
        if (z == x) add(1.0, H1[w * na + y]);
        if (z == y) add(-1.0, H1[w * na + x]);
        if (w == x) add(-1.0, H1[z * na + y]);
        s.h_heff[(size_t(k) * np + r) * np + q] = v;
      }
  }
  if (np) {
    upload(c, s.d_heff, s.h_heff.data(), sizeof(cplx) * s.h_heff.size());
    int* d_err = (int*)c.dalloc(sizeof(int));
    CK(cudaMemsetAsync(d_err, 0, sizeof(int), c.stream));
    k_fs_eig<<<c.ninst, 32, 0, c.stream>>>(s.d_heff, np, s.d_blk, s.d_blk_off, c.G, s.d_eig, d_err);
    KCHECK(c);
    int err = 0;
    s.h_eig.resize(size_t(np) * c.ninst);
    CK(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(s.h_eig.data(), s.d_eig, sizeof(cplx) * s.h_eig.size(), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    if (err == 1) throw ExpError{EXP_EINVAL, "an irrep block of the (0h,2p) H_eff is larger than 32"};
    if (err == 2) throw ExpError{EXP_ENUMERIC, "(0h,2p) H_eff eigensolver did not converge"};
  }
  s.done = true;
}

exp_status fs2_entry(Ctx& c, int inst, double* heff, double* eig_re, double* eig_im, int* n_iter) {
  if (c.nact < 2) throw ExpError{EXP_ESTATE, "the (0h,2p) sector needs at least two active spinors"};
  if (inst < 0 || inst >= c.ninst) throw ExpError{EXP_EINVAL, "instance out of range"};
  if (!c.fs_state || !F(c).done) {
    const exp_status st = fs_entry(c, inst, nullptr, nullptr, nullptr, nullptr);
    if (st != EXP_OK) throw ExpError{EXP_ESTATE, "the (0h,1p) sector has not converged"};
  }
  if (!F(c).converged) throw ExpError{EXP_ESTATE, "the (0h,1p) sector has not converged"};
  if (!F(c).fs2) {
    fs2_setup(c);
    fs2_run(c);
  }
  Fs2State& s = F2(c);
  const int np = s.npair;
  if (heff)
    for (int k = 0; k < np * np; ++k) {
      heff[2 * k] = s.h_heff[size_t(inst) * np * np + k].x;
      heff[2 * k + 1] = s.h_heff[size_t(inst) * np * np + k].y;
    }
  std::vector<std::complex<double>> w(np);
  for (int k = 0; k < np; ++k) w[k] = {s.h_eig[size_t(inst) * np + k].x, s.h_eig[size_t(inst) * np + k].y};
  std::sort(w.begin(), w.end(), [](const std::complex<double>& a, const std::complex<double>& b) {
    return a.real() != b.real() ? a.real() < b.real() : a.imag() < b.imag();
  });
  for (int k = 0; k < np; ++k) {
    if (eig_re) eig_re[k] = w[k].real();
    if (eig_im) eig_im[k] = w[k].imag();
  }
  if (n_iter) *n_iter = s.n_iter;
  return s.converged ? EXP_OK : EXP_ENOTCONV;
}
