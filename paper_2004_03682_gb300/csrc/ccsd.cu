// CCSD for the (0h,0p) sector on the GPU: the amplitude equations of
// Eq. (amplitudes) truncated to singles and doubles, written as Stanton-Gauss
// intermediates, every term one TTGT contraction on symmetry-blocked tensors
// (Sec. II.B / II.C).  Plus the FP64 update t_new = RHS/D, the residual, the
// energy and DIIS, all on the device; one iteration is replayed as a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <functional>

#include "ccsd.h"
#include "emu.h"
#include "packed.h"

static const cplx ONE = {1.0, 0.0};
static inline cplx C(double x) { return make_double2(x, 0.0); }

// Integral classes: V(p,q,r,s) by the spaces of its arguments.
static const IntRef OOOO{{SP_OCC, SP_OCC, SP_OCC, SP_OCC}};
static const IntRef OOOV{{SP_OCC, SP_OCC, SP_OCC, SP_VIRT}};
static const IntRef OOVO{{SP_OCC, SP_OCC, SP_VIRT, SP_OCC}};
static const IntRef OOVV{{SP_OCC, SP_OCC, SP_VIRT, SP_VIRT}};
static const IntRef OVOV{{SP_OCC, SP_VIRT, SP_OCC, SP_VIRT}};
static const IntRef OVVO{{SP_OCC, SP_VIRT, SP_VIRT, SP_OCC}};
static const IntRef OVVV{{SP_OCC, SP_VIRT, SP_VIRT, SP_VIRT}};
static const IntRef OVOO{{SP_OCC, SP_VIRT, SP_OCC, SP_OCC}};
static const IntRef VOVV{{SP_VIRT, SP_OCC, SP_VIRT, SP_VIRT}};
static const IntRef VVVO{{SP_VIRT, SP_VIRT, SP_VIRT, SP_OCC}};
static const IntRef VVVV{{SP_VIRT, SP_VIRT, SP_VIRT, SP_VIRT}};

Layout L4(Ctx& c, int s0, int g0, int s1, int g1, int s2, int g2, int s3, int g3, int nrow) {
  const int sp[4] = {s0, s1, s2, s3}, sg[4] = {g0, g1, g2, g3};
  return make_layout(c.spaces, c.G, 4, sp, sg, nrow);
}
Layout L2(Ctx& c, int s0, int g0, int s1, int g1) {
  const int sp[2] = {s0, s1}, sg[2] = {g0, g1};
  return make_layout(c.spaces, c.G, 2, sp, sg, 1);
}

// ---------------------------------------------------------------------------
// Reductions: per-CTA partials in fixed order, then a one-CTA finaliser, so
// every run is bitwise reproducible.
#define RED_BLOCKS 152
#define RED_THREADS 256

template <typename T, typename Op>
__device__ T block_reduce(T v, Op op, T* sh) {
  for (int o = 16; o; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < (blockDim.x >> 5)) ? sh[l] : T(0);  // 0 is neutral for both sums and max of |.|
    for (int o = 16; o; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}
// max that propagates NaN (fmax would drop it and let a diverged instance look converged)
__device__ __forceinline__ double nanmax(double a, double b) { return (b != b || b > a) ? b : a; }
struct MaxOp { __device__ double operator()(double a, double b) const { return nanmax(a, b); } };
struct AddOp { __device__ double operator()(double a, double b) const { return a + b; } };

// Dinv = 1 / (D - sigma), once per context (the update then needs no FP64 divide)
// (with an intruder-state shift ds, D~ = dyn_shift(D) stands for D: the shifted equations)
__global__ void k_inv_denom(const double* __restrict__ D, double* __restrict__ Dinv, int64_t n, double shift,
                            double ds, int dn) {
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
    Dinv[k] = 1.0 / (dyn_shift(D[k], ds, dn) - shift);
}

// t_new = (R - sigma t) / (D - sigma) over the whole amplitude vector (sigma = 0:
// R / D); e = t_new - t.  Writes t_new and e into the next DIIS slot and the
// per-CTA max |e|^2 (k_finalize_update takes the root).  Frozen instances skip.
//
// dpart != nullptr: also the DIIS inner products Re<e, e_j> of the new error vector with
// itself (j = 0) and with the stored ones of the window (j = 1..count, newest first),
// per CTA into dpart (the partials k_diis_solve sums) -- the same grid and element
// order as k_diis_dots, so the same bits, without reading e back.
__global__ void __launch_bounds__(RED_THREADS) k_update(const cplx* __restrict__ R, const double* __restrict__ Dinv,
                                                        const cplx* __restrict__ T, cplx* __restrict__ Tn,
                                                        cplx* __restrict__ En, int64_t namp, int dim,
                                                        const int* __restrict__ state, double* __restrict__ part,
                                                        double shift, double* __restrict__ dpart) {
  __shared__ double sh[32];
  const int inst = blockIdx.y;
  const int* st = state + inst * 4;
  const int slot = dim > 0 ? (st[1] + 1) % dim : 0;
  const int nd = (dpart && dim > 0) ? min(st[0] + 1, dim) : 0;  // dots after this push
  const int64_t off = int64_t(inst) * namp;
  const int64_t soff = (int64_t(inst) * (dim > 0 ? dim : 1) + slot) * namp;
  double m = 0.0;
  double acc[EXP_MAX_DIIS];
#pragma unroll
  for (int j = 0; j < EXP_MAX_DIIS; ++j) acc[j] = 0.0;
  if (!st[2]) {
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < namp; k += int64_t(gridDim.x) * blockDim.x) {
      const cplx r = R[off + k];
      const double q = Dinv[off + k];
      const cplx t = T[off + k];
      const cplx tn = make_double2(fma(-shift, t.x, r.x) * q, fma(-shift, t.y, r.y) * q);
      const cplx e = make_double2(tn.x - t.x, tn.y - t.y);
      Tn[soff + k] = tn;
      En[soff + k] = e;
      m = nanmax(m, fma(e.x, e.x, e.y * e.y));
      if (nd) {
        acc[0] += e.x * e.x + e.y * e.y;
#pragma unroll
        for (int j = 1; j < EXP_MAX_DIIS; ++j)
          if (j < nd) {
            const cplx b = En[(int64_t(inst) * dim + (slot - j + dim) % dim) * namp + k];
            acc[j] += e.x * b.x + e.y * b.y;
          }
      }
    }
  }
  m = block_reduce(m, MaxOp(), sh);
  if (threadIdx.x == 0) part[(inst * gridDim.x + blockIdx.x) * 8] = m;
  if (dpart && dim > 0)
#pragma unroll
    for (int j = 0; j < EXP_MAX_DIIS; ++j)
      if (j < dim) {  // dim is uniform over the block (the reduction synchronises)
        const double a = block_reduce(acc[j], AddOp(), sh);
        if (threadIdx.x == 0) dpart[(inst * gridDim.x + blockIdx.x) * EXP_MAX_DIIS + j] = a;
      }
}

// sum of the nb per-CTA partials part[(inst * nb + b) * stride + j] over one warp:
// lane l adds b = l, l + 32, ... in order, then a fixed shuffle tree (reproducible)
__device__ __forceinline__ double warp_sum_partials(const double* __restrict__ part, int inst, int nb, int stride,
                                                    int j) {
  const int l = threadIdx.x & 31;
  double s = 0.0;
  for (int b = l; b < nb; b += 32) s += part[(int64_t(inst) * nb + b) * stride + j];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// per instance (one warp): residual, NaN check, convergence, DIIS push.
__global__ void k_finalize_update(const double* __restrict__ part, int nb, int* __restrict__ state,
                                  double* __restrict__ stats, int dim, double tol) {
  const int inst = blockIdx.x;
  if (threadIdx.x >= 32) return;
  int* st = state + inst * 4;
  double* s = stats + inst * 8;
  if (st[2]) {
    if (threadIdx.x == 0) s[0] = 0.0;
    return;
  }
  double m = 0.0;
  bool bad = false;
  for (int b = threadIdx.x; b < nb; b += 32) {
    const double v = part[(inst * nb + b) * 8];
    if (!(v == v) || isinf(v)) bad = true;
    m = nanmax(m, v);
  }
  for (int o = 16; o; o >>= 1) m = nanmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  bad = __any_sync(0xffffffffu, bad);
  if (threadIdx.x) return;
  m = sqrt(m);  // the update kernels reduce |e|^2
  s[0] = bad ? INFINITY : m;
  s[4] = bad ? 1.0 : 0.0;
  if (bad) {  // this instance failed: freeze it as failed (2), the others go on
    st[2] = 2;
    return;
  }
  if (dim > 0) {
    st[1] = (st[1] + 1) % dim;
    st[0] = min(st[0] + 1, dim);
  }
  if (m < tol && !bad) st[3] = 1;  // converged this iteration (freeze after extrapolation)
}

// Energy partial sums E = 1/4 sum conj(<ab||ij>) tau_ij^ab (<ij||ab> = conj <ab||ij>), with
// tau formed on the fly from the amplitude vector T = [t1 | t2]
// (tau_ij^ab = t2 + t1_ai t1_bj - t1_bi t1_aj): CTA b walks the t2 sub-block chunks
// b, b + gridDim.x, ... in a fixed order, so the result is reproducible.
__global__ void __launch_bounds__(RED_THREADS) k_energy_tau(const cplx* __restrict__ Vd, int64_t vis,
                                                            const cplx* __restrict__ T, int64_t tis, int64_t n1,
                                                            const int32_t* __restrict__ t1i,
                                                            const GenTask* __restrict__ tasks,
                                                            const ChunkRef* __restrict__ chunks, int n_chunks, int no,
                                                            int vbase, const int* __restrict__ state,
                                                            double* __restrict__ part, int skip_frozen) {
  __shared__ double sh[32];
  const int inst = blockIdx.y;
  double er = 0.0, ei = 0.0;
  if (!(skip_frozen && state[inst * 4 + 2])) {
    const cplx* v = Vd + inst * vis;
    const cplx* t1 = T + inst * tis;
    const cplx* t2 = t1 + n1;
    for (int cidx = blockIdx.x; cidx < n_chunks; cidx += gridDim.x) {
      const ChunkRef ch = chunks[cidx];
      const GenTask Tk = tasks[ch.task];
      const uint32_t n1_ = Tk.n[1], n2_ = Tk.n[2], n3_ = Tk.n[3];
      const uint32_t end = uint32_t(min(ch.start + (int64_t)EXP_CHUNK, Tk.count));
      for (uint32_t e = uint32_t(ch.start) + threadIdx.x; e < end; e += blockDim.x) {
        uint32_t r = e;
        const int i3 = int(r % n3_);
        r /= n3_;
        const int i2 = int(r % n2_);
        r /= n2_;
        const int i1 = int(r % n1_);
        const int i0 = int(r / n1_);
        const int a = Tk.g0[0] + i0 - vbase, b = Tk.g0[1] + i1 - vbase;
        const int ii = Tk.g0[2] + i2, jj = Tk.g0[3] + i3;
        const int64_t p = Tk.base + i0 * Tk.st[0] + i1 * Tk.st[1] + i2 * Tk.st[2] + i3 * Tk.st[3];
        cplx x = t2[p];
        const int kai = t1i[a * no + ii], kbj = t1i[b * no + jj];
        if (kai >= 0 && kbj >= 0) {
          const cplx u = t1[kai], w = t1[kbj];
          x.x += u.x * w.x - u.y * w.y;
          x.y += u.x * w.y + u.y * w.x;
        }
        const int kbi = t1i[b * no + ii], kaj = t1i[a * no + jj];
        if (kbi >= 0 && kaj >= 0) {
          const cplx u = t1[kbi], w = t1[kaj];
          x.x -= u.x * w.x - u.y * w.y;
          x.y -= u.x * w.y + u.y * w.x;
        }
        const cplx va = v[p];
        er += va.x * x.x + va.y * x.y;
        ei += va.x * x.y - va.y * x.x;
      }
    }
  }
  er = block_reduce(er, AddOp(), sh);
  ei = block_reduce(ei, AddOp(), sh);
  if (threadIdx.x == 0) {
    part[(inst * gridDim.x + blockIdx.x) * 8 + 1] = er;
    part[(inst * gridDim.x + blockIdx.x) * 8 + 2] = ei;
  }
}

__global__ void k_finalize_energy(const double* __restrict__ part, int nb, const int* __restrict__ state,
                                  double* __restrict__ stats, int skip_frozen, double scale) {
  const int inst = blockIdx.x;
  if (threadIdx.x >= 32) return;
  if (skip_frozen && state[inst * 4 + 2]) return;
  const double er = warp_sum_partials(part, inst, nb, 8, 1);
  const double ei = warp_sum_partials(part, inst, nb, 8, 2);
  if (threadIdx.x) return;
  stats[inst * 8 + 1] = scale * er;
  stats[inst * 8 + 2] = scale * ei;
}

// DIIS: dots of the newest error vector with every stored one (Re <e_new, e_k>).
__global__ void __launch_bounds__(RED_THREADS) k_diis_dots(const cplx* __restrict__ E, int64_t namp, int dim,
                                                           const int* __restrict__ state,
                                                           double* __restrict__ part) {
  __shared__ double sh[32];
  const int inst = blockIdx.y;
  const int* st = state + inst * 4;
  const int cnt = st[0], head = st[1];
  const bool active = !st[2];
  const cplx* en = E + (int64_t(inst) * dim + head) * namp;
  for (int j = 0; j < dim; ++j) {
    double acc = 0.0;
    if (active && j < cnt) {
      const int slot = (head - j + dim) % dim;
      const cplx* ek = E + (int64_t(inst) * dim + slot) * namp;
      for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < namp; k += int64_t(gridDim.x) * blockDim.x) {
        const cplx a = en[k], b = ek[k];
        acc += a.x * b.x + a.y * b.y;
      }
    }
    acc = block_reduce(acc, AddOp(), sh);
    if (threadIdx.x == 0) part[((inst * gridDim.x + blockIdx.x) * EXP_MAX_DIIS + j)] = acc;
  }
}

// DIIS solve per instance: B over slots (by age), bordered system, Gaussian
// elimination with partial pivoting; a pivot below 1e-14 max diag drops the
// oldest vector.  Writes coefficients per slot (0 for unused).
__global__ void k_diis_solve(const double* __restrict__ part, int nb, int dim, int* __restrict__ state,
                             double* __restrict__ Bm, double* __restrict__ coef, double* __restrict__ stats) {
  const int inst = blockIdx.x;
  if (threadIdx.x >= 32) return;
  int* st = state + inst * 4;
  double* cf = coef + inst * EXP_MAX_DIIS;
  if (st[2]) {
    if (threadIdx.x < EXP_MAX_DIIS) cf[threadIdx.x] = 0.0;
    return;
  }
  const int head = st[1], cnt0 = st[0];
  double* B = Bm + inst * EXP_MAX_DIIS * EXP_MAX_DIIS;  // B[slot][slot]
  // new row / column from the dots (partials summed over the warp)
  for (int j = 0; j < cnt0; ++j) {
    const double s = warp_sum_partials(part, inst, nb, EXP_MAX_DIIS, j);
    if (threadIdx.x == 0) {
      const int slot = (head - j + dim) % dim;
      B[head * EXP_MAX_DIIS + slot] = s;
      B[slot * EXP_MAX_DIIS + head] = s;
    }
  }
  if (threadIdx.x) return;
  for (int k = 0; k < EXP_MAX_DIIS; ++k) cf[k] = 0.0;
  int cnt = st[0];
  while (cnt >= 2) {
    // order by age: index 0 = oldest
    int sl[EXP_MAX_DIIS];
    for (int k = 0; k < cnt; ++k) sl[k] = (head - (cnt - 1 - k) + dim) % dim;
    const int m = cnt + 1;
    double A[EXP_MAX_DIIS + 1][EXP_MAX_DIIS + 1], y[EXP_MAX_DIIS + 1];
    double dmax = 0.0;
    for (int k = 0; k < cnt; ++k) {
      for (int l = 0; l < cnt; ++l) A[k][l] = B[sl[k] * EXP_MAX_DIIS + sl[l]];
      A[k][cnt] = -1.0;
      A[cnt][k] = -1.0;
      y[k] = 0.0;
      dmax = fmax(dmax, A[k][k]);
    }
    A[cnt][cnt] = 0.0;
    y[cnt] = -1.0;
    const double tiny = 1e-14 * dmax;
    bool ok = true;
    for (int k = 0; k < m && ok; ++k) {
      int p = k;
      for (int r = k + 1; r < m; ++r)
        if (fabs(A[r][k]) > fabs(A[p][k])) p = r;
      if (fabs(A[p][k]) < tiny) { ok = false; break; }
      if (p != k) {
        for (int c2 = 0; c2 < m; ++c2) { const double t = A[k][c2]; A[k][c2] = A[p][c2]; A[p][c2] = t; }
        const double t = y[k]; y[k] = y[p]; y[p] = t;
      }
      for (int r = k + 1; r < m; ++r) {
        const double f = A[r][k] / A[k][k];
        for (int c2 = k; c2 < m; ++c2) A[r][c2] -= f * A[k][c2];
        y[r] -= f * y[k];
      }
    }
    if (ok) {
      double x[EXP_MAX_DIIS + 1];
      for (int k = m - 1; k >= 0; --k) {
        double s = y[k];
        for (int c2 = k + 1; c2 < m; ++c2) s -= A[k][c2] * x[c2];
        x[k] = s / A[k][k];
      }
      for (int k = 0; k < cnt; ++k) cf[sl[k]] = x[k];
      st[0] = cnt;
      stats[inst * 8 + 3] = cnt;
      return;
    }
    --cnt;  // drop the oldest
    st[0] = cnt;
  }
  cf[head] = 1.0;  // fewer than 2 vectors: plain update
  stats[inst * 8 + 3] = st[0];
}

// T = sum_k c_k t_new_k (or t_new when DIIS is off / not yet active).
__global__ void __launch_bounds__(256) k_extrapolate(cplx* __restrict__ T, const cplx* __restrict__ Tn,
                                                     int64_t namp, int dim, const double* __restrict__ coef,
                                                     int* __restrict__ state) {
  const int inst = blockIdx.y;
  const int* st = state + inst * 4;
  if (st[2]) return;
  const int D = dim > 0 ? dim : 1;
  const double* cf = coef + inst * EXP_MAX_DIIS;
  const bool plain = dim == 0 || st[3];
  const int head = dim > 0 ? st[1] : 0;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < namp; k += int64_t(gridDim.x) * blockDim.x) {
    double vr = 0.0, vi = 0.0;
    if (plain) {
      const cplx x = Tn[(int64_t(inst) * D + head) * namp + k];
      vr = x.x; vi = x.y;
    } else {
      for (int s = 0; s < D; ++s) {
        const double c = cf[s];
        if (c != 0.0) {
          const cplx x = Tn[(int64_t(inst) * D + s) * namp + k];
          vr += c * x.x;
          vi += c * x.y;
        }
      }
    }
    T[int64_t(inst) * namp + k] = make_double2(vr, vi);
  }
}

// converged instances freeze after their final t_new has been taken
__global__ void k_freeze(int* __restrict__ state, int ninst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ninst && state[i * 4 + 3] && state[i * 4 + 2] == 0) state[i * 4 + 2] = 1;
}

// ---------------------------------------------------------------------------
// The pair-packed amplitude vector: t1, then the entries a<b, i<j of t2 (rows and
// columns of the doubles layout as pair-packed tables).  t2 is antisymmetric in
// (a, b) and in (i, j), so these entries determine it; the update, the DIIS vectors,
// the extrapolation and the energy act on them alone (a quarter of the FP64 work
// and of the DIIS storage), and the extrapolation writes the four signed copies.
#define PK_THREADS 1024

// offset in one instance's full t2 of packed t2 entry e
__device__ __forceinline__ int64_t pk_full(const PackDims& D, const int32_t* __restrict__ rfull,
                                           const int32_t* __restrict__ cfull, int64_t e) {
  const int g = find_block(D.blk, D.G, e);
  const uint32_t loc = uint32_t(e - D.blk[g]);
  const uint32_t p = loc / uint32_t(D.nc[g]), q = loc - p * uint32_t(D.nc[g]);
  return D.fblk[g] + int64_t(rfull[D.roff[g] + p]) * D.fnc[g] + cfull[D.coff[g] + q];
}

// Dinv = 1 / (D - sigma) on the packed vector
__global__ void k_inv_denom_pk(const double* __restrict__ Dn, double* __restrict__ Dinv, int64_t namp, int64_t npk,
                               int64_t n1, PackDims D, const int32_t* __restrict__ rfull,
                               const int32_t* __restrict__ cfull, double shift, double ds, int dn) {
  const int inst = blockIdx.y;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < npk; k += int64_t(gridDim.x) * blockDim.x) {
    const int64_t f = k < n1 ? k : n1 + pk_full(D, rfull, cfull, k - n1);
    Dinv[inst * npk + k] = 1.0 / (dyn_shift(Dn[inst * namp + f], ds, dn) - shift);
  }
}

// k_update on the packed vector: R and T are read at each entry's full offset,
// t_new and e go packed into the DIIS slot.  A stored t2 error is doubled: it
// stands for the four entries +-e of the full vector, so inner products of stored
// errors equal those of the full error vectors (the weight of t2 against t1 in
// the DIIS matrix is unchanged).
__global__ void __launch_bounds__(PK_THREADS) k_update_pk(const cplx* __restrict__ R, const double* __restrict__ Dinv,
                                                          const cplx* __restrict__ T, cplx* __restrict__ Tn,
                                                          cplx* __restrict__ En, int64_t namp, int64_t npk, int64_t n1,
                                                          PackDims D, const int32_t* __restrict__ rfull,
                                                          const int32_t* __restrict__ cfull, int dim,
                                                          const int* __restrict__ state, double* __restrict__ part,
                                                          double shift, double* __restrict__ dpart) {
  __shared__ double sh[32];
  const int inst = blockIdx.y;
  const int* st = state + inst * 4;
  const int slot = dim > 0 ? (st[1] + 1) % dim : 0;
  const int nd = dim > 0 ? min(st[0] + 1, dim) : 0;
  const int64_t off = int64_t(inst) * namp;
  const int64_t soff = (int64_t(inst) * (dim > 0 ? dim : 1) + slot) * npk;
  double m = 0.0;
  double acc[EXP_MAX_DIIS];
#pragma unroll
  for (int j = 0; j < EXP_MAX_DIIS; ++j) acc[j] = 0.0;
  if (!st[2]) {
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < npk; k += int64_t(gridDim.x) * blockDim.x) {
      const int64_t f = k < n1 ? k : n1 + pk_full(D, rfull, cfull, k - n1);
      const cplx r = R[off + f];
      const double q = Dinv[int64_t(inst) * npk + k];
      const cplx t = T[off + f];
      const cplx tn = make_double2(fma(-shift, t.x, r.x) * q, fma(-shift, t.y, r.y) * q);
      const cplx e = make_double2(tn.x - t.x, tn.y - t.y);
      Tn[soff + k] = tn;
      m = nanmax(m, fma(e.x, e.x, e.y * e.y));
      const cplx ew = k < n1 ? e : make_double2(e.x + e.x, e.y + e.y);
      En[soff + k] = ew;
      if (nd) {
        acc[0] += ew.x * ew.x + ew.y * ew.y;
#pragma unroll
        for (int j = 1; j < EXP_MAX_DIIS; ++j)
          if (j < nd) {
            const cplx b = En[(int64_t(inst) * dim + (slot - j + dim) % dim) * npk + k];
            acc[j] += ew.x * b.x + ew.y * b.y;
          }
      }
    }
  }
  m = block_reduce(m, MaxOp(), sh);
  if (threadIdx.x == 0) part[(inst * gridDim.x + blockIdx.x) * 8] = m;
  if (dim > 0)
#pragma unroll
    for (int j = 0; j < EXP_MAX_DIIS; ++j)
      if (j < dim) {  // dim is uniform over the block (the reduction synchronises)
        const double a = block_reduce(acc[j], AddOp(), sh);
        if (threadIdx.x == 0) dpart[(inst * gridDim.x + blockIdx.x) * EXP_MAX_DIIS + j] = a;
      }
}

// T = sum_k c_k t_new_k on the packed vector, written to the full amplitude vector:
// t1 as is, each t2 entry to (a,b,i,j) and (b,a,j,i), its negative to (b,a,i,j)
// and (a,b,j,i).  The entries a = b or i = j are never written (they stay zero).
__global__ void __launch_bounds__(256) k_extrapolate_pk(cplx* __restrict__ T, const cplx* __restrict__ Tn,
                                                        int64_t namp, int64_t npk, int64_t n1, PackDims D,
                                                        const int32_t* __restrict__ rfull,
                                                        const int32_t* __restrict__ rswp,
                                                        const int32_t* __restrict__ cfull,
                                                        const int32_t* __restrict__ cswp, int dim,
                                                        const double* __restrict__ coef,
                                                        const int* __restrict__ state) {
  const int inst = blockIdx.y;
  const int* st = state + inst * 4;
  if (st[2]) return;
  const int Dm = dim > 0 ? dim : 1;
  const double* cf = coef + inst * EXP_MAX_DIIS;
  const bool plain = dim == 0 || st[3];
  const int head = dim > 0 ? st[1] : 0;
  cplx* t = T + int64_t(inst) * namp;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < npk; k += int64_t(gridDim.x) * blockDim.x) {
    double vr = 0.0, vi = 0.0;
    if (plain) {
      const cplx x = Tn[(int64_t(inst) * Dm + head) * npk + k];
      vr = x.x; vi = x.y;
    } else {
      for (int s = 0; s < Dm; ++s) {
        const double c = cf[s];
        if (c != 0.0) {
          const cplx x = Tn[(int64_t(inst) * Dm + s) * npk + k];
          vr += c * x.x;
          vi += c * x.y;
        }
      }
    }
    if (k < n1) {
      t[k] = make_double2(vr, vi);
      continue;
    }
    const int64_t e = k - n1;
    const int g = find_block(D.blk, D.G, e);
    const uint32_t loc = uint32_t(e - D.blk[g]);
    const uint32_t p = loc / uint32_t(D.nc[g]), q = loc - p * uint32_t(D.nc[g]);
    const int64_t nc = D.fnc[g];
    const int64_t r0 = int64_t(rfull[D.roff[g] + p]) * nc, r1 = int64_t(rswp[D.roff[g] + p]) * nc;
    const int64_t c0 = cfull[D.coff[g] + q], c1 = cswp[D.coff[g] + q];
    cplx* b = t + n1 + D.fblk[g];
    b[r0 + c0] = make_double2(vr, vi);
    b[r1 + c1] = make_double2(vr, vi);
    b[r1 + c0] = make_double2(-vr, -vi);
    b[r0 + c1] = make_double2(-vr, -vi);
  }
}

// E = sum over a<b, i<j of conj(<ab||ij>) tau_ij^ab (the 1/4 sum over every entry of
// the two antisymmetric tensors), tau from the newest packed t_new of each active
// instance; partials as k_energy_tau writes them.
__global__ void __launch_bounds__(PK_THREADS) k_energy_pk(const cplx* __restrict__ Vp, const cplx* __restrict__ Tn,
                                                          int64_t npk, int64_t n1, int dim, PackDims D,
                                                          const int32_t* __restrict__ rpair,
                                                          const int32_t* __restrict__ cpair,
                                                          const int32_t* __restrict__ t1i, int no,
                                                          const int* __restrict__ state, double* __restrict__ part) {
  __shared__ double sh[32];
  const int inst = blockIdx.y;
  const int* st = state + inst * 4;
  double er = 0.0, ei = 0.0;
  if (!st[2]) {
    const int head = dim > 0 ? st[1] : 0;
    const cplx* t1 = Tn + (int64_t(inst) * (dim > 0 ? dim : 1) + head) * npk;
    const cplx* t2 = t1 + n1;
    const cplx* v = Vp + int64_t(inst) * (npk - n1);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < npk - n1;
         e += int64_t(gridDim.x) * blockDim.x) {
      const int g = find_block(D.blk, D.G, e);
      const uint32_t loc = uint32_t(e - D.blk[g]);
      const uint32_t p = loc / uint32_t(D.nc[g]), q = loc - p * uint32_t(D.nc[g]);
      const int32_t pr = rpair[D.roff[g] + p], pc = cpair[D.coff[g] + q];
      const int a = (pr >> 16) - no, b = (pr & 0xffff) - no, ii = pc >> 16, jj = pc & 0xffff;
      cplx x = t2[e];
      const int kai = t1i[a * no + ii], kbj = t1i[b * no + jj];
      if (kai >= 0 && kbj >= 0) {
        const cplx u = t1[kai], w = t1[kbj];
        x.x += u.x * w.x - u.y * w.y;
        x.y += u.x * w.y + u.y * w.x;
      }
      const int kbi = t1i[b * no + ii], kaj = t1i[a * no + jj];
      if (kbi >= 0 && kaj >= 0) {
        const cplx u = t1[kbi], w = t1[kaj];
        x.x -= u.x * w.x - u.y * w.y;
        x.y -= u.x * w.y + u.y * w.x;
      }
      const cplx va = v[e];
      er += va.x * x.x + va.y * x.y;
      ei += va.x * x.y - va.y * x.x;
    }
  }
  er = block_reduce(er, AddOp(), sh);
  ei = block_reduce(ei, AddOp(), sh);
  if (threadIdx.x == 0) {
    part[(inst * gridDim.x + blockIdx.x) * 8 + 1] = er;
    part[(inst * gridDim.x + blockIdx.x) * 8 + 2] = ei;
  }
}

// the entries a = b or i = j of t2 set to zero (the packed update never writes them)
__global__ void k_zero_pair_diag(cplx* __restrict__ T2, int64_t namp, PackDims D, const int32_t* __restrict__ rinv,
                                 const int32_t* __restrict__ cinv) {
  const int inst = blockIdx.y;
  const int64_t total = D.fblk[D.G];
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int g = find_block(D.fblk, D.G, e);
    const uint32_t loc = uint32_t(e - D.fblk[g]);
    const uint32_t r = loc / uint32_t(D.fnc[g]), cc = loc - r * uint32_t(D.fnc[g]);
    if (rinv[D.froff[g] + r] == 0 || cinv[D.fcoff[g] + cc] == 0) T2[inst * namp + e] = make_double2(0.0, 0.0);
  }
}

// scale pass: max |V_abij / D_ij^ab| per instance
__global__ void __launch_bounds__(RED_THREADS) k_maxratio(const cplx* __restrict__ V, int64_t vis,
                                                          const double* __restrict__ D, int64_t dis, int64_t off,
                                                          int64_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  const int inst = blockIdx.y;
  double m = 0.0;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
    const cplx v = V[inst * vis + k];
    m = nanmax(m, hypot(v.x, v.y) / fabs(D[inst * dis + off + k]));
  }
  m = block_reduce(m, MaxOp(), sh);
  if (threadIdx.x == 0) part[(inst * gridDim.x + blockIdx.x) * 8] = m;
}

__global__ void k_set_scale(const double* __restrict__ part, int nb, const double* __restrict__ mult,
                            double* __restrict__ scale) {
  const int inst = blockIdx.x;
  if (threadIdx.x) return;
  double m = 0.0;
  for (int b = 0; b < nb; ++b) m = fmax(m, part[(inst * nb + b) * 8]);
  scale[inst] = 0.05 / m * mult[inst];
}

__global__ void k_rescale(cplx* __restrict__ V, int64_t vis, int64_t n, const double* __restrict__ scale) {
  const int inst = blockIdx.y;
  const double s = scale[inst];
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
    cplx v = V[inst * vis + k];
    V[inst * vis + k] = make_double2(s * v.x, s * v.y);
  }
}

// t2 = V_abij / D (MP2 first-order amplitudes), t1 = 0
// (with an intruder-state shift: V / D~, the first Jacobi step of the shifted equations)
__global__ void k_mp2_guess(cplx* __restrict__ T, const double* __restrict__ D, const cplx* __restrict__ Vd,
                            int64_t vis, int64_t n1, int64_t namp, double ds, int dn) {
  const int inst = blockIdx.y;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < namp; k += int64_t(gridDim.x) * blockDim.x) {
    cplx out = make_double2(0, 0);
    if (k >= n1) {
      const cplx v = Vd[inst * vis + (k - n1)];
      const double d = dyn_shift(D[inst * namp + k], ds, dn);
      out = make_double2(v.x / d, v.y / d);
    }
    T[inst * namp + k] = out;
  }
}

// ---------------------------------------------------------------------------
static int grid_for(int64_t n, int threads = 256, int cap = 4 * 152) {
  int64_t b = (n + threads - 1) / threads;
  return int(std::max<int64_t>(1, std::min<int64_t>(b, cap)));
}

struct TauTasks {
  GenTask* d_tasks = nullptr;
  ChunkRef* d_chunks = nullptr;
  int n_chunks = 0;
};

struct CcsdState {
  TauTasks t2tasks;
  TauTasks t1tasks;
  int32_t* d_t1i = nullptr;
  double* d_part = nullptr;
  double* d_dots = nullptr;  // DIIS inner-product partials formed in the update kernel
  double* d_coef = nullptr;
  const Tensor* Vd = nullptr;  // <ab||ij> in the t2 layout
  double* d_Dinv = nullptr;    // 1 / (D - sigma), filled on the first (eager) iteration
  bool dinv_ready = false;
  // the pair-packed amplitude vector (packed contexts): t1, then t2 over a<b, i<j
  struct {
    bool on = false;
    PackDims D{};
    const PairTable *vv = nullptr, *oo = nullptr;
    int64_t n = 0;             // n1 + packed t2 entries
    double* d_Dinv = nullptr;  // [ninst][n]
    cplx* d_V = nullptr;       // [ninst][n - n1] <ab||ij> on the packed entries
  } pk;
};

static CcsdState& S(Ctx& c) { return *reinterpret_cast<CcsdState*>(c.ccsd_state); }

void ccsd_setup(Ctx& c) {
  CcsdState* s = new CcsdState();
  c.ccsd_state = s;
  c.t1.L = L2(c, SP_VIRT, +1, SP_OCC, -1);
  c.t2.L = L4(c, SP_VIRT, +1, SP_VIRT, +1, SP_OCC, -1, SP_OCC, -1, 2);
  c.n1 = c.t1.L.size;
  c.n2 = c.t2.L.size;
  c.namp = c.n1 + c.n2;
  const int64_t na = c.namp, ni = c.ninst;
  c.d_T = (cplx*)c.dalloc(sizeof(cplx) * na * ni);
  c.d_R = (cplx*)c.dalloc(sizeof(cplx) * na * ni);
  c.d_D = (double*)c.dalloc(sizeof(double) * na * ni);
  if (c.cfg.packed) {
    s->pk.D = packed_t2_space(c, c.t2.L, &s->pk.vv, &s->pk.oo);
    s->pk.n = c.n1 + s->pk.D.blk[s->pk.D.G];
    s->pk.d_Dinv = (double*)c.dalloc(sizeof(double) * s->pk.n * ni);
    s->pk.d_V = (cplx*)c.dalloc(sizeof(cplx) * std::max<int64_t>(s->pk.n - c.n1, 1) * ni);
    s->pk.on = true;
  } else {
    s->d_Dinv = (double*)c.dalloc(sizeof(double) * na * ni);
  }
  CK(cudaMemsetAsync(c.d_T, 0, sizeof(cplx) * na * ni, c.stream));
  const int dslots = std::max(c.cfg.diis_dim, 1);
  c.d_diis_t = (cplx*)c.dalloc(sizeof(cplx) * na * ni * dslots);
  c.d_diis_e = (cplx*)c.dalloc(sizeof(cplx) * na * ni * dslots);
  c.d_diis_B = (double*)c.dalloc(sizeof(double) * EXP_MAX_DIIS * EXP_MAX_DIIS * ni);
  c.d_diis_state = (int*)c.dalloc(sizeof(int) * 4 * ni);
  c.d_stats = (double*)c.dalloc(sizeof(double) * 8 * ni);
  CK(cudaMemsetAsync(c.d_diis_state, 0, sizeof(int) * 4 * ni, c.stream));
  CK(cudaMemsetAsync(c.d_stats, 0, sizeof(double) * 8 * ni, c.stream));
  CK(cudaMemsetAsync(c.d_diis_B, 0, sizeof(double) * EXP_MAX_DIIS * EXP_MAX_DIIS * ni, c.stream));
  CK(cudaMallocHost(&c.h_stats, sizeof(double) * 8 * ni));
  s->d_part = (double*)c.dalloc(sizeof(double) * 8 * RED_BLOCKS * ni * EXP_MAX_DIIS);
  s->d_dots = (double*)c.dalloc(sizeof(double) * RED_BLOCKS * ni * EXP_MAX_DIIS);
  s->d_coef = (double*)c.dalloc(sizeof(double) * EXP_MAX_DIIS * ni);
  c.t1.d = c.d_T;
  c.t1.is = na;
  c.t2.d = c.d_T + c.n1;
  c.t2.is = na;
  c.r1 = c.t1;
  c.r1.d = c.d_R;
  c.r2 = c.t2;
  c.r2.d = c.d_R + c.n1;
  c.r2.pair_canon = c.cfg.packed != 0;  // the packed update reads R2 at a<b, i<j only
  // denominators
  {
    std::vector<GenTask> tk;
    std::vector<ChunkRef> ch;
    gen_tasks(c, c.t1.L, tk, ch);
    if (!ch.empty()) {
      GenTask* dt = (GenTask*)c.dalloc(tk.size() * sizeof(GenTask));
      ChunkRef* dc = (ChunkRef*)c.dalloc(ch.size() * sizeof(ChunkRef));
      upload(c, dt, tk.data(), tk.size() * sizeof(GenTask));
      upload(c, dc, ch.data(), ch.size() * sizeof(ChunkRef));
      const int sg[2] = {+1, -1};
      launch_fill_denom(c, c.d_D, na, dt, dc, int(ch.size()), 2, sg, nullptr);
      s->t1tasks.d_tasks = dt;
      s->t1tasks.d_chunks = dc;
      s->t1tasks.n_chunks = int(ch.size());
    }
    tk.clear();
    ch.clear();
    gen_tasks(c, c.t2.L, tk, ch);
    if (!ch.empty()) {
      GenTask* dt = (GenTask*)c.dalloc(tk.size() * sizeof(GenTask));
      ChunkRef* dc = (ChunkRef*)c.dalloc(ch.size() * sizeof(ChunkRef));
      upload(c, dt, tk.data(), tk.size() * sizeof(GenTask));
      upload(c, dc, ch.data(), ch.size() * sizeof(ChunkRef));
      const int sg[4] = {+1, +1, -1, -1};
      launch_fill_denom(c, c.d_D + c.n1, na, dt, dc, int(ch.size()), 4, sg, nullptr);
      s->t2tasks.d_tasks = dt;
      s->t2tasks.d_chunks = dc;
      s->t2tasks.n_chunks = int(ch.size());
    }
  }
  // t1 index table: offset of t1_ai (a, i local) or -1
  {
    std::vector<int32_t> idx(size_t(c.nv) * c.no, -1);
    std::vector<SubBlock> sb;
    enumerate_blocks(c.t1.L, c.spaces, sb);
    for (auto& b : sb) {
      const int a0 = c.spaces[SP_VIRT].off[b.irr[0]], i0 = c.spaces[SP_OCC].off[b.irr[1]];
      for (int a = 0; a < b.n[0]; ++a)
        for (int i = 0; i < b.n[1]; ++i) idx[size_t(a0 + a) * c.no + i0 + i] = int32_t(b.base + a * b.st[0] + i * b.st[1]);
    }
    s->d_t1i = (int32_t*)c.dalloc(idx.size() * sizeof(int32_t));
    upload(c, s->d_t1i, idx.data(), idx.size() * sizeof(int32_t));
  }
}

void ccsd_release(Ctx& c) {
  delete reinterpret_cast<CcsdState*>(c.ccsd_state);
  c.ccsd_state = nullptr;
}

// Generate the driver <ab||ij> unscaled, fix the per-instance scale so that
// max |t_MP2| = 0.05 (times the caller's multiplier), rescale it.
void ccsd_init_integrals(Ctx& c, const double* h_mult) {
  CcsdState& s = S(c);
  std::vector<double> ones(c.ninst, 1.0);
  upload(c, c.d_scale, ones.data(), sizeof(double) * c.ninst);
  c.have_integrals = true;
  const int arg[4] = {0, 1, 2, 3};
  const IntRef VVOO{{SP_VIRT, SP_VIRT, SP_OCC, SP_OCC}};
  const Tensor* Vd = integral(c, VVOO, arg, 2);
  s.Vd = Vd;
  const int nb = RED_BLOCKS;
  k_maxratio<<<dim3(nb, c.ninst), RED_THREADS, 0, c.stream>>>(Vd->d, Vd->is, c.d_D, c.namp, c.n1, c.n2, s.d_part);
  KCHECK(c);
  double* d_mult = (double*)c.dalloc(sizeof(double) * c.ninst);
  upload(c, d_mult, h_mult, sizeof(double) * c.ninst);
  k_set_scale<<<c.ninst, 32, 0, c.stream>>>(s.d_part, nb, d_mult, c.d_scale);
  KCHECK(c);
  k_rescale<<<dim3(grid_for(c.n2), c.ninst), 256, 0, c.stream>>>(const_cast<cplx*>(Vd->d), Vd->is, c.n2, c.d_scale);
  KCHECK(c);
  if (s.pk.on)  // <ab||ij> on the packed entries, for the packed energy
    launch_pack_gather(c, s.pk.d_V, s.pk.n - c.n1, Vd->d, Vd->is, s.pk.D, *s.pk.vv, *s.pk.oo);
  c.h_scale.resize(c.ninst);
  CK(cudaMemcpyAsync(c.h_scale.data(), c.d_scale, sizeof(double) * c.ninst, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  c.integrals_scaled = true;
}

// Packed contexts: the pair-diagonal entries of a freshly set t2 made zero (the
// packed update writes only a<b, i<j and their signed copies).
static void zero_pair_diag(Ctx& c) {
  CcsdState& s = S(c);
  const int64_t nf = s.pk.on ? s.pk.D.fblk[s.pk.D.G] : 0;
  if (!nf) return;
  k_zero_pair_diag<<<dim3(grid_for(nf), c.ninst), 256, 0, c.stream>>>(c.d_T + c.n1, c.namp, s.pk.D, s.pk.vv->d_inv,
                                                                     s.pk.oo->d_inv);
  KCHECK(c);
}

void ccsd_guess(Ctx& c) {
  CcsdState& s = S(c);
  k_mp2_guess<<<dim3(grid_for(c.namp), c.ninst), 256, 0, c.stream>>>(c.d_T, c.d_D, s.Vd->d, s.Vd->is, c.n1, c.namp,
                                                                      c.cfg.denom_shift, c.cfg.denom_shift_n);
  KCHECK(c);
  ccsd_mark_guessed(c);
}

void ccsd_reset_diis(Ctx& c) {
  CK(cudaMemsetAsync(c.d_diis_state, 0, sizeof(int) * 4 * c.ninst, c.stream));
  CK(cudaMemsetAsync(c.d_diis_B, 0, sizeof(double) * EXP_MAX_DIIS * EXP_MAX_DIIS * c.ninst, c.stream));
  CK(cudaMemsetAsync(c.d_stats, 0, sizeof(double) * 8 * c.ninst, c.stream));
  c.iter_done = 0;
}

// E of the amplitude vector at `T` (per instance) into stats[1..2].
void ccsd_energy_of(Ctx& c, const cplx* T, bool skip_frozen) {
  CcsdState& s = S(c);
  const int nb = RED_BLOCKS;
  k_energy_tau<<<dim3(nb, c.ninst), RED_THREADS, 0, c.stream>>>(s.Vd->d, s.Vd->is, T, c.namp, c.n1, s.d_t1i,
                                                                s.t2tasks.d_tasks, s.t2tasks.d_chunks,
                                                                s.t2tasks.n_chunks, c.no, c.no, c.d_diis_state,
                                                                s.d_part, skip_frozen);
  KCHECK(c);
  k_finalize_energy<<<c.ninst, 32, 0, c.stream>>>(s.d_part, nb, c.d_diis_state, c.d_stats, skip_frozen, 0.25);
  KCHECK(c);
}

// ---------------------------------------------------------------------------
// The right-hand sides R1, R2 of the T1 and T2 equations at the current T.
static void copy_int(Ctx& c, Tensor& dst, const Tensor* src) {
  if (src->L.size != dst.L.size) throw ExpError{EXP_EINVAL, "copy between different layouts"};
  CK(cudaMemcpy2DAsync(dst.d, dst.is * sizeof(cplx), src->d, src->is * sizeof(cplx), dst.L.size * sizeof(cplx),
                       c.ninst, cudaMemcpyDeviceToDevice, c.stream));
}

static void copy_t(Ctx& c, Tensor& dst, const Tensor& src) {
  if (src.L.size != dst.L.size) throw ExpError{EXP_EINVAL, "copy between different layouts"};
  CK(cudaMemcpy2DAsync(dst.d, dst.is * sizeof(cplx), src.d, src.is * sizeof(cplx), dst.L.size * sizeof(cplx),
                       c.ninst, cudaMemcpyDeviceToDevice, c.stream));
}

// delta_mj on the occupied space, layout (O, -1 | O, +1): a contraction with it over
// (m, j) is the trace over m = j
static const Tensor& delta_oo(Ctx& c) {
  auto it = c.work.find("delta_oo");
  if (it != c.work.end()) return *it->second;
  const Layout L = L2(c, SP_OCC, -1, SP_OCC, +1);
  Tensor* t = work_tensor(c, "delta_oo", L);
  std::vector<SubBlock> sb;
  enumerate_blocks(L, c.spaces, sb);
  std::vector<cplx> h(size_t(t->is) * c.ninst, make_double2(0.0, 0.0));
  for (const SubBlock& b : sb) {
    if (b.irr[0] != b.irr[1]) continue;  // the block rule allows no other
    for (int inst = 0; inst < c.ninst; ++inst)
      for (int x = 0; x < b.n[0]; ++x) h[size_t(inst) * t->is + b.base + x * b.st[0] + x * b.st[1]] = make_double2(1.0, 0.0);
  }
  upload(c, t->d, h.data(), h.size() * sizeof(cplx));
  return *t;
}

void ccsd_rhs(Ctx& c) {
  const int V = SP_VIRT, O = SP_OCC;
  Tensor& t1 = c.t1;
  Tensor& t2 = c.t2;
  Tensor& r1 = c.r1;
  Tensor& r2 = c.r2;
  Tensor& tau = *work_tensor(c, "tau", t2.L);
  Tensor& taut = *work_tensor(c, "taut", t2.L);
  Tensor& zeta = *work_tensor(c, "zeta", t2.L);
  Tensor& Fae = *work_tensor(c, "Fae", L2(c, V, +1, V, -1));
  Tensor& Fmi = *work_tensor(c, "Fmi", L2(c, O, +1, O, -1));
  Tensor& Fme = *work_tensor(c, "Fme", L2(c, O, +1, V, -1));
  Tensor& Fp = *work_tensor(c, "Fp", L2(c, V, +1, V, -1));
  Tensor& Fq = *work_tensor(c, "Fq", L2(c, O, +1, O, -1));
  Tensor& Wmnij = *work_tensor(c, "Wmnij", L4(c, O, +1, O, +1, O, -1, O, -1, 2));
  Tensor& Wmbej = *work_tensor(c, "Wemjb", L4(c, V, -1, O, +1, O, -1, V, +1, 2));  // labels "emjb"
  Tensor& X = *work_tensor(c, "Xamij", L4(c, V, +1, O, +1, O, -1, O, -1, 2));
  Tensor& Q = *work_tensor(c, "Qaijb", L4(c, V, +1, O, -1, O, -1, V, +1, 2));
  Tensor& Z = *work_tensor(c, "Zmbji", L4(c, O, +1, V, +1, O, -1, O, -1, 3));
  CcsdState& s = S(c);

  // tau = t2 + t1^t1 (antisymmetrised), taut = t2 + t1^t1 / 2, zeta = t2 / 2 + t_i^a t_j^b
  launch_tau3(c, tau.d, taut.d, zeta.d, tau.is, c.t2.d, c.t1.d, c.namp, s.d_t1i, s.t2tasks.d_tasks,
              s.t2tasks.d_chunks, s.t2tasks.n_chunks);
  // pair-packed operands: tau over c<d, i<j once per iteration for the four products that sum over a tau pair
  const bool packed = c.cfg.packed != 0;
  if (packed) packed_tau(c, tau);

  // F_ae = Y_ae - 1/2 sum_mnf taut_mn^af <mn||ef>,  Y_ae = sum_mf t_m^f <ma||fe>   (f_ov = 0, f diagonal)
  Tensor& Y = *work_tensor(c, "Yae", L2(c, V, +1, V, -1));
  einsum(c, "Fae1", ONE, {nullptr, &OVVV, "mafe"}, {&t1, nullptr, "fm"}, Y, "ae", false);
  copy_t(c, Fae, Y);
  einsum(c, "Fae2", C(-0.5), {&taut, nullptr, "afmn"}, {nullptr, &OOVV, "mnef"}, Fae, "ae", true);
  // F_me = sum_nf t_n^f <mn||ef>
  einsum(c, "Fme", ONE, {nullptr, &OOVV, "mnef"}, {&t1, nullptr, "fn"}, Fme, "me", false);
  // X2_mnij = 1/2 sum_ef tau_ij^ef <mn||ef>, the tau part of W_mnij (factor 1/2 instead
  // of 1/4: it carries the (1/4) tau <mn||ef> part of W_abef too)
  Tensor& X2 = *work_tensor(c, "X2mnij", Wmnij.L);
  if (packed) {
    CK(cudaMemset2DAsync(X2.d, X2.is * sizeof(cplx), 0, X2.L.size * sizeof(cplx), c.ninst, c.stream));
    packed_wmnij(c, X2);
  } else {
    einsum(c, "Wmnij2", C(0.5), {nullptr, &OOVV, "mnef"}, {&tau, nullptr, "efij"}, X2, "mnij", false);
  }
  // F_mi = sum_ne t_n^e <mn||ie> + 1/2 sum_nef taut_in^ef <mn||ef>, the second term as
  // sum_n X2_mn,in - 1/2 sum_e t_i^e F_me: taut = tau - 1/2 (t_i^e t_n^f - t_i^f t_n^e)
  // and <mn||ef> = -<mn||fe> leave 1/4 sum_nef <mn||ef> (t_i^e t_n^f - t_i^f t_n^e) =
  // 1/2 sum_e t_i^e F_me.  No product over a t2-sized operand.
  einsum(c, "Fmi1", ONE, {nullptr, &OOOV, "mnie"}, {&t1, nullptr, "en"}, Fmi, "mi", false);
  einsum(c, "Fmi2x", ONE, {&X2, nullptr, "mnij"}, {&delta_oo(c), nullptr, "nj"}, Fmi, "mi", true);
  einsum(c, "Fmi2t", C(-0.5), {&Fme, nullptr, "me"}, {&t1, nullptr, "ei"}, Fmi, "mi", true);
  // W_mnij = <mn||ij> + P(ij) sum_e t_j^e <mn||ie> + X2_mnij
  {
    const int arg[4] = {0, 1, 2, 3};
    copy_int(c, Wmnij, integral(c, OOOO, arg, 2));
  }
  einsum(c, "Wmnij1", ONE, {nullptr, &OOOV, "mnie"}, {&t1, nullptr, "ej"}, Wmnij, "mnij", true,
         {{1.0, "mnij"}, {-1.0, "mnji"}});
  permute_into(c, "WmnijX2", Wmnij, "mnij", X2, "mnij", true);
  // W_mbej = <mb||ej> + sum_f t_j^f <mb||ef> - sum_n t_n^b <mn||ej> - sum_nf zeta_jn^fb <mn||ef>
  {
    const int arg[4] = {2, 0, 3, 1};  // storage (e, m, j, b) <- V(m, b, e, j)
    copy_int(c, Wmbej, integral(c, OVVO, arg, 2));
  }
  einsum(c, "Wmbej1", ONE, {nullptr, &OVVV, "mbef"}, {&t1, nullptr, "fj"}, Wmbej, "emjb", true);
  einsum(c, "Wmbej2", C(-1.0), {nullptr, &OOVO, "mnej"}, {&t1, nullptr, "bn"}, Wmbej, "emjb", true);
  einsum(c, "Wmbej3", C(-1.0), {nullptr, &OOVV, "mnef"}, {&zeta, nullptr, "fbjn"}, Wmbej, "emjb", true);

  // ---- T1 equation
  CK(cudaMemset2DAsync(r1.d, r1.is * sizeof(cplx), 0, r1.L.size * sizeof(cplx), c.ninst, c.stream));
  einsum(c, "R1a", ONE, {&Fae, nullptr, "ae"}, {&t1, nullptr, "ei"}, r1, "ai", true);
  einsum(c, "R1b", C(-1.0), {&t1, nullptr, "am"}, {&Fmi, nullptr, "mi"}, r1, "ai", true);
  // t2 in the (ai | em) order of the ring product's A operand, permuted once for both
  // products that read it that way (R1's t_im^ae F_me term and the ring product)
  Tensor& t2x = *work_tensor(c, "t2aiem", L4(c, V, +1, O, -1, V, +1, O, -1, 2));
  permute_into(c, "T2aiem", t2x, "aiem", t2, "aeim", false);
  einsum(c, "R1c", ONE, {&t2x, nullptr, "aiem"}, {&Fme, nullptr, "me"}, r1, "ai", true);
  einsum(c, "R1d", C(-1.0), {nullptr, &OVOV, "naif"}, {&t1, nullptr, "fn"}, r1, "ai", true);
  // -1/2 sum_mef <ma||ef> t_im^ef = 1/2 sum_m X_am,im - sum_e Y_ae t_i^e, with
  // X_amij = sum_ef <am||ef> tau_ij^ef (the W_abef t1 intermediate below): tau - t2 =
  // t_i^e t_m^f - t_i^f t_m^e and <am||ef> = -<am||fe> = -<ma||ef> = <ma||fe> leave
  // sum_mef <am||ef> (tau - t2)_im^ef = 2 sum_e t_i^e Y_ae.  No product over the
  // o v^3 integral; the X trace is added once X is formed.
  einsum(c, "R1ey", C(-1.0), {&Y, nullptr, "ae"}, {&t1, nullptr, "ei"}, r1, "ai", true);
  einsum(c, "R1f", C(-0.5), {&t2, nullptr, "aemn"}, {nullptr, &OOVO, "nmei"}, r1, "ai", true);

  // ---- T2 equation
  if (r2.pair_canon && c.canon_pairs)
    permute_into(c, "R2V", r2, "abij", *s.Vd, "abij", false);  // canonical entries only
  else
    copy_int(c, r2, s.Vd);
  // F'_be = F_be - 1/2 sum_m t_m^b F_me ;  + P(ab) sum_e t_ij^ae F'_be
  copy_t(c, Fp, Fae);
  einsum(c, "Fp", C(-0.5), {&t1, nullptr, "bm"}, {&Fme, nullptr, "me"}, Fp, "be", true);
  einsum(c, "R2a", ONE, {&Fp, nullptr, "be"}, {&t2, nullptr, "aeij"}, r2, "abij", true,
         {{1.0, "abij"}, {-1.0, "baij"}});
  // F'_mj = F_mj + 1/2 sum_e t_j^e F_me ;  - P(ij) sum_m t_im^ab F'_mj
  copy_t(c, Fq, Fmi);
  einsum(c, "Fq", C(0.5), {&Fme, nullptr, "me"}, {&t1, nullptr, "ej"}, Fq, "mj", true);
  einsum(c, "R2b", C(-1.0), {&t2, nullptr, "abim"}, {&Fq, nullptr, "mj"}, r2, "abij", true,
         {{1.0, "abij"}, {-1.0, "abji"}});
  // hole-hole ladder: 1/2 sum_mn tau_mn^ab W_mnij
  if (packed)
    packed_hh(c, Wmnij, r2);
  else
    einsum(c, "R2hh", C(0.5), {&tau, nullptr, "abmn"}, {&Wmnij, nullptr, "mnij"}, r2, "abij", true);
  // particle-particle ladder: 1/2 sum_ef <ab||ef> tau_ij^ef
  if (packed)
    packed_ladder(c, r2);
  else
    einsum(c, "R2pp", C(0.5), {nullptr, &VVVV, "abef"}, {&tau, nullptr, "efij"}, r2, "abij", true);
  // W_abef's t1 term: -1/2 P(ab) sum_m t_m^b X_amij,  X_amij = sum_ef <am||ef> tau_ij^ef
  if (packed)
    packed_xamij(c, X);
  else
    einsum(c, "Xamij", ONE, {nullptr, &VOVV, "amef"}, {&tau, nullptr, "efij"}, X, "amij", false);
  einsum(c, "R2x", C(-0.5), {&X, nullptr, "amij"}, {&t1, nullptr, "bm"}, r2, "abij", true,
         {{1.0, "abij"}, {-1.0, "baij"}});
  // the X trace of the T1 equation (see R1ey): + 1/2 sum_m X_am,im
  einsum(c, "R1ex", C(0.5), {&X, nullptr, "amij"}, {&delta_oo(c), nullptr, "mj"}, r1, "ai", true);
  // ring: P(ij)P(ab) [ sum_me t_im^ae W_mbej - sum_me t_i^e t_m^a <mb||ej> ]
  einsum(c, "Qring", ONE, {&t2x, nullptr, "aiem"}, {&Wmbej, nullptr, "emjb"}, Q, "aijb", false);
  einsum(c, "Zmbji", ONE, {nullptr, &OVVO, "mbej"}, {&t1, nullptr, "ei"}, Z, "mbji", false);
  einsum(c, "Qt1t1", C(-1.0), {&t1, nullptr, "am"}, {&Z, nullptr, "mbji"}, Q, "aijb", true);
  permute_into(c, "R2ring", r2, "abij", Q, "aijb", true,
               {{1.0, "abij"}, {-1.0, "abji"}, {-1.0, "baij"}, {1.0, "baji"}});
  // + P(ij) sum_e t_i^e <ab||ej>
  einsum(c, "R2c", ONE, {nullptr, &VVVO, "abej"}, {&t1, nullptr, "ei"}, r2, "abij", true,
         {{1.0, "abij"}, {-1.0, "abji"}});
  // - P(ab) sum_m t_m^a <mb||ij>
  einsum(c, "R2d", C(-1.0), {&t1, nullptr, "am"}, {nullptr, &OVOO, "mbij"}, r2, "abij", true,
         {{1.0, "abij"}, {-1.0, "baij"}});
}

// copy the newest t_new of every (active) instance into dst (namp-strided)
__global__ void k_copy_newest(cplx* __restrict__ dst, const cplx* __restrict__ Tn, int64_t namp, int dim,
                              const int* __restrict__ state) {
  const int inst = blockIdx.y;
  const int* st = state + inst * 4;
  if (st[2]) return;
  const int D = dim > 0 ? dim : 1;
  const int head = dim > 0 ? st[1] : 0;
  const cplx* src = Tn + (int64_t(inst) * D + head) * namp;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < namp; k += int64_t(gridDim.x) * blockDim.x)
    dst[int64_t(inst) * namp + k] = src[k];
}

void copy_newest(Ctx& c, cplx* dst) {
  k_copy_newest<<<dim3(grid_for(c.namp), c.ninst), 256, 0, c.stream>>>(dst, c.d_diis_t, c.namp, c.cfg.diis_dim,
                                                                      c.d_diis_state);
  KCHECK(c);
}

// Update + residual + (energy) + DIIS for every instance.  `upd` launches the
// update kernel that writes t_new and the error into the next DIIS slot and the
// per-CTA max |error| into part (RED_BLOCKS CTAs per instance).
void ccsd_update_step(Ctx& c, const std::function<void(double*, int)>& upd, bool energy, bool dots_done,
                      bool packed) {
  CcsdState& s = S(c);
  const int dim = c.cfg.diis_dim;
  const int64_t nvec = packed ? s.pk.n : c.namp;  // length of the DIIS vectors
  // packed kernels (PK_THREADS per CTA): no more CTAs per instance than the vector fills,
  // so a batch of small instances does not launch mostly idle blocks
  const int nb = packed ? int(std::max<int64_t>(1, std::min<int64_t>(RED_BLOCKS, (nvec + PK_THREADS - 1) / PK_THREADS)))
                        : RED_BLOCKS;
  upd(s.d_part, nb);
  k_finalize_update<<<c.ninst, 32, 0, c.stream>>>(s.d_part, nb, c.d_diis_state, c.d_stats, dim, c.cfg.conv_tol);
  KCHECK(c);
  if (dim > 0) {
    if (!dots_done) {
      k_diis_dots<<<dim3(nb, c.ninst), RED_THREADS, 0, c.stream>>>(c.d_diis_e, nvec, dim, c.d_diis_state, s.d_dots);
      KCHECK(c);
    }
    k_diis_solve<<<c.ninst, 32, 0, c.stream>>>(s.d_dots, nb, dim, c.d_diis_state, c.d_diis_B, s.d_coef, c.d_stats);
    KCHECK(c);
  }
  if (energy && packed) {  // energy of the newest packed t_new, read in place
    k_energy_pk<<<dim3(nb, c.ninst), PK_THREADS, 0, c.stream>>>(s.pk.d_V, c.d_diis_t, s.pk.n, c.n1, dim, s.pk.D,
                                                               s.pk.vv->d_pair, s.pk.oo->d_pair, s.d_t1i, c.no,
                                                               c.d_diis_state, s.d_part);
    KCHECK(c);
    k_finalize_energy<<<c.ninst, 32, 0, c.stream>>>(s.d_part, nb, c.d_diis_state, c.d_stats, 1, 1.0);
    KCHECK(c);
  } else if (energy) {
    // energy of t_new: gather the newest t_new of every instance into R (free by
    // now), then tau + dot
    copy_newest(c, c.d_R);
    ccsd_energy_of(c, c.d_R, true);
  }
  if (packed) {
    k_extrapolate_pk<<<dim3(grid_for(s.pk.n), c.ninst), 256, 0, c.stream>>>(
        c.d_T, c.d_diis_t, c.namp, s.pk.n, c.n1, s.pk.D, s.pk.vv->d_full, s.pk.vv->d_swp, s.pk.oo->d_full,
        s.pk.oo->d_swp, dim, s.d_coef, c.d_diis_state);
  } else {
    k_extrapolate<<<dim3(grid_for(c.namp), c.ninst), 256, 0, c.stream>>>(c.d_T, c.d_diis_t, c.namp, dim, s.d_coef,
                                                                         c.d_diis_state);
  }
  KCHECK(c);
  k_freeze<<<(c.ninst + 127) / 128, 128, 0, c.stream>>>(c.d_diis_state, c.ninst);
  KCHECK(c);
}

// One full iteration: RHS, update, residual, energy, DIIS.
void ccsd_iteration(Ctx& c) {
  CcsdState& s = S(c);
  if (!s.dinv_ready) {  // D and sigma are fixed for the context's life
    if (s.pk.on)
      k_inv_denom_pk<<<dim3(grid_for(s.pk.n), c.ninst), 256, 0, c.stream>>>(
          c.d_D, s.pk.d_Dinv, c.namp, s.pk.n, c.n1, s.pk.D, s.pk.vv->d_full, s.pk.oo->d_full, c.cfg.level_shift,
          c.cfg.denom_shift, c.cfg.denom_shift_n);
    else
      k_inv_denom<<<dim3(grid_for(c.namp * c.ninst)), 256, 0, c.stream>>>(c.d_D, s.d_Dinv, c.namp * c.ninst,
                                                                          c.cfg.level_shift, c.cfg.denom_shift,
                                                                          c.cfg.denom_shift_n);
    KCHECK(c);
    s.dinv_ready = true;
  }
  if (s.pk.on) {
    // R2 is needed at the canonical entries a<b, i<j only: every write into it skips the rest
    c.canon_pairs = true;
    try {
      ccsd_rhs(c);
    } catch (...) {
      c.canon_pairs = false;
      throw;
    }
    c.canon_pairs = false;
    ccsd_update_step(c, [&](double* part, int nb) {
      k_update_pk<<<dim3(nb, c.ninst), PK_THREADS, 0, c.stream>>>(
          c.d_R, s.pk.d_Dinv, c.d_T, c.d_diis_t, c.d_diis_e, c.namp, s.pk.n, c.n1, s.pk.D, s.pk.vv->d_full,
          s.pk.oo->d_full, c.cfg.diis_dim, c.d_diis_state, part, c.cfg.level_shift, s.d_dots);
      KCHECK(c);
    }, true, true, true);
    return;
  }
  ccsd_rhs(c);
  ccsd_update_step(c, [&](double* part, int nb) {
    k_update<<<dim3(nb, c.ninst), RED_THREADS, 0, c.stream>>>(c.d_R, s.d_Dinv, c.d_T, c.d_diis_t, c.d_diis_e, c.namp,
                                                              c.cfg.diis_dim, c.d_diis_state, part, c.cfg.level_shift,
                                                              s.d_dots);
    KCHECK(c);
  }, true, true);
}

// Instances frozen as converged (-1 if any instance failed with NaN/Inf).  Synchronises.
int ccsd_count_converged(Ctx& c) {
  std::vector<int> st(4 * c.ninst);
  CK(cudaMemcpyAsync(st.data(), c.d_diis_state, sizeof(int) * 4 * c.ninst, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaMemcpyAsync(c.h_stats, c.d_stats, sizeof(double) * 8 * c.ninst, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  int n = 0;
  for (int k = 0; k < c.ninst; ++k) {
    if (st[k * 4 + 2] == 2) return -1;
    if (st[k * 4 + 2] == 1) ++n;
  }
  return n;
}


// Dense <-> blocked amplitude copies: t1[i][a], t2[i][j][a][b].
__global__ void k_dense_io(cplx* __restrict__ T, int64_t off, int64_t namp, cplx* __restrict__ dense,
                           const GenTask* __restrict__ tasks, const ChunkRef* __restrict__ chunks, int rank,
                           int no, int nv, int to_dense, const int* __restrict__ occreal, int no_real) {
  const ChunkRef ch = chunks[blockIdx.x];
  const GenTask Tk = tasks[ch.task];
  const int64_t end = min(ch.start + (int64_t)4096, Tk.count);
  for (int64_t e = ch.start + threadIdx.x; e < end; e += blockDim.x) {
    int64_t r = e;
    int i[4];
    i[3] = int(r % Tk.n[3]); r /= Tk.n[3];
    i[2] = int(r % Tk.n[2]); r /= Tk.n[2];
    i[1] = int(r % Tk.n[1]);
    i[0] = int(r / Tk.n[1]);
    const int64_t p = off + Tk.base + i[0] * Tk.st[0] + i[1] * Tk.st[1] + i[2] * Tk.st[2] + i[3] * Tk.st[3];
    int64_t dp;
    if (rank == 2) {  // slots (a, i) in dims 2, 3
      const int a = Tk.g0[2] + i[2] - no, ii = occreal[Tk.g0[3] + i[3]];
      if (ii < 0) continue;  // ghost spinor: not part of the dense amplitudes
      dp = int64_t(ii) * nv + a;
    } else {  // slots (a, b, i, j)
      const int a = Tk.g0[0] + i[0] - no, b = Tk.g0[1] + i[1] - no;
      const int ii = occreal[Tk.g0[2] + i[2]], jj = occreal[Tk.g0[3] + i[3]];
      if (ii < 0 || jj < 0) continue;
      dp = ((int64_t(ii) * no_real + jj) * nv + a) * nv + b;
    }
    if (to_dense) dense[dp] = T[p];
    else T[p] = dense[dp];
  }
}

void ccsd_dense_io(Ctx& c, int inst, cplx* t1d, cplx* t2d, bool to_dense) {
  CcsdState& s = S(c);
  if (to_dense) {
    CK(cudaMemsetAsync(t1d, 0, sizeof(cplx) * c.no_real * c.nv, c.stream));
    CK(cudaMemsetAsync(t2d, 0, sizeof(cplx) * size_t(c.no_real) * c.no_real * c.nv * c.nv, c.stream));
  }
  const int64_t off = int64_t(inst) * c.namp;
  if (s.t1tasks.n_chunks) {
    k_dense_io<<<s.t1tasks.n_chunks, 256, 0, c.stream>>>(c.d_T, off, c.namp, t1d, s.t1tasks.d_tasks,
                                                         s.t1tasks.d_chunks, 2, c.no, c.nv, to_dense, c.d_occreal,
                                                         c.no_real);
    KCHECK(c);
  }
  if (s.t2tasks.n_chunks) {
    k_dense_io<<<s.t2tasks.n_chunks, 256, 0, c.stream>>>(c.d_T, off + c.n1, c.namp, t2d, s.t2tasks.d_tasks,
                                                         s.t2tasks.d_chunks, 4, c.no, c.nv, to_dense, c.d_occreal,
                                                         c.no_real);
    KCHECK(c);
  }
}

// <ab||ij> of instance inst (the scaled driver integral, held in the t2 layout) as the
// dense dst[i][j][a][b]; symmetry-forbidden entries are zero.  A context without ghost
// spinors only.
void ccsd_dense_driver_integral(Ctx& c, int inst, cplx* dst) {
  CcsdState& s = S(c);
  CK(cudaMemsetAsync(dst, 0, sizeof(cplx) * size_t(c.no_real) * c.no_real * c.nv * c.nv, c.stream));
  if (s.t2tasks.n_chunks) {
    k_dense_io<<<s.t2tasks.n_chunks, 256, 0, c.stream>>>(const_cast<cplx*>(s.Vd->d), int64_t(inst) * s.Vd->is,
                                                         s.Vd->is, dst, s.t2tasks.d_tasks, s.t2tasks.d_chunks, 4,
                                                         c.no, c.nv, 1, c.d_occreal, c.no_real);
    KCHECK(c);
  }
}

const Tensor* ccsd_driver_integral(Ctx& c) { return S(c).Vd; }

void ccsd_mark_guessed(Ctx& c) {
  zero_pair_diag(c);
  ccsd_reset_diis(c);
  ccsd_energy_of(c, c.d_T, false);
  c.guessed = true;
}
