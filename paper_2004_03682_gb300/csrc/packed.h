// Pair-packed storage of antisymmetric index pairs (the a<b, c<d, i<j packing of
// the symmetry-blocked layouts, Sec. II.C): a compound of two slots of the same
// space keeps only p<q, per pair irrep h = (Gamma_p + Gamma_q) mod G, the irrep
// pairs Gamma_p < Gamma_q as full rectangles and Gamma_p = Gamma_q as a strict
// upper triangle.  Used for the particle-particle ladder of Eq. (amplitudes),
// Z_ij^ab = 1/2 sum_cd <ab||cd> tau_ij^cd = sum_{c<d} <ab||cd> tau_ij^cd.
#pragma once
#include "engine.h"

#define PK_MAXG 32

// One two-slot compound of a blocked layout, per block g: its packed (p<q)
// enumeration, or every tuple in layout order when not packed.
struct PairTable {
  int G = 1;
  std::vector<int32_t> n, off;    // [G] entries per block, prefix into pair / full
  std::vector<int32_t> fn, foff;  // [G] full compound size per block, prefix into inv
  std::vector<int32_t> pair;      // global spinor indices (p << 16 | q) per entry
  std::vector<int32_t> full;      // full compound index (within its block) per entry
  std::vector<int32_t> inv;       // per full compound index: +(k+1) entry k as is,
                                  // -(k+1) entry k with the pair swapped, 0 for p = q
  std::vector<int32_t> swp;       // full compound index of the swapped pair (q, p) per entry
                                  // (= full when not packed)
  int32_t* d_pair = nullptr;
  int32_t* d_full = nullptr;
  int32_t* d_inv = nullptr;
  int32_t* d_swp = nullptr;
};

// Shapes passed by value to the pack / unpack / generate kernels: a packed matrix
// with blocks (rows of table R) x (cols of table C), and the full blocked matrix
// it is gathered from or scattered into.
struct PackDims {
  int G;
  int64_t blk[PK_MAXG + 1];   // packed block offsets, blk[G] = total
  int64_t fblk[PK_MAXG + 1];  // full block offsets, fblk[G] = total
  int32_t nr[PK_MAXG], nc[PK_MAXG];
  int32_t roff[PK_MAXG], coff[PK_MAXG];
  int32_t fnr[PK_MAXG], fnc[PK_MAXG];
  int32_t froff[PK_MAXG], fcoff[PK_MAXG];
};

// block of element e of a matrix with block offsets off[0..G]
__device__ __forceinline__ int find_block(const int64_t* off, int G, int64_t e) {
  int g = 0;
  while (g + 1 < G && e >= off[g + 1]) ++g;
  return g;
}

// rows = the first two slots of L (nrow must be 2), else the last two
void build_pair_table(Ctx& c, const Layout& L, bool rows, bool packed, PairTable& T);
PackDims pack_dims(const PairTable& R, const PairTable& C);

// dst[packed] = src[full]
void launch_pack_gather(Ctx& c, cplx* dst, int64_t dis, const cplx* src, int64_t sis, const PackDims& D,
                        const PairTable& R, const PairTable& C);
// dst[full] (+)= sign * src[packed], sign from the pair swaps (p = q entries untouched
// when accumulating, zero otherwise); coef = +1 or -1
void launch_pack_scatter(Ctx& c, cplx* dst, int64_t dis, const cplx* src, int64_t sis, const PackDims& D,
                         const PairTable& R, const PairTable& C, double coef, bool accumulate);
// dst[packed](p, q, r, s) = scale * V(p, q, r, s) with (p, q) from R and (r, s) from C (tensor.cu)
void launch_generate_pairs(Ctx& c, cplx* dst, int64_t is, const PackDims& D, const PairTable& R,
                           const PairTable& C);

// Packed contractions over tau pair indices (packed.cu).  packed_tau gathers tau
// (c<d, i<j) once per iteration; the others then use it:
//   packed_ladder  r2 += sum_{c<d} <ab||cd> tau_ij^cd
//   packed_xamij   X_amij = 2 sum_{e<f} <am||ef> tau_ij^ef      (= sum_ef; overwrites X)
//   packed_wmnij   W_mnij += sum_{e<f} <mn||ef> tau_ij^ef
//   packed_hh      r2 += sum_{m<n} tau_mn^ab W_mnij             (W complete)
// The pair-packed space of the doubles layout L (rows a<b, cols i<j): its tables and
// dims, built once per context (the update / DIIS / energy of the amplitude vector
// act on these unique entries of the antisymmetric t2).
const PackDims& packed_t2_space(Ctx& c, const Layout& L, const PairTable** vv, const PairTable** oo);
void packed_tau(Ctx& c, const Tensor& tau);
void packed_ladder(Ctx& c, Tensor& r2);
void packed_xamij(Ctx& c, Tensor& X);
void packed_wmnij(Ctx& c, Tensor& W);
void packed_hh(Ctx& c, const Tensor& W, Tensor& r2);
void packed_release(Ctx& c);
