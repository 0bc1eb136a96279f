// Split-precision emulation of complex-FP64 GEMM on the BF16 tensor cores
// (tcgen05), used for the large CCSD contractions.
#pragma once
#include "engine.h"

// largest K of an emulated product (K' = 2K padded and every slice offset stay in range)
#define EMU_MAX_K (1 << 26)
// the particle-particle ladder and ring products (exp_config.n_slices_major), by call site
bool emu_major_site(const std::string& site);

bool emu_wanted(Ctx& c, const GemmPlan& g, const std::string& site);
// b_shareable: B is a lasting tensor, so a later product reading the same tensor in
// the same layout may reuse this plan's B slices
// site: the contraction's call site (selects n_slices or n_slices_major)
EmuPlan* emu_plan(Ctx& c, const GemmPlan& g, const Tensor* A, const Tensor* B, bool a_const,
                  bool b_const, bool b_shareable, const std::string& site);
// gemm_only: launch only the tensor-core kernel on the slices of the previous run
// (timing); the split-K reduction and the slicing passes are skipped
void emu_run(Ctx& c, EmuPlan* p, const GemmPlan& g, const cplx* A, const cplx* B, cplx* C,
             int64_t ais, int64_t bis, int64_t cis, cplx alpha, bool beta, bool gemm_only = false);
void emu_release(Ctx& c);

// Operand sets for grouped products whose operand pairing is chosen at run time (the
// products of the (T) correction).  The members of a set are sliced together; a
// product pairs an A member (rows x K, row-major) with a B member (K x cols,
// row-major) of the same K and writes C (rows x cols, row-major) = alpha A B, or the
// sum of up to three such pairs (segments) with equal rows and cols: C = alpha
// sum_w A_w B_w, accumulated exactly over the concatenated K (a product whose
// segments all have K = 0 leaves its C as it is).  Members of one
// exponent group (same rows / cols) share their row (A) or column (B) exponents, the
// maximum over the group; the segments of one product must come from one A group and
// one B group.  The products of one call share one launch; each product needs a total
// K short enough for one exact int64 accumulation (K' up to 2^(13 - 7 (S - 6)) KC
// terms: far above (T)'s).
struct EmuSet;
struct EmuSetMat {
  int64_t src;  // element offset of the member in the source array
  int rows;     // A: rows; B: columns
  int K;
  int ex_group = -1;  // members with the same group >= 0 share one exponent vector
};
struct EmuSetProd {
  int a, b;       // member indices in the A and the B set (first segment)
  int64_t c_off;  // element offset of the product's C in the output array
  int a1 = -1, b1 = -1, a2 = -1, b2 = -1;  // second and third segments (-1: none)
};
EmuSet* emu_set_new(Ctx& c, int S, bool b_side);
// lay out the members (growing the set's device buffers when needed), then scan
// their exponents and write their slice tiles from src
void emu_set_slice(Ctx& c, EmuSet* s, const std::vector<EmuSetMat>& mats, const cplx* src);
void emu_set_multiply(Ctx& c, const EmuSet* A, const EmuSet* B, const std::vector<EmuSetProd>& prods, cplx* C,
                      cplx alpha);
void emu_set_free(Ctx& c, EmuSet* s);
