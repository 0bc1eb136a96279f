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

