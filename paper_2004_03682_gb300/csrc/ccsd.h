// CCSD (0h,0p) driver entry points used by the C ABI.
#pragma once
#include <functional>

#include "engine.h"

// intruder-state dynamic shift of an energy denominator (exp_config.denom_shift):
// D~ = D - s (s / (s + |D|))^n; s = 0 leaves D unchanged
__host__ __device__ __forceinline__ double dyn_shift(double D, double s, int n) {
  if (!(s > 0.0)) return D;
  const double r = s / (s + fabs(D));
  double p = s;
  for (int k = 0; k < n; ++k) p *= r;
  return D - p;
}

Layout L4(Ctx& c, int s0, int g0, int s1, int g1, int s2, int g2, int s3, int g3, int nrow);
Layout L2(Ctx& c, int s0, int g0, int s1, int g1);
void ccsd_setup(Ctx& c);
void ccsd_release(Ctx& c);
void ccsd_init_integrals(Ctx& c, const double* h_mult);
void ccsd_guess(Ctx& c);
void ccsd_reset_diis(Ctx& c);
void ccsd_energy_of(Ctx& c, const cplx* T, bool skip_frozen);
void ccsd_rhs(Ctx& c);
void ccsd_iteration(Ctx& c);
void ccsd_dense_io(Ctx& c, int inst, cplx* t1_dense, cplx* t2_dense, bool to_dense);
// dots_done: `upd` also formed the DIIS inner products of the new error vector;
// packed: the DIIS vectors are the pair-packed amplitude vector (t1, t2 over a<b, i<j)
void ccsd_update_step(Ctx& c, const std::function<void(double*, int)>& upd, bool energy, bool dots_done = false,
                      bool packed = false);
int ccsd_count_converged(Ctx& c);
const Tensor* ccsd_driver_integral(Ctx& c);
// <ab||ij> of instance inst as the dense [i][j][a][b] (zero where symmetry forbids);
// contexts without ghost spinors
void ccsd_dense_driver_integral(Ctx& c, int inst, cplx* dst);
void ccsd_mark_guessed(Ctx& c);
// the (T) correction of instance inst (triples.cu)
void ccsd_t(Ctx& c, int inst, int block, exp_t3_info* info, double* per_triple);
