// (0h,1p) and (0h,2p) Fock-space sector drivers.
#pragma once
#include "engine.h"

void fs_release(Ctx& c);
void fs_step(Ctx& c, const double* Dfs, const int8_t* role, const cplx* XV, const int64_t* mir, int64_t n_mir);
exp_status fs_entry(Ctx& c, int inst, double* heff, double* eig_re, double* eig_im, int* n_iter);
// the (0h,2p) sector (runs the (0h,1p) sector first when needed)
exp_status fs2_entry(Ctx& c, int inst, double* heff, double* eig_re, double* eig_im, int* n_iter);
