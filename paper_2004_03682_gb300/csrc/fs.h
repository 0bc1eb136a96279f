// (0h,1p) Fock-space sector driver.
#pragma once
#include "engine.h"

void fs_release(Ctx& c);
void fs_step(Ctx& c, const double* Dfs, const int8_t* role, const cplx* XV);
exp_status fs_entry(Ctx& c, int inst, double* heff, double* eig_re, double* eig_im, int* n_iter);
